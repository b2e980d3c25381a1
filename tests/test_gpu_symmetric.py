"""The symmetric tensor-core product (launch shape 3: only the 128 x 128 tiles
on and above the diagonal of the 16-bit D are read, each serving D_IJ X_J
and D_IJ^T X_I, the second with the staged tile read MN-major) against the
FP64 oracle and against the stream-K product over all of D16 (shape 1).

Both shapes form the same 16-bit-D product with FP32 accumulation in another
order, so they agree to FP32 rounding of the sums.  The RPY tensor is long
ranged: sum_j |D_ij x_j| is far above |y_i|, and the rounding of 3N-term FP32
sums grows with 3N (measured between the shapes: under 1e-5 of max|Y| at
3N = 9000, 3.3e-5 at 3N = 24 000).  A Chebyshev series also re-rounds every
V_p to 16 bits for the next product, where an FP32 order difference can flip
a half-precision rounding (2^-12 of that element) and carry on (1.7e-5 over
40 terms at 3N = 900).  Between the shapes the bar is 1e-4 of max|Y|, ten
times or more inside the oracle bars.  Against the oracle the mixed-mode bars hold (2e-3 for a product, 1e-3
for Chebyshev, 1e-5 for the refined drift).  Sizes: one band of 2 tiles (50 beads), a ragged band and ragged
last tile (700 and 77 beads), several bands (3000 beads), and the N = 8000
benchmark system on sampled oracle rows."""
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


def mixed(bnd, n_chains, nb, seed, prec="mixed_f16", c=2.0, **kw):
    cfg = inputs.SystemConfig(n_chains=n_chains, nb=nb, c_over_cstar=c, seed=seed)
    p = cfg.params()
    R = inputs.make_chains(cfg)
    plan = bnd.Plan(p, prec, **kw)
    Rg = torch.tensor(R, device="cuda")
    D = plan.alloc_D()
    plan.build_D(Rg, D)
    torch.cuda.synchronize()
    return cfg, p, R, plan, Rg, D


def both_shapes(plan, D, X):
    Xg = torch.tensor(X, device="cuda")
    out = []
    for shape in (1, 3):
        plan.set_shape(shape)
        Y = torch.empty_like(Xg)
        plan.apply(D, Xg, Y)
        out.append(Y.cpu().numpy())
    return out


@pytest.mark.parametrize("n_chains,nb,m,prec", [(5, 10, 16, "mixed_f16"), (5, 10, 17, "mixed_f16"),
                                                (7, 11, 5, "mixed_f16"), (70, 10, 16, "mixed_f16"),
                                                (70, 10, 17, "mixed_f16"), (70, 10, 32, "mixed_f16"),
                                                (70, 10, 17, "mixed_bf16")])
def test_symmetric_apply_vs_oracle(bnd, n_chains, nb, m, prec):
    cfg, p, R, plan, Rg, D = mixed(bnd, n_chains, nb, 81, prec, max_rhs=32)
    X = inputs.make_wiener(3 * cfg.n, m, 1.0, 82)
    Y1, Y3 = both_shapes(plan, D, X)
    assert relerr(Y3, Y1) <= 1e-4
    ref = oracle.apply_D(oracle.build_D(p, R), X)
    tol = 2e-3 if prec == "mixed_f16" else 1e-2
    assert relerr(Y3, ref) <= tol
    for j in range(m):
        assert relerr(Y3[j], ref[j]) <= tol


def test_symmetric_many_bands(bnd):
    """3000 beads: 71 tiles per side in 9 bands (the last of 7 rows), 2556
    tiles shared by up to 152 CTAs; against the stream-K shape and against
    sampled oracle rows."""
    cfg, p, R, plan, Rg, D = mixed(bnd, 300, 10, 83, max_rhs=17)
    X = inputs.make_wiener(3 * cfg.n, 17, 1.0, 84)
    Y1, Y3 = both_shapes(plan, D, X)
    assert relerr(Y3, Y1) <= 1e-4
    scale = np.max(np.abs(Y3))
    for b in (0, 1, 1024, 2047, 2999):
        rows = oracle.build_D_rows(p, R, b, b + 1)
        ref = rows @ X.T                      # 3 x m
        assert np.max(np.abs(Y3[:, 3 * b:3 * b + 3].T - ref)) <= 2e-3 * scale


def test_symmetric_chebyshev(bnd):
    cfg, p, R, plan, Rg, D = mixed(bnd, 30, 10, 85, max_rhs=16, max_cheb=64)
    Dr = oracle.build_D(p, R)
    lmin, lmax = oracle.exact_eigs(Dr)
    dmin, dmax = 0.9 * lmin, 1.05 * lmax
    m, nch = 16, 40
    dW = inputs.make_wiener(3 * cfg.n, m, p["dt"], 86)
    bounds = torch.tensor([dmin, dmax], dtype=torch.float64, device="cuda")
    dWg = torch.tensor(dW, device="cuda")
    out = []
    for shape in (1, 3):
        plan.set_shape(shape)
        dS = torch.empty_like(dWg)
        plan.chebyshev(D, bounds, nch, dWg, dS)
        out.append(dS.cpu().numpy())
    assert relerr(out[1], out[0]) <= 1e-4
    dS_r, _ = oracle.cheb_sqrt(Dr, dmin, dmax, nch, dW)
    assert relerr(out[1], dS_r) <= 1e-3


def test_symmetric_lagged_steps(bnd):
    """Two steps with lagged Lanczos bounds (the Lanczos vector rides as an
    extra product column: the epilogue's w = D q_j and dot partials) in both
    shapes: the same bounds, drift and displacements to FP32 rounding; the
    second step against the oracle step at its own bounds."""
    cfg, _ = inputs.preset("c1")
    p = cfg.params()
    R = inputs.make_chains(cfg)
    m, nch = 4, 30
    res = []
    for shape in (1, 3):
        plan = bnd.Plan(p, "mixed_f16", max_rhs=m, max_cheb=64)
        plan.set_shape(shape)
        Rg = torch.tensor(R, device="cuda")
        D = plan.alloc_D()
        DF = torch.empty(3 * cfg.n, dtype=torch.float64, device="cuda")
        dS = torch.empty(m, 3 * cfg.n, dtype=torch.float64, device="cuda")
        stats = bnd.new_stats()
        for k in range(2):
            R_before = Rg.cpu().numpy().copy()
            dW = inputs.make_wiener(3 * cfg.n, m, p["dt"], 90 + k)
            plan.step(Rg, D, torch.tensor(dW, device="cuda"), m=m, n_cheb=nch, lanczos_iters=40,
                      bounds_mode=1, DF=DF, dS=dS, stats=stats, step_index=k)
            st = bnd.read_stats(stats)
            assert st["status"] == 0 and st["accepted"] == 1
        res.append((st, DF.cpu().numpy(), dS.cpu().numpy(), R_before, dW))
        plan.close()
    (s1, DF1, dS1, Rb1, dW), (s3, DF3, dS3, Rb3, _) = res
    # the bottom Ritz value of a few dozen lagged Lanczos steps has not
    # converged (clustered small eigenvalues) and moves with the summation
    # order of the products (measured 2.4e-4 relative); the top one converges
    assert abs(s3["d_min"] - s1["d_min"]) <= 2e-3 * s1["d_min"]
    assert abs(s3["d_max"] - s1["d_max"]) <= 1e-4 * s1["d_max"]
    assert relerr(DF3, DF1) <= 1e-5
    # each shape's Brownian term is taken on its own Chebyshev interval, so the
    # two agree only to the mixed-mode bar; each matches the oracle at its bounds
    assert relerr(dS3, dS1) <= 1e-3
    for st, DFg, dSg, Rb in ((s1, DF1, dS1, Rb1), (s3, DF3, dS3, Rb3)):
        R_ref, code, DF_r, dS_r, _ = oracle.step(p, Rb.reshape(R.shape), dW, st["d_min"], st["d_max"], nch)
        assert code == 0
        assert relerr(DFg, DF_r) <= 1e-5
        assert relerr(dSg, dS_r) <= 1e-3


def test_symmetric_n8000_sampled_rows(bnd):
    """The N = 8000 benchmark system (188 tiles per side, 17 766 tiles on
    and above the diagonal over 152 CTAs): rows of the symmetric product
    against oracle rows of D times the same X."""
    cfg, _ = inputs.preset("c4")
    p = cfg.params()
    R = inputs.make_chains(cfg)
    plan = bnd.Plan(p, "mixed_f16", max_rhs=17)
    Rg = torch.tensor(R, device="cuda")
    D = plan.alloc_D()
    plan.build_D(Rg, D)
    X = inputs.make_wiener(3 * cfg.n, 17, 1.0, 87)
    Y1, Y3 = both_shapes(plan, D, X)
    assert relerr(Y3, Y1) <= 1e-4
    scale = np.max(np.abs(Y3))
    for b in (0, 2345, 4095, 7999):
        rows = oracle.build_D_rows(p, R, b, b + 1)
        assert np.max(np.abs(Y3[:, 3 * b:3 * b + 3].T - rows @ X.T)) <= 2e-3 * scale


def test_step_capture_replay_matches_direct(bnd):
    """bd_step_capture / bd_step_replay: one lagged mixed step recorded as a
    CUDA graph replays the same kernels in the same order as bd_step with the
    device step counter, so three replays after one direct step land on the
    same positions, bit for bit, as four direct steps; adaptive N_Ch and an
    empty replay are refused."""
    cfg, _ = inputs.preset("c1")
    p = cfg.params()
    R0 = inputs.make_chains(cfg)
    kw = dict(m=4, n_cheb=30, lanczos_iters=40, bounds_mode=1, flags=bnd.BD_STEP_DEVICE_COUNTER)
    out = []
    for graph in (False, True):
        plan = bnd.Plan(p, "mixed_f16", max_rhs=4, max_cheb=64)
        plan.set_shape(bnd.BD_SHAPE_SYMMETRIC)
        R = torch.tensor(R0.reshape(-1), device="cuda")
        D = plan.alloc_D()
        stats = bnd.new_stats()
        plan.set_step_counter(100)
        plan.step(R, D, None, stats=stats, **kw)
        if graph:
            with pytest.raises(bnd.BDError):
                plan.step_replay()
            with pytest.raises(bnd.BDError):
                plan.step_capture(R, D, m=4, n_cheb=0, bounds_mode=1, stats=stats)
            plan.step_capture(R, D, stats=stats, **kw)
            for _ in range(3):
                plan.step_replay()
        else:
            for _ in range(3):
                plan.step(R, D, None, stats=stats, **kw)
        torch.cuda.synchronize()
        st = bnd.read_stats(stats)
        assert st["status"] == 0 and st["accepted"] == 1
        out.append(R.cpu().numpy())
        plan.close()
    assert np.array_equal(out[0], out[1])
    assert np.max(np.abs(out[0] - R0.reshape(-1))) > 0
