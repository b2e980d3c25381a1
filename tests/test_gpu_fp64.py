"""FP64 parity of the CUDA path against the CPU oracle, through the C ABI.

Bar: max-norm relative error <= 1e-11 (FP64 mode), element by element, on
the same seeded inputs.  Sizes span several 16-bead tiles and ragged tails;
the N = 8000 theta solution is checked on sampled 3x3 blocks.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1203_6208_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-11


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


def gpu_D(bnd, p, R, precision="fp64", **kw):
    plan = bnd.Plan(p, precision, **kw)
    Rg = torch.tensor(np.ascontiguousarray(R), device="cuda")
    D = plan.alloc_D()
    plan.build_D(Rg, D)
    torch.cuda.synchronize()
    return plan, Rg, D


CASES = {
    "c1_ev": lambda: inputs.preset("c1")[0],
    "ragged_n37": lambda: inputs.SystemConfig(n_chains=1, nb=37, c_over_cstar=3.0, seed=7),
    "alpha_x0.6": lambda: inputs.SystemConfig(n_chains=5, nb=10, c_over_cstar=2.0,
                                              alpha_factor=0.6, seed=8),
    "alpha_x2": lambda: inputs.SystemConfig(n_chains=5, nb=10, c_over_cstar=2.0,
                                            alpha_factor=2.0, seed=9),
    "fene_n1000_c4": lambda: inputs.SystemConfig(n_chains=100, nb=10, c_over_cstar=4.0,
                                                 spring=1, fene_b=50.0, seed=1002),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_build_D_parity(bnd, case):
    cfg = CASES[case]()
    p = cfg.params()
    R = inputs.make_chains(cfg)
    plan, Rg, D = gpu_D(bnd, p, R)
    Dg = plan.D_view(D).cpu().numpy()
    Dr = oracle.build_D(p, R)
    assert relerr(Dg, Dr) <= TOL
    assert np.array_equal(Dg, Dg.T)            # mirrored writes: exactly symmetric


def test_build_D_close_overlap_and_coincident(bnd):
    """Images far inside 2a (series branch) and two coincident beads."""
    cfg = inputs.SystemConfig(n_chains=2, nb=10, c_over_cstar=1.0, seed=21)
    p = cfg.params()
    R = inputs.make_chains(cfg)
    a = p["a"]
    e = np.array([0.6, -0.48, 0.64])
    R[3] = R[2] + 1e-3 * a * e
    R[7] = R[6] + 0.05 * a * e
    R[12] = R[4] + 0.7 * a * e + p["L"] * np.array([1.0, -2.0, 0.0])  # overlap via an image
    R[15] = R[14]                                                     # coincident
    plan, Rg, D = gpu_D(bnd, p, R)
    Dg = plan.D_view(D).cpu().numpy()
    Dr = oracle.build_D(p, R)
    assert relerr(Dg, Dr) <= TOL
    assert np.allclose(Dg[45:48, 42:45], Dg[42:45, 42:45], atol=1e-14)


def test_build_D_n8000_sampled_blocks(bnd):
    """The 24000 x 24000 theta-solution matrix: 300 random blocks, the full
    block rows of beads 0 and 7999, and the symmetric mirror."""
    cfg, _ = inputs.preset("c4")
    p = cfg.params()
    R = inputs.make_chains(cfg)
    plan, Rg, D = gpu_D(bnd, p, R)
    Dv = plan.D_view(D)
    rng = np.random.default_rng(5)
    pairs = [(int(a), int(b)) for a, b in rng.integers(0, cfg.n, size=(300, 2))]
    pairs += [(i, i) for i in (0, 4000, 7999)]
    # add close pairs (overlap branch)
    d = R[None, :200] - R[:200, None]
    d -= p["L"] * np.round(d / p["L"])
    close = np.argwhere((np.linalg.norm(d, axis=-1) < 2 * p["a"]) & ~np.eye(200, dtype=bool))
    pairs += [tuple(map(int, c)) for c in close[:20]]
    worst = 0.0
    for nu, mu in pairs:
        Bg = Dv[3 * nu:3 * nu + 3, 3 * mu:3 * mu + 3].cpu().numpy()
        Br = oracle.D_block(p, R, nu, mu)
        worst = max(worst, float(np.max(np.abs(Bg - Br))))
    assert worst <= TOL * 0.9
    rows = Dv[0:3].cpu().numpy()
    ref = oracle.build_D_rows(p, R, 0, 1)
    assert relerr(rows, ref) <= TOL
    rows = Dv[3 * 7999:].cpu().numpy()
    ref = oracle.build_D_rows(p, R, 7999, 8000)
    assert relerr(rows, ref) <= TOL
    blk = Dv[3000:3300, 21000:21300]
    assert torch.equal(blk, Dv[21000:21300, 3000:3300].T)


@pytest.mark.parametrize("m", [1, 2, 3, 16, 17])
def test_apply_parity(bnd, m):
    cfg = inputs.SystemConfig(n_chains=30, nb=10, c_over_cstar=2.0, seed=31)
    p = cfg.params()
    R = inputs.make_chains(cfg)
    plan, Rg, D = gpu_D(bnd, p, R, max_rhs=32)
    Dr = oracle.build_D(p, R)
    X = inputs.make_wiener(3 * cfg.n, m, 1.0, 99)
    Xg = torch.tensor(X, device="cuda")
    Y = torch.empty_like(Xg)
    plan.apply(D, Xg, Y)
    assert relerr(Y.cpu().numpy(), oracle.apply_D(Dr, X)) <= TOL


def test_forces_parity(bnd):
    for cfg in (inputs.preset("c1")[0],
                inputs.SystemConfig(n_chains=40, nb=10, c_over_cstar=2.0, spring=1,
                                    fene_b=50.0, ev_on=1, seed=41)):
        p = cfg.params()
        R = inputs.make_chains(cfg)
        plan = bnd.Plan(p, "fp64", max_rhs=1)
        Rg = torch.tensor(R, device="cuda")
        F = torch.empty(3 * cfg.n, dtype=torch.float64, device="cuda")
        nbad = torch.zeros(1, dtype=torch.int32, device="cuda")
        plan.forces(Rg, F, nbad)
        Fr, bad = oracle.forces(p, R)
        assert int(nbad.item()) == bad == 0
        assert relerr(F.cpu().numpy(), Fr) <= TOL


def test_fene_overstretch_counted(bnd):
    cfg = inputs.SystemConfig(n_chains=2, nb=5, c_over_cstar=1.0, spring=1, fene_b=4.0)
    p = cfg.params()
    R = inputs.make_chains(cfg)
    R[3] = R[2] + np.array([2.5, 0.0, 0.0])
    plan = bnd.Plan(p, "fp64", max_rhs=1)
    F = torch.empty(30, dtype=torch.float64, device="cuda")
    nbad = torch.zeros(1, dtype=torch.int32, device="cuda")
    plan.forces(torch.tensor(R, device="cuda"), F, nbad)
    _, bad = oracle.forces(p, R)
    assert bad >= 1 and int(nbad.item()) == bad


@pytest.mark.parametrize("m,nch", [(1, 20), (4, 40), (16, 12)])
def test_chebyshev_parity(bnd, m, nch):
    cfg = inputs.SystemConfig(n_chains=20, nb=10, c_over_cstar=2.0, seed=51)
    p = cfg.params()
    R = inputs.make_chains(cfg)
    plan, Rg, D = gpu_D(bnd, p, R, max_rhs=32, max_cheb=64)
    Dr = oracle.build_D(p, R)
    lmin, lmax = oracle.exact_eigs(Dr)
    dmin, dmax = 0.9 * lmin, 1.05 * lmax
    dW = inputs.make_wiener(3 * cfg.n, m, p["dt"], 52)
    bounds = torch.tensor([dmin, dmax], dtype=torch.float64, device="cuda")
    dWg = torch.tensor(dW, device="cuda")
    dS = torch.empty_like(dWg)
    Ef = torch.empty(m, dtype=torch.float64, device="cuda")
    plan.chebyshev(D, bounds, nch, dWg, dS, Ef)
    dS_r, Ef_r = oracle.cheb_sqrt(Dr, dmin, dmax, nch, dW)
    assert relerr(dS.cpu().numpy(), dS_r) <= TOL
    assert np.allclose(Ef.cpu().numpy(), Ef_r, rtol=1e-6, atol=1e-12)


def test_eig_bounds_bracket_spectrum(bnd):
    cfg, _ = inputs.preset("c1")
    p = cfg.params()
    R = inputs.make_chains(cfg)
    plan, Rg, D = gpu_D(bnd, p, R)
    Dr = oracle.build_D(p, R)
    lmin, lmax = oracle.exact_eigs(Dr)
    bounds = torch.empty(2, dtype=torch.float64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    plan.eig_bounds(D, 60, 0.02, 0.5, bounds, status)
    dmin, dmax = bounds.cpu().numpy()
    assert int(status.item()) == 0
    assert lmax <= dmax <= 1.03 * lmax
    assert 0.0 < dmin <= lmin


def test_eig_bounds_tiny_system_breakdown(bnd):
    """3N smaller than the requested Lanczos steps: the Krylov space becomes
    invariant and the bounds still bracket the spectrum."""
    cfg = inputs.SystemConfig(n_chains=1, nb=4, c_over_cstar=1.0, seed=3)
    p = cfg.params()
    R = inputs.make_chains(cfg)
    plan, Rg, D = gpu_D(bnd, p, R)
    lmin, lmax = oracle.exact_eigs(oracle.build_D(p, R))
    bounds = torch.empty(2, dtype=torch.float64, device="cuda")
    plan.eig_bounds(D, 40, 0.01, 0.9, bounds)
    dmin, dmax = bounds.cpu().numpy()
    assert lmax <= dmax and 0 < dmin <= lmin


def test_step_parity_and_stats(bnd):
    cfg, extra = inputs.preset("c1")
    p = cfg.params()
    R = inputs.make_chains(cfg)
    dW = inputs.make_wiener(3 * cfg.n, 2, p["dt"], cfg.seed + 1)
    plan = bnd.Plan(p, "fp64", max_rhs=2, max_cheb=64)
    Rg = torch.tensor(R, device="cuda")
    D = plan.alloc_D()
    DF = torch.empty(3 * cfg.n, dtype=torch.float64, device="cuda")
    dS = torch.empty(2, 3 * cfg.n, dtype=torch.float64, device="cuda")
    stats = bnd.new_stats()
    plan.step(Rg, D, torch.tensor(dW, device="cuda"), m=2, n_cheb=30, lanczos_iters=60,
              bound_safety=0.02, dmin_fraction=0.5, DF=DF, dS=dS, stats=stats)
    st = bnd.read_stats(stats)
    assert st["status"] == 0 and st["accepted"] == 1 and st["n_cheb"] == 30
    R_ref, code, DF_r, dS_r, Ef_r = oracle.step(p, R, dW, st["d_min"], st["d_max"], 30)
    assert code == 0
    assert relerr(DF.cpu().numpy(), DF_r) <= TOL
    assert relerr(dS.cpu().numpy(), dS_r) <= TOL
    assert relerr(Rg.cpu().numpy(), R_ref) <= TOL
    assert abs(st["ef_max"] - float(np.max(Ef_r))) <= 1e-6 * max(1e-12, float(np.max(Ef_r)))
    lmin, lmax = oracle.exact_eigs(oracle.build_D(p, R))
    assert st["d_max"] >= lmax and 0 < st["d_min"] <= lmin


def test_step_fene_rejection(bnd):
    cfg = inputs.SystemConfig(n_chains=2, nb=4, c_over_cstar=1.0, spring=1, fene_b=4.0,
                              dt=0.01)
    p = cfg.params()
    R = np.array([[0, 0, 0], [1.9, 0, 0], [2.5, 0.3, 0], [3.0, 1.0, 0.5],
                  [4, 4, 4], [4.5, 4, 4], [5, 4.5, 4], [5.5, 4.6, 4.2]], dtype=float)
    dW = np.zeros((1, 24))
    dW[0, 4] = 4.0
    plan = bnd.Plan(p, "fp64", max_rhs=1, max_cheb=32)
    Rg = torch.tensor(R, device="cuda")
    D = plan.alloc_D()
    stats = bnd.new_stats()
    plan.step(Rg, D, torch.tensor(dW, device="cuda"), m=1, n_cheb=20, lanczos_iters=20,
              dmin_fraction=0.5, stats=stats)
    st = bnd.read_stats(stats)
    _, code, *_ = oracle.step(p, R, dW, st["d_min"], st["d_max"], 20)
    assert code > 0 and st["accepted"] == 0 and st["n_overstretched"] == code
    assert st["status"] == 5
    assert np.array_equal(Rg.cpu().numpy(), R)


def test_wiener_matches_oracle_philox(bnd):
    cfg, _ = inputs.preset("c1")
    plan = bnd.Plan(cfg.params(), "fp64", max_rhs=1)
    out = torch.empty(3001, dtype=torch.float64, device="cuda")
    plan.wiener(1234567, 89, out)
    ref = oracle.wiener_philox(1234567, 89, 3001, cfg.params()["dt"])
    assert relerr(out.cpu().numpy(), ref) <= 1e-14


def test_step_device_wiener_matches_explicit(bnd):
    cfg, _ = inputs.preset("c1")
    p = cfg.params()
    R = inputs.make_chains(cfg)
    plan = bnd.Plan(p, "fp64", max_rhs=1, max_cheb=32)
    D = plan.alloc_D()
    R1 = torch.tensor(R, device="cuda")
    R2 = torch.tensor(R, device="cuda")
    plan.step(R1, D, None, m=1, n_cheb=16, lanczos_iters=30, seed=77, step_index=5)
    w = torch.empty(3 * cfg.n, dtype=torch.float64, device="cuda")
    plan.wiener(77, 5, w)
    plan.step(R2, D, w.view(1, -1), m=1, n_cheb=16, lanczos_iters=30)
    assert torch.allclose(R1, R2, rtol=0, atol=1e-12)


def test_invalid_arguments_raise(bnd):
    cfg, _ = inputs.preset("c1")
    p = cfg.params()
    with pytest.raises(bnd.BDError) as e:
        bnd.Plan(dict(p, n=101), "fp64")
    assert e.value.status == 1
    plan = bnd.Plan(p, "fp64", max_rhs=2)
    D = plan.alloc_D()
    X = torch.zeros(3, 3 * cfg.n, dtype=torch.float64, device="cuda")
    with pytest.raises(bnd.BDError):
        plan.apply(D, X, torch.empty_like(X))
    with pytest.raises(bnd.BDError):
        plan.build_D(torch.zeros(cfg.n, 3, dtype=torch.float64, device="cuda"), D[8:])


@pytest.mark.parametrize("prec,tol", [("fp64", TOL), ("mixed_f16", 2e-6)])
def test_build_D_periodic_images_of_beads(bnd, prec, tol):
    """Shifting each bead by its own integer multiple of L (unwrapped
    trajectories) leaves D unchanged: the wrap into the box and the
    separation of close pairs across the boundary keep full precision."""
    cfg = inputs.SystemConfig(n_chains=6, nb=10, c_over_cstar=3.0, seed=33)
    p = cfg.params()
    R = inputs.make_chains(cfg)
    shifts = np.random.default_rng(34).integers(-40, 40, size=R.shape) * p["L"]
    plan = bnd.Plan(p, prec, max_rhs=1)
    Dr = oracle.build_D(p, R)
    for Rx in (R, R + shifts):
        Rg = torch.tensor(Rx, device="cuda")
        D = plan.alloc_D()
        plan.build_D(Rg, D)
        Dg = plan.D_view(D).double().cpu().numpy()
        assert relerr(Dg, Dr) <= tol
