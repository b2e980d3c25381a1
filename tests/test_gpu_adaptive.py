"""Adaptive number of Chebyshev terms (Sec. IV): the GPU's moment-based
choice of N_Ch against the oracle's loop over full series, on the same
bounds and Wiener block.

Checks: the N_Ch chosen equals the oracle's (the tolerance is placed between
a record low of the oracle's E_f and every earlier E_f -- E_f is not
monotone in N -- so the decision is not a rounding tie);
dS at that N_Ch within 1e-11 of the oracle (FP64); a loose tolerance stops at
Eq. (nint); an unreachable one reports BD_ERR_CHEB_NOCONV with max_cheb
terms; bd_step with n_cheb = 0 on the FENE + EV system (N = 1000) reports
the oracle's N_Ch for its own bounds and moves R like the oracle step; the
mixed plan's choice stays within one term of the oracle's.
"""
import math

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


def system(n_chains=12, nb=10, seed=71):
    cfg = inputs.SystemConfig(n_chains=n_chains, nb=nb, c_over_cstar=2.0, seed=seed)
    p = cfg.params()
    R = inputs.make_chains(cfg)
    return cfg, p, R


def tol_for_record(D, dmin, dmax, dW, n0, n_from, n_cap):
    """E_f is not monotone in N_Ch: find the first N >= n_from whose E_f is
    below every E_f(N0..N-1) by a clear margin, and a tolerance between the
    two, so the oracle decision is N with no rounding tie."""
    best = float("inf")
    for n in range(n0, n_cap):
        _, e = oracle.cheb_sqrt(D, dmin, dmax, n, dW)
        e = float(np.max(e))
        if n >= n_from and e < 0.8 * best:
            return n, math.sqrt(e * best)
        best = min(best, e)
    raise AssertionError("no record low of E_f below the cap")


@pytest.mark.parametrize("m", [1, 3])
def test_adaptive_matches_oracle_fp64(bnd, m):
    cfg, p, R = system()
    D = oracle.build_D(p, R)
    lmin, lmax = oracle.exact_eigs(D)
    dmin, dmax = 0.9 * lmin, 1.1 * lmax
    dW = inputs.make_wiener(D.shape[0], m, p["dt"], 72)
    n0 = oracle.nch_initial(dmin, dmax)
    n_t, tol = tol_for_record(D, dmin, dmax, dW, n0, n0 + 4, 120)
    dS_r, Ef_r, n_r, ok_r = oracle.cheb_sqrt_adaptive(D, dmin, dmax, dW, tol, 120)
    assert ok_r and n_r == n_t
    plan = bnd.Plan(p, "fp64", max_rhs=m, max_cheb=120)
    Dg = plan.alloc_D()
    plan.build_D(torch.tensor(R, device="cuda"), Dg)
    bounds = torch.tensor([dmin, dmax], dtype=torch.float64, device="cuda")
    dWg = torch.tensor(dW, device="cuda")
    dS = torch.empty_like(dWg)
    Ef = torch.empty(m, dtype=torch.float64, device="cuda")
    n, ok = plan.chebyshev_adaptive(Dg, bounds, tol, dWg, dS, Ef)
    assert ok and n == n_r
    assert relerr(dS.cpu().numpy(), dS_r) <= 1e-11
    assert relerr(Ef.cpu().numpy(), Ef_r) <= 1e-6
    # the same N_Ch through the fixed series gives the same dS
    dS2 = torch.empty_like(dWg)
    plan.chebyshev(Dg, bounds, n, dWg, dS2)
    assert relerr(dS.cpu().numpy(), dS2.cpu().numpy()) <= 1e-12


def test_adaptive_loose_and_unreachable(bnd):
    cfg, p, R = system(n_chains=6, seed=73)
    D = oracle.build_D(p, R)
    lmin, lmax = oracle.exact_eigs(D)
    dmin, dmax = 0.9 * lmin, 1.1 * lmax
    dW = inputs.make_wiener(D.shape[0], 1, p["dt"], 74)
    n0 = oracle.nch_initial(dmin, dmax)
    plan = bnd.Plan(p, "fp64", max_rhs=1, max_cheb=n0 + 4)
    Dg = plan.alloc_D()
    plan.build_D(torch.tensor(R, device="cuda"), Dg)
    bounds = torch.tensor([dmin, dmax], dtype=torch.float64, device="cuda")
    dWg = torch.tensor(dW, device="cuda")
    dS = torch.empty_like(dWg)
    n, ok = plan.chebyshev_adaptive(Dg, bounds, 10.0, dWg, dS)
    assert ok and n == n0
    n, ok = plan.chebyshev_adaptive(Dg, bounds, 1e-300, dWg, dS)
    assert not ok and n == n0 + 4
    dS_r, _ = oracle.cheb_sqrt(D, dmin, dmax, n0 + 4, dW)
    assert relerr(dS.cpu().numpy(), dS_r) <= 1e-11


def test_step_adaptive_fene_ev(bnd):
    """bd_step with n_cheb = 0 on 100 FENE chains x 10 beads with EV."""
    cfg, extra = inputs.preset("c2")
    p = cfg.params()
    R = inputs.make_chains(cfg)
    tol = extra["tol"]
    dW = inputs.make_wiener(3 * cfg.n, 1, p["dt"], 75)
    plan = bnd.Plan(p, "fp64", max_rhs=1, max_cheb=100)
    Rg = torch.tensor(R.reshape(-1), device="cuda")
    D = plan.alloc_D()
    stats = bnd.new_stats()
    dS = torch.empty(1, 3 * cfg.n, dtype=torch.float64, device="cuda")
    plan.step(Rg, D, torch.tensor(dW, device="cuda"), m=1, n_cheb=0, ef_tol=tol,
              lanczos_iters=100, bound_safety=0.05, dmin_fraction=0.3, dS=dS, stats=stats)
    st = bnd.read_stats(stats)
    assert st["status"] in (0, 6)
    Dr = oracle.build_D(p, R)
    dS_r, Ef_r, n_r, ok_r = oracle.cheb_sqrt_adaptive(Dr, st["d_min"], st["d_max"], dW, tol, 100)
    assert st["n_cheb"] == n_r
    assert (st["status"] == 0) == ok_r
    assert relerr(dS.cpu().numpy(), dS_r) <= 1e-11
    R_ref, st_ref, _, _, _ = oracle.step(p, R, dW, st["d_min"], st["d_max"], n_r)
    if st_ref == 0:
        assert st["accepted"] == 1
        disp = Rg.cpu().numpy() - R.reshape(-1)
        assert relerr(disp, R_ref.reshape(-1) - R.reshape(-1)) <= 1e-11


def test_adaptive_mixed_close_to_oracle(bnd):
    cfg, p, R = system(n_chains=30, seed=76)
    D = oracle.build_D(p, R)
    w = np.linalg.eigvalsh(D)
    dmin, dmax = 0.9 * w[0], 1.1 * w[-1]
    dW = inputs.make_wiener(D.shape[0], 2, p["dt"], 77)
    tol = 2e-2
    dS_r, _, n_r, ok_r = oracle.cheb_sqrt_adaptive(D, dmin, dmax, dW, tol, 120)
    plan = bnd.Plan(p, "mixed_f16", max_rhs=2, max_cheb=120)
    Dg = plan.alloc_D()
    plan.build_D(torch.tensor(R, device="cuda"), Dg)
    bounds = torch.tensor([dmin, dmax], dtype=torch.float64, device="cuda")
    dWg = torch.tensor(dW, device="cuda")
    dS = torch.empty_like(dWg)
    Ef = torch.empty(2, dtype=torch.float64, device="cuda")
    n, ok = plan.chebyshev_adaptive(Dg, bounds, tol, dWg, dS, Ef)
    assert ok_r and ok and abs(n - n_r) <= 1
    dS_n, _ = oracle.cheb_sqrt(D, dmin, dmax, n, dW)
    assert relerr(dS.cpu().numpy(), dS_n) <= 1e-3


@pytest.mark.parametrize("prec,mode", [("fp64", 2), ("fp64", 3), ("mixed_f16", 3)])
def test_step_fixman_bounds(bnd, prec, mode):
    """Sec. IV bounds from Fixman's quadratic forms, carried as two extra
    columns of the first product: the step's d_min, d_max against the oracle
    formulas on the oracle D (FP64 1e-11; mixed, 16-bit D, 2e-3)."""
    cfg, p, R = system(n_chains=20, nb=10, seed=78)
    C = 8.0
    plan = bnd.Plan(p, prec, max_rhs=16, max_cheb=30)
    Rg = torch.tensor(R.reshape(-1), device="cuda")
    D = plan.alloc_D()
    stats = bnd.new_stats()
    plan.step(Rg, D, None, m=16, n_cheb=30, bounds_mode=mode, fixman_c=C, seed=5, stats=stats)
    st = bnd.read_stats(stats)
    Dr = oracle.build_D(p, R)
    dmin, dmax, _, _ = oracle.fixman_bounds(Dr, cfg.n, "dilute" if mode == 2 else "semidilute", C)
    tol = 1e-11 if prec == "fp64" else 2e-3
    assert abs(st["d_max"] / dmax - 1) <= tol and abs(st["d_min"] / dmin - 1) <= tol
    assert st["status"] in (0, 5)
