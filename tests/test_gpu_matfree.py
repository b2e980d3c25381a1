"""Matrix-free products and steps (the paper's LMA: D(R) X recomputed per
product, D never stored) against the oracle's D and against the dense path.

Bars: FP64 products within 1e-11 of the oracle's D X (max-norm relative);
FP32 (mixed plans) within 2e-6 (the FP32 D bar); matrix-free and dense FP64
steps each within 1e-11 of the oracle step at their own bounds; the N = 8000
workload's matrix-free rows against oracle rows.
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


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("mixed_f16", 2e-6)])
@pytest.mark.parametrize("n_chains,nb,m,ev,spring", [(7, 11, 1, 0, 0), (7, 11, 5, 0, 0),
                                                      (100, 10, 3, 1, 1), (20, 10, 19, 0, 0)])
def test_matfree_product_vs_oracle(bnd, prec, tol, n_chains, nb, m, ev, spring):
    cfg = inputs.SystemConfig(n_chains=n_chains, nb=nb, c_over_cstar=2.0, seed=81, ev_on=ev,
                              spring=spring)
    p = cfg.params()
    R = inputs.make_chains(cfg)
    X = inputs.make_wiener(3 * cfg.n, m, 1.0, 82)
    plan = bnd.Plan(p, prec, max_rhs=max(m - 3, 1), max_cheb=8)
    Y = torch.empty(m, 3 * cfg.n, dtype=torch.float64, device="cuda")
    plan.apply_matfree(torch.tensor(R, device="cuda"), torch.tensor(X, device="cuda"), Y)
    ref = oracle.apply_D(oracle.build_D(p, R), X)
    assert relerr(Y.cpu().numpy(), ref) <= tol


def test_matfree_step_fp64_vs_oracle(bnd):
    """Dense and matrix-free FP64 steps, each against the oracle step run with
    that step's own Lanczos bounds (theta_min is sensitive to the rounding of
    the products, so the two paths' bounds agree only to ~1e-6)."""
    cfg, _ = inputs.preset("c5", n_chains=20)
    p = cfg.params()
    R = inputs.make_chains(cfg)
    m, nch = 2, 20
    dW_h = inputs.make_wiener(3 * cfg.n, m, p["dt"], 83)
    dW = torch.tensor(dW_h, device="cuda")
    bounds = {}
    for mf in (False, True):
        plan = bnd.Plan(p, "fp64", max_rhs=m, max_cheb=nch)
        Rg = torch.tensor(R.reshape(-1), device="cuda")
        D = None if mf else plan.alloc_D()
        DF = torch.empty(3 * cfg.n, dtype=torch.float64, device="cuda")
        dS = torch.empty(m, 3 * cfg.n, dtype=torch.float64, device="cuda")
        stats = bnd.new_stats()
        plan.step(Rg, D, dW, m=m, n_cheb=nch, lanczos_iters=40, DF=DF, dS=dS, stats=stats,
                  flags=bnd.BD_STEP_MATRIX_FREE if mf else 0)
        st = bnd.read_stats(stats)
        assert st["status"] == 0 and st["accepted"] == 1
        bounds[mf] = (st["d_min"], st["d_max"])
        R_ref, st_ref, DF_r, dS_r, _ = oracle.step(p, R, dW_h, st["d_min"], st["d_max"], nch)
        assert st_ref == 0
        assert relerr(DF.cpu().numpy(), DF_r) <= 1e-11
        assert relerr(dS.cpu().numpy(), dS_r) <= 1e-11
        disp = Rg.cpu().numpy() - R.reshape(-1)
        assert relerr(disp, R_ref.reshape(-1) - R.reshape(-1)) <= 1e-11
    assert abs(bounds[True][1] / bounds[False][1] - 1) < 1e-9
    assert abs(bounds[True][0] / bounds[False][0] - 1) < 1e-3


def test_matfree_step_mixed_vs_oracle(bnd):
    cfg, _ = inputs.preset("c5", n_chains=20)
    p = cfg.params()
    R = inputs.make_chains(cfg)
    m, nch = 1, 20
    dW = inputs.make_wiener(3 * cfg.n, m, p["dt"], 84)
    plan = bnd.Plan(p, "mixed_f16", max_rhs=m, max_cheb=nch)
    Rg = torch.tensor(R.reshape(-1), device="cuda")
    DF = torch.empty(3 * cfg.n, dtype=torch.float64, device="cuda")
    dS = torch.empty(m, 3 * cfg.n, dtype=torch.float64, device="cuda")
    stats = bnd.new_stats()
    plan.step(Rg, None, torch.tensor(dW, device="cuda"), m=m, n_cheb=nch, lanczos_iters=40,
              DF=DF, dS=dS, stats=stats, flags=bnd.BD_STEP_MATRIX_FREE)
    st = bnd.read_stats(stats)
    assert st["status"] == 0 and st["accepted"] == 1
    R_ref, st_ref, DF_r, dS_r, _ = oracle.step(p, R, dW, st["d_min"], st["d_max"], nch)
    assert st_ref == 0
    assert relerr(DF.cpu().numpy(), DF_r) <= 2e-6
    assert relerr(dS.cpu().numpy(), dS_r) <= 2e-5


def test_matfree_n8000_sampled_rows(bnd):
    cfg, _ = inputs.preset("c4", alpha_factor=1.75)
    p = cfg.params()
    R = inputs.make_chains(cfg)
    m = 4
    X = inputs.make_wiener(3 * cfg.n, m, 1.0, 85)
    plan = bnd.Plan(p, "mixed_f16", max_rhs=m, max_cheb=8)
    Y = torch.empty(m, 3 * cfg.n, dtype=torch.float64, device="cuda")
    plan.apply_matfree(torch.tensor(R, device="cuda"), torch.tensor(X, device="cuda"), Y)
    Yh = Y.cpu().numpy()
    for b in (0, 3333, 7999):
        rows = oracle.build_D_rows(p, R, b, b + 1)
        ref = rows @ X.T
        assert np.max(np.abs(Yh[:, 3 * b:3 * b + 3].T - ref)) <= 2e-6 * np.max(np.abs(Yh))
