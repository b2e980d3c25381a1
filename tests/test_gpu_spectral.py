"""Spectral matrix-free products (real space over cell lists with r_c < L/2,
reciprocal sum on a B-spline mesh) against the oracle's truncated Ewald D.

The mesh approximates the same k-sphere sum as the dense D, with an error
that falls as the mesh is refined and the spline order raised; the real-space
part is exact.  Measured on this system (max-norm relative to D X, FP64):
(K, p) = (64, 6) 5.6e-6, (64, 8) 1.2e-7, (96, 10) 2.6e-11, (128, 10)
1.3e-12 -- roughly (m_eff/K)^p with m_eff ~ M L/(pi r_c) the mesh index where
the Gaussian of Eq. (M2) has decayed.  Bars: the error falls along that
sequence; (128, 10) within 1e-11 in FP64; FP32 (mixed plans, arithmetic floor
~5e-7) within 2e-6 at (64, 8); the real-space part alone (n2max = 0) within
1e-11 (FP64).  A matrix-free step through the spectral products against the
oracle step at the step's own bounds.
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


def system(n_chains=24, nb=10, c=2.0, seed=91, f=6.0, **kw):
    cfg = inputs.SystemConfig(n_chains=n_chains, nb=nb, c_over_cstar=c, seed=seed,
                              alpha_factor=f, **kw)
    p = cfg.params()
    assert p["rc"] < 0.5 * p["L"]
    return cfg, p, inputs.make_chains(cfg)


@pytest.fixture(scope="module")
def ref():
    cfg, p, R = system()
    X = inputs.make_wiener(3 * cfg.n, 5, 1.0, 92)
    return cfg, p, R, X, oracle.apply_D(oracle.build_D(p, R), X)


def spectral(bnd, p, R, X, prec, K, order):
    q = dict(p, pme_grid=K, pme_order=order)
    plan = bnd.Plan(q, prec, max_rhs=X.shape[0], max_cheb=8)
    Y = torch.empty(X.shape, dtype=torch.float64, device="cuda")
    plan.apply_matfree(torch.tensor(R, device="cuda"), torch.tensor(X, device="cuda"), Y)
    return Y.cpu().numpy()


def test_spectral_fp64_converges(bnd, ref):
    cfg, p, R, X, Y_ref = ref
    errs = [relerr(spectral(bnd, p, R, X, "fp64", K, order), Y_ref)
            for K, order in ((64, 6), (64, 8), (96, 10), (128, 10))]
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] <= 1e-11


def test_spectral_fp32(bnd, ref):
    cfg, p, R, X, Y_ref = ref
    assert relerr(spectral(bnd, p, R, X, "mixed_f16", 64, 8), Y_ref) <= 2e-6


@pytest.mark.parametrize("n_chains,f", [(24, 6.0), (60, 8.0), (200, 9.0)])
def test_real_space_cells_exact(bnd, n_chains, f):
    """n2max = 0: only the real-space sum and the self term, against the
    oracle with no k-sum; alpha = f sqrt(pi)/L gives one cell (f = 6) or
    6 and 7 cells per edge searched two deep (f = 8 and 9)."""
    cfg, p, R = system(n_chains=n_chains, f=f, c=4.0)
    p = dict(p, n2max=0)
    X = inputs.make_wiener(3 * cfg.n, 3, 1.0, 93)
    Y = spectral(bnd, p, R, X, "fp64", 8, 4)
    assert relerr(Y, oracle.apply_D(oracle.build_D(p, R), X)) <= 1e-11


def test_spectral_step_vs_oracle(bnd):
    cfg, p, R = system(n_chains=24, seed=94)
    q = dict(p, pme_grid=128, pme_order=10)
    m, nch = 2, 16
    dW = inputs.make_wiener(3 * cfg.n, m, p["dt"], 95)
    plan = bnd.Plan(q, "fp64", max_rhs=m, max_cheb=nch)
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
    e = {"DF": relerr(DF.cpu().numpy(), DF_r), "dS": relerr(dS.cpu().numpy(), dS_r)}
    assert e["DF"] <= 1e-11 and e["dS"] <= 1e-11, e
