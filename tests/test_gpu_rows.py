"""Launch shape 5 of the mixed products: the 16-bit D streamed row by row on
the CUDA cores with an FP32 operand (a few columns), and the Chebyshev loop
of the step in one persistent launch.

Bars: products within 1e-3 of the oracle's D X (max-norm relative; the
16-bit D rounds each entry by 2^-12 relative and the operand is FP32, not
16-bit as on the tensor cores), ragged row lengths (3N not a multiple of 8),
column counts 1 .. 4 through bd_apply_D and up to 7 through the first
product of a step (F, m = 4 Wiener columns, Fixman's two vectors, or the
Lanczos vector); steps against the oracle step at the step's
own bounds at the mixed-mode bars of the method (1e-5 on the refined D.F,
1e-3 on the Brownian term), with fresh and with lagged bounds.
"""
import numpy as np
import pytest

import oracle
from paper_1203_6208_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BD_SHAPE_ROWS = 5


def relerr(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.fixture(scope="module")
def bnd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_6208_gb300 import binding, build
    build.build()
    binding.load()
    return binding


@pytest.mark.parametrize("prec", ["mixed_f16", "mixed_bf16"])
@pytest.mark.parametrize("n_chains,nb,c", [(1, 2, 0.01), (7, 11, 3.0), (41, 5, 3.0), (30, 20, 3.0)])
def test_rows_product_vs_oracle(bnd, prec, n_chains, nb, c):
    """3N = 6, 231, 615 (not multiples of 8) and 1800; m = 1 .. 4 columns."""
    cfg = inputs.SystemConfig(n_chains=n_chains, nb=nb, c_over_cstar=c, seed=121)
    p = cfg.params()
    R = inputs.make_chains(cfg)
    plan = bnd.Plan(p, prec, max_rhs=4, max_cheb=8)
    plan.set_shape(BD_SHAPE_ROWS)
    D = plan.alloc_D()
    plan.build_D(torch.tensor(R, device="cuda"), D)
    Dr = oracle.build_D(p, R)
    tol = 1e-3 if prec == "mixed_f16" else 8e-3
    for m in range(1, 5):
        X = inputs.make_wiener(3 * cfg.n, m, 1.0, 122 + m)
        Y = torch.empty(m, 3 * cfg.n, dtype=torch.float64, device="cuda")
        plan.apply(D, torch.tensor(X, device="cuda"), Y)
        torch.cuda.synchronize()
        assert relerr(Y.cpu().numpy(), oracle.apply_D(Dr, X)) <= tol, m
    plan.close()


@pytest.mark.parametrize("bounds_mode,m", [(0, 2), (1, 2), (1, 4), (3, 4)])
def test_rows_steps_vs_oracle(bnd, bounds_mode, m):
    """Three steps (N = 600, c/c* = 4, N_Ch = 24), each against the oracle
    step from the same positions with the same noise and bounds: fresh
    Lanczos, lagged Lanczos (m + 2 columns in the first product), Fixman's
    semidilute estimates (m + 3 columns)."""
    cfg = inputs.SystemConfig(n_chains=30, nb=20, c_over_cstar=4.0, seed=123)
    p = cfg.params()
    n3, nch = 3 * cfg.n, 24
    plan = bnd.Plan(p, "mixed_f16", max_rhs=4, max_cheb=nch)
    plan.set_shape(BD_SHAPE_ROWS)
    R = torch.tensor(inputs.make_chains(cfg), device="cuda")
    D = plan.alloc_D()
    stats = bnd.new_stats()
    DF = torch.empty(n3, dtype=torch.float64, device="cuda")
    dS = torch.empty(m, n3, dtype=torch.float64, device="cuda")
    for k in range(3):
        R_in = R.cpu().numpy().copy()
        dW = inputs.make_wiener(n3, m, p["dt"], 124 + k)
        plan.step(R, D, torch.tensor(dW, device="cuda"), m=m, n_cheb=nch, lanczos_iters=30,
                  bound_safety=0.05, dmin_fraction=0.5, DF=DF, dS=dS, stats=stats,
                  bounds_mode=bounds_mode, fixman_c=8.0)
        torch.cuda.synchronize()
        st = bnd.read_stats(stats)
        assert st["status"] == 0 and st["accepted"] == 1
        R_ref, code, DF_r, dS_r, _ = oracle.step(p, R_in, dW, st["d_min"], st["d_max"], nch)
        assert code == 0
        assert relerr(DF.cpu().numpy(), DF_r) <= 1e-5
        assert relerr(dS.cpu().numpy(), dS_r) <= 1e-3
        disp = R.cpu().numpy().reshape(-1) - R_in.reshape(-1)
        assert relerr(disp, R_ref.reshape(-1) - R_in.reshape(-1)) <= 1e-3
    plan.close()


def test_rows_shape_limits(bnd):
    cfg = inputs.SystemConfig(n_chains=4, nb=10, c_over_cstar=1.0, seed=125)
    p = cfg.params()
    big = bnd.Plan(p, "mixed_f16", max_rhs=5, max_cheb=8)
    with pytest.raises(bnd.BDError):
        big.set_shape(BD_SHAPE_ROWS)          # a first product could carry 9 columns
    big.close()
    fp64 = bnd.Plan(p, "fp64", max_rhs=1, max_cheb=8)
    fp64.set_shape(BD_SHAPE_ROWS)             # FP64 plans keep their FP64 products
    fp64.close()
