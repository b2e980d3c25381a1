"""Reverse mode of the drift product D(R).F and of the Chebyshev term
P(D(R)) dW, on the differentiable-step system (N = 2000: 100 chains x 20
beads, c/c* = 2) and a small one.

Checks: the GPU gradient against the oracle's FP64 gradient (analytic,
itself pinned by finite differences); directional derivatives along 50
seeded random directions against central differences (h = 1e-6) of the GPU
forward; FP32 (mixed plan) gradients against FP64; torch.autograd end to end.
The finite-difference budget includes the truncation jump of D at r = r_c
and |k| = k_c (~1e-8 absolute per image crossing) divided by 2h.
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
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_6208_gb300 import autograd, binding, build
    build.build()
    binding.load()
    return binding, autograd


def c5(n_chains=100):
    cfg, _ = inputs.preset("c5", n_chains=n_chains)
    p = cfg.params()
    return cfg, p, inputs.make_chains(cfg)


@pytest.mark.parametrize("n_chains", [4, 100])
def test_drift_gradient_vs_oracle(mods, n_chains):
    bnd, ag = mods
    cfg, p, R = c5(n_chains)
    rng = np.random.default_rng(91)
    F = rng.standard_normal(3 * cfg.n)
    g = rng.standard_normal(3 * cfg.n)
    plan = bnd.Plan(p, "fp64", max_rhs=1)
    Rg = torch.tensor(R, device="cuda")
    D = plan.alloc_D()
    plan.build_D(Rg, D)
    gR = torch.empty(3 * cfg.n, dtype=torch.float64, device="cuda")
    gF = torch.empty(3 * cfg.n, dtype=torch.float64, device="cuda")
    plan.apply_backward(Rg, D, torch.tensor(F, device="cuda"), torch.tensor(g, device="cuda"),
                        gR, gF)
    gR_ref, gF_ref = oracle.grad_DF(p, R, F, g)
    assert relerr(gR.cpu().numpy().reshape(-1, 3), gR_ref) <= 1e-11
    assert relerr(gF.cpu().numpy(), gF_ref) <= 1e-11


def test_drift_gradient_central_differences(mods):
    bnd, ag = mods
    cfg, p, R = c5()
    sysm = ag.BDSystem(p, "fp64")
    rng = np.random.default_rng(92)
    Rg = torch.tensor(R, device="cuda", requires_grad=True)
    F = torch.tensor(rng.standard_normal(3 * cfg.n), device="cuda", requires_grad=True)
    g = torch.tensor(rng.standard_normal(3 * cfg.n), device="cuda")
    Y = ag.drift(Rg, F, sysm)
    gR, gF = torch.autograd.grad(Y, (Rg, F), g)
    h = 1e-6
    worst = 0.0
    for k in range(50):
        dirn = torch.tensor(rng.standard_normal((cfg.n, 3)), device="cuda")
        dirn /= dirn.norm()
        with torch.no_grad():
            Lp = float(g @ ag.drift(Rg + h * dirn, F, sysm))
            Lm = float(g @ ag.drift(Rg - h * dirn, F, sysm))
        fd = (Lp - Lm) / (2 * h)
        an = float((gR * dirn).sum())
        worst = max(worst, abs(fd - an) / max(abs(an), 1e-3 * float(gR.norm())))
    assert worst <= 1e-4
    # F enters linearly: gF = D g exactly
    with torch.no_grad():
        Dg = ag.drift(Rg, g, sysm)
    assert torch.allclose(gF, Dg, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("n_chains", [4, 100])
def test_chebyshev_gradient_vs_oracle(mods, n_chains):
    bnd, ag = mods
    cfg, p, R = c5(n_chains)
    nch = 20
    D = oracle.build_D(p, R)
    if n_chains <= 10:
        lmin, lmax = oracle.exact_eigs(D)
    else:
        w = np.linalg.eigvalsh(D)
        lmin, lmax = w[0], w[-1]
    dmin, dmax = 0.8 * lmin, 1.05 * lmax
    rng = np.random.default_rng(93)
    dW = inputs.make_wiener(3 * cfg.n, 1, p["dt"], 94)
    h = rng.standard_normal((1, 3 * cfg.n))
    plan = bnd.Plan(p, "fp64", max_rhs=1, max_cheb=nch)
    Rg = torch.tensor(R, device="cuda")
    Dg = plan.alloc_D()
    plan.build_D(Rg, Dg)
    bounds = torch.tensor([dmin, dmax], dtype=torch.float64, device="cuda")
    gR = torch.empty(3 * cfg.n, dtype=torch.float64, device="cuda")
    gdW = torch.empty(1, 3 * cfg.n, dtype=torch.float64, device="cuda")
    plan.chebyshev_backward(Rg, Dg, bounds, nch, torch.tensor(dW, device="cuda"),
                            torch.tensor(h, device="cuda"), gR, gdW)
    X, Y, U0 = oracle.cheb_adjoint(D, dmin, dmax, nch, dW, h)
    gR_ref = oracle.grad_pairs(p, R, X, Y)
    assert relerr(gR.cpu().numpy().reshape(-1, 3), gR_ref) <= 1e-11
    assert relerr(gdW.cpu().numpy(), U0) <= 1e-11


def test_chebyshev_gradient_central_differences_and_autograd(mods):
    bnd, ag = mods
    cfg, p, R = c5()
    nch = 20
    sysm = ag.BDSystem(p, "fp64", max_rhs=1, max_cheb=nch)
    Rg = torch.tensor(R, device="cuda", requires_grad=True)
    sysm.build(Rg)
    bounds = torch.empty(2, dtype=torch.float64, device="cuda")
    sysm.plan.eig_bounds(sysm.D, 40, 0.05, 0.5, bounds)
    rng = np.random.default_rng(95)
    dW = torch.tensor(inputs.make_wiener(3 * cfg.n, 1, p["dt"], 96), device="cuda",
                      requires_grad=True)
    h = torch.tensor(rng.standard_normal((1, 3 * cfg.n)), device="cuda")
    dS = ag.brownian(Rg, dW, bounds, nch, sysm)
    gR, gdW = torch.autograd.grad(dS, (Rg, dW), h)
    hh = 1e-6
    worst = 0.0
    for k in range(50):
        dirn = torch.tensor(rng.standard_normal((cfg.n, 3)), device="cuda")
        dirn /= dirn.norm()
        with torch.no_grad():
            Lp = float((h * ag.brownian(Rg + hh * dirn, dW, bounds, nch, sysm)).sum())
            Lm = float((h * ag.brownian(Rg - hh * dirn, dW, bounds, nch, sysm)).sum())
        fd = (Lp - Lm) / (2 * hh)
        an = float((gR * dirn).sum())
        worst = max(worst, abs(fd - an) / max(abs(an), 1e-3 * float(gR.norm())))
    assert worst <= 1e-4
    with torch.no_grad():
        Ph = ag.brownian(Rg, h, bounds, nch, sysm)    # dS is linear in dW: gdW = P(D) h
    assert torch.allclose(gdW, Ph, rtol=1e-12, atol=1e-14)


def test_fp32_gradients_close_to_fp64(mods):
    """The mixed plan differentiates in FP32 arithmetic (FP64 accumulation of
    the pair sums); its gradients stay within 1e-4 of the FP64 ones."""
    bnd, ag = mods
    cfg, p, R = c5()
    rng = np.random.default_rng(97)
    F = torch.tensor(rng.standard_normal(3 * cfg.n), device="cuda")
    g = torch.tensor(rng.standard_normal(3 * cfg.n), device="cuda")
    out = {}
    for prec in ("fp64", "mixed_f16"):
        plan = bnd.Plan(p, prec, max_rhs=1)
        Rg = torch.tensor(R, device="cuda")
        D = plan.alloc_D()
        plan.build_D(Rg, D)
        gR = torch.empty(3 * cfg.n, dtype=torch.float64, device="cuda")
        gF = torch.empty(3 * cfg.n, dtype=torch.float64, device="cuda")
        plan.apply_backward(Rg, D, F, g, gR, gF)
        out[prec] = (gR.cpu().numpy(), gF.cpu().numpy())
    assert relerr(out["mixed_f16"][0], out["fp64"][0]) <= 1e-4
    assert relerr(out["mixed_f16"][1], out["fp64"][1]) <= 1e-5
