"""Eigenvalue bounds bracket the spectrum (Sec. IV: d_min <= lambda_min and
d_max >= lambda_max) at the sizes of the eigenvalue study and of the
benchmark, with the benchmark's settings: 30 Lanczos steps, d_max = 1.05
theta_max, d_min = 0.5 min(theta_min, theta_pair).

FP64 plans take fresh bounds every step; mixed plans take lagged ones (the
previous step's Lanczos recurrence, carried in the products) with d_min
tightened by the current D's pair estimate.  The reference spectrum is the
exact one of the very matrix the step used (FP32 eigvalsh of its upper
triangle on the device; FP32 rounding moves the extreme eigenvalues by
~1e-6, far inside the margins checked).  For mixed plans the 16-bit copy
that the Chebyshev products multiply by is checked too.
"""
import numpy as np
import pytest

from paper_1203_6208_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SETTINGS = dict(lanczos_iters=30, bound_safety=0.05, dmin_fraction=0.5)


@pytest.fixture(scope="module")
def bnd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_6208_gb300 import binding, build
    build.build()
    binding.load()
    return binding


def extremes(A):
    """Smallest and largest eigenvalue of the symmetric matrix whose upper
    triangle A holds (device FP32 eigvalsh)."""
    w = torch.linalg.eigvalsh(A.float(), UPLO="U")
    out = float(w[0]), float(w[-1])
    del w
    torch.cuda.empty_cache()
    return out


def theta_system(chains, alpha_factor):
    cfg, _ = inputs.preset("c4", alpha_factor=alpha_factor, n_chains=chains)
    return cfg, cfg.params(), inputs.make_chains(cfg)


@pytest.mark.parametrize("chains", [150, 400])
def test_fresh_bounds_bracket_fp64_step(bnd, chains):
    """N = 3000 and 8000 (c/c* = 4, the FP64 benchmark's alpha = 1.5 sqrt(pi)/L)."""
    cfg, p, R0 = theta_system(chains, 1.5)
    plan = bnd.Plan(p, "fp64", max_rhs=16, max_cheb=40)
    R = torch.tensor(R0, device="cuda")
    D = plan.alloc_D()
    stats = bnd.new_stats()
    plan.step(R, D, None, m=16, n_cheb=40, seed=11, step_index=0, stats=stats, bounds_mode=0,
              **SETTINGS)
    torch.cuda.synchronize()
    st = bnd.read_stats(stats)
    lmin, lmax = extremes(plan.D_view(D))
    assert st["status"] == 0
    assert st["d_min"] <= lmin and lmax <= st["d_max"]
    # the estimate is tight (pair modes): d_min is half of a value within
    # ~10 % of lambda_min, not an arbitrarily small floor
    assert st["d_min"] >= 0.4 * lmin
    # the stand-alone entry point gives the same bounds on the same D
    b = torch.empty(2, dtype=torch.float64, device="cuda")
    plan.eig_bounds(D, 30, 0.05, 0.5, b)
    torch.cuda.synchronize()
    np.testing.assert_allclose(b.cpu().numpy(), [st["d_min"], st["d_max"]], rtol=1e-12)
    plan.close()


@pytest.mark.parametrize("chains", [150, 400])
def test_lagged_bounds_bracket_mixed_steps(bnd, chains):
    """The benchmark's mixed step: symmetric product shape, m = 16, N_Ch = 40,
    alpha = 2 sqrt(pi)/L, lagged bounds; the first step runs fresh Lanczos,
    the next three use the previous step's recurrence."""
    cfg, p, R0 = theta_system(chains, 2.0)
    plan = bnd.Plan(p, "mixed_f16", max_rhs=16, max_cheb=40)
    plan.set_shape(bnd.BD_SHAPE_SYMMETRIC)
    R = torch.tensor(R0, device="cuda")
    D = plan.alloc_D()
    stats = bnd.new_stats()
    for k in range(4):
        plan.step(R, D, None, m=16, n_cheb=40, seed=12, step_index=k, stats=stats,
                  bounds_mode=1, **SETTINGS)
        torch.cuda.synchronize()
        st = bnd.read_stats(stats)
        assert st["status"] == 0 and st["accepted"] == 1
        for which in ("f32", "f16"):
            lmin, lmax = extremes(plan.D_view(D, which))
            assert st["d_min"] <= lmin, (k, which, st["d_min"], lmin)
            assert lmax <= st["d_max"], (k, which, lmax, st["d_max"])
        assert st["d_min"] >= 0.4 * lmin
    plan.close()


def test_pair_estimate_matches_block_eigenvalues(bnd):
    """bd_eig_bounds' d_min on a dense solution (N = 1000, c/c* = 4) is
    0.5 theta_pair, theta_pair = d_s - max rho(D_{nu mu}) computed here from
    the 3x3 blocks with LAPACK (the Lanczos value is far above it at 30
    steps); and it brackets lambda_min from below."""
    cfg, p, R0 = theta_system(50, 1.0)
    plan = bnd.Plan(p, "fp64", max_rhs=1, max_cheb=8)
    D = plan.alloc_D()
    plan.build_D(torch.tensor(R0, device="cuda"), D)
    b = torch.empty(2, dtype=torch.float64, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    plan.eig_bounds(D, 30, 0.05, 0.5, b, st)
    torch.cuda.synchronize()
    Dh = plan.D_view(D).cpu().numpy()
    n = cfg.n
    blocks = Dh.reshape(n, 3, n, 3).transpose(0, 2, 1, 3)[np.triu_indices(n, 1)]
    rho = np.max(np.abs(np.linalg.eigvalsh(0.5 * (blocks + blocks.transpose(0, 2, 1)))))
    theta = Dh[0, 0] - rho
    assert int(st.item()) == 0
    np.testing.assert_allclose(float(b[0]), 0.5 * theta, rtol=2e-5)
    w = np.linalg.eigvalsh(Dh)
    assert float(b[0]) <= w[0] <= theta and w[-1] <= float(b[1])
    plan.close()
