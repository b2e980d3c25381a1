"""Non-finite positions: the assembly and the matrix-free product return.

With a NaN or infinite position the separation of every pair with that bead
is not finite.  The real-space image search then enumerates no images (its
range tests would otherwise be false forever).  The reciprocal terms carry
the NaN into that bead's rows and columns only, so every other entry of D,
and every product row that does not involve the bead, stays finite.
"""
import numpy as np
import pytest

from paper_1203_6208_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bnd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_6208_gb300 import binding, build
    build.build()
    binding.load()
    return binding


@pytest.mark.parametrize("prec", ["fp64", "mixed_f16"])
def test_build_D_nonfinite_bead(bnd, prec):
    cfg = inputs.SystemConfig(n_chains=6, nb=10, c_over_cstar=2.0, seed=71)
    p = cfg.params()
    R = inputs.make_chains(cfg)
    bad = (7, 33)
    R[bad[0]] = [np.nan, 0.5, 0.5]
    R[bad[1]] = [1.0, np.inf, -2.0]
    plan = bnd.Plan(p, prec, max_rhs=2)
    Rg = torch.tensor(R, device="cuda")
    D = plan.alloc_D()
    plan.build_D(Rg, D)
    torch.cuda.synchronize()
    Dv = plan.D_view(D).double().cpu().numpy()
    rows = np.zeros(3 * cfg.n, dtype=bool)
    for b in bad:
        rows[3 * b:3 * b + 3] = True
    assert not np.all(np.isfinite(Dv[rows]))
    assert np.all(np.isfinite(Dv[np.ix_(~rows, ~rows)]))
    plan.close()


def test_matfree_nonfinite_bead(bnd):
    """The matrix-free product recomputes the real-space pairs per product."""
    cfg = inputs.SystemConfig(n_chains=6, nb=10, c_over_cstar=2.0, seed=72)
    p = cfg.params()
    R = inputs.make_chains(cfg)
    R[12] = [np.nan, np.nan, np.nan]
    plan = bnd.Plan(p, "fp64", max_rhs=2)
    X = torch.tensor(inputs.make_wiener(3 * cfg.n, 2, 1.0, 73), device="cuda")
    Y = torch.empty_like(X)
    plan.apply_matfree(torch.tensor(R, device="cuda"), X, Y)
    torch.cuda.synchronize()
    assert Y.shape == X.shape
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed_f16"])
def test_build_D_far_coordinate(bnd, prec):
    """A finite coordinate far outside the box (1e30) is reduced into [0, L)
    exactly (fmod), so the assembly returns, D is finite everywhere and it
    equals, bit for bit, D built from that bead's exactly reduced position."""
    cfg = inputs.SystemConfig(n_chains=6, nb=10, c_over_cstar=2.0, seed=74)
    p = cfg.params()
    R = inputs.make_chains(cfg)
    far = R.copy()
    far[9] = [1e30, -3.3e29, 7.1e26]
    near = R.copy()
    near[9] = np.mod(far[9], p["L"])          # fmod, plus L where negative
    plan = bnd.Plan(p, prec, max_rhs=2)
    out = []
    for pos in (far, near):
        D = plan.alloc_D()
        plan.build_D(torch.tensor(pos, device="cuda"), D)
        torch.cuda.synchronize()
        out.append(plan.D_view(D).double().cpu().numpy())
    assert np.all(np.isfinite(out[0]))
    assert np.array_equal(out[0], out[1])
    plan.close()


def test_adjoint_far_coordinate(bnd):
    """The adjoint takes minimum-image separations of the unwrapped positions
    with an exact remainder: a bead at 1e30 leaves every gradient finite."""
    cfg = inputs.SystemConfig(n_chains=6, nb=10, c_over_cstar=2.0, seed=75)
    p = cfg.params()
    R = inputs.make_chains(cfg)
    R[21] = [-1e30, 2.5e29, 4.0]
    plan = bnd.Plan(p, "fp64", max_rhs=2)
    Rg = torch.tensor(R, device="cuda")
    D = plan.alloc_D()
    plan.build_D(Rg, D)
    F = torch.tensor(inputs.make_wiener(3 * cfg.n, 1, 1.0, 76)[0], device="cuda")
    gY = torch.tensor(inputs.make_wiener(3 * cfg.n, 1, 1.0, 77)[0], device="cuda")
    gR = torch.empty_like(F)
    plan.apply_backward(Rg, D, F, gY, gR)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(gR).all())
    plan.close()
