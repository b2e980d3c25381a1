"""The bounded-wait failure path of the symmetric tensor-core product,
exercised without any GPU fault.

bd_plan_test_stall arms a symmetric product of a plan (the next one, or a
given product of a Chebyshev series, whose first D tiles are loaded before the
previous kernel's results are visible): one of its CTAs
waits on an mbarrier that nothing completes, gives up after a bounded spin as
a wait that ran out does, lets its copies in flight land, frees its TMEM and
returns.  Checked here: the step holding that product returns, reports
BD_ERR_TIMEOUT and leaves the positions unchanged; the hook is one-shot; the
next product on the same plan is bit-identical to the one before the stall
(the sums run in a fixed order) and the next step is accepted.
"""
import pytest

from paper_1203_6208_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BD_ERR_TIMEOUT = 7


@pytest.fixture(scope="module")
def bnd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_6208_gb300 import binding, build
    build.build()
    binding.load()
    return binding


def test_symmetric_product_timeout_path(bnd):
    cfg = inputs.SystemConfig(n_chains=50, nb=20, c_over_cstar=4.0, seed=61)   # N = 1000
    p = cfg.params()
    plan = bnd.Plan(p, "mixed_f16", max_rhs=4, max_cheb=16)
    plan.set_shape(bnd.BD_SHAPE_SYMMETRIC)
    R0 = torch.tensor(inputs.make_chains(cfg), device="cuda")
    R = R0.clone()
    D = plan.alloc_D()
    plan.build_D(R, D)
    X = torch.tensor(inputs.make_wiener(3 * cfg.n, 4, 1.0, 62), device="cuda")
    Y_ref = torch.empty_like(X)
    plan.apply(D, X, Y_ref)
    torch.cuda.synchronize()

    kw = dict(m=4, n_cheb=12, lanczos_iters=20, bound_safety=0.05, dmin_fraction=0.5,
              seed=5, bounds_mode=0)
    stats = bnd.new_stats()
    plan.test_stall(0)
    plan.step(R, D, None, step_index=0, stats=stats, **kw)
    torch.cuda.synchronize()                       # the stalled CTA gave up and returned
    st = bnd.read_stats(stats)
    assert st["status"] == BD_ERR_TIMEOUT
    assert st["accepted"] == 0
    assert torch.equal(R, R0)

    Y = torch.empty_like(X)
    plan.apply(D, X, Y)
    torch.cuda.synchronize()
    assert torch.equal(Y, Y_ref)

    plan.step(R, D, None, step_index=1, stats=stats, **kw)
    torch.cuda.synchronize()
    st = bnd.read_stats(stats)
    assert st["status"] == 0 and st["accepted"] == 1
    assert not torch.equal(R, R0)
    plan.close()


@pytest.mark.parametrize("cta,term", [(0, 1), (5, 3)])
def test_series_product_timeout_path(bnd, cta, term):
    """The stall in a product of the Chebyshev series, whose first D tiles are
    loaded ahead of the dependency wait: the CTA that gives up still lets
    those tiles land (it completes their stages) before it returns."""
    cfg = inputs.SystemConfig(n_chains=50, nb=20, c_over_cstar=4.0, seed=65)   # N = 1000
    p = cfg.params()
    plan = bnd.Plan(p, "mixed_f16", max_rhs=4, max_cheb=16)
    plan.set_shape(bnd.BD_SHAPE_SYMMETRIC)
    R0 = torch.tensor(inputs.make_chains(cfg), device="cuda")
    R = R0.clone()
    D = plan.alloc_D()
    plan.build_D(R, D)
    X = torch.tensor(inputs.make_wiener(3 * cfg.n, 4, 1.0, 66), device="cuda")
    Y_ref = torch.empty_like(X)
    plan.apply(D, X, Y_ref)
    torch.cuda.synchronize()

    kw = dict(m=4, n_cheb=12, lanczos_iters=20, bound_safety=0.05, dmin_fraction=0.5,
              seed=7, bounds_mode=0)
    stats = bnd.new_stats()
    plan.test_stall(cta, term)
    plan.step(R, D, None, step_index=0, stats=stats, **kw)
    torch.cuda.synchronize()
    st = bnd.read_stats(stats)
    assert st["status"] == BD_ERR_TIMEOUT
    assert st["accepted"] == 0
    assert torch.equal(R, R0)

    Y = torch.empty_like(X)
    plan.apply(D, X, Y)
    torch.cuda.synchronize()
    assert torch.equal(Y, Y_ref)

    plan.step(R, D, None, step_index=1, stats=stats, **kw)
    torch.cuda.synchronize()
    st = bnd.read_stats(stats)
    assert st["status"] == 0 and st["accepted"] == 1
    assert not torch.equal(R, R0)
    plan.close()


def test_stall_hook_arguments(bnd):
    cfg = inputs.SystemConfig(n_chains=5, nb=10, c_over_cstar=1.0, seed=63)
    p = cfg.params()
    fp64 = bnd.Plan(p, "fp64", max_rhs=1, max_cheb=8)
    with pytest.raises(bnd.BDError):
        fp64.test_stall(0)
    fp64.test_stall(-1)                            # disarming is always allowed
    mixed = bnd.Plan(p, "mixed_f16", max_rhs=1, max_cheb=8)
    mixed.set_shape(1)
    with pytest.raises(bnd.BDError):               # not the symmetric shape
        mixed.test_stall(0)
    mixed.set_shape(bnd.BD_SHAPE_SYMMETRIC)
    with pytest.raises(bnd.BDError):
        mixed.test_stall(100000)
    with pytest.raises(bnd.BDError):
        mixed.test_stall(0, -1)
    fp64.close()
    mixed.close()
