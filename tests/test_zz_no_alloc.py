"""bd_eig_bounds_noalloc: the Lanczos bounds for callers that cannot
allocate device memory (no plan, scratch in a fixed device array).

It must give the bounds of the plan-based bd_eig_bounds on the same matrix,
on two calls in a row (the shared array keeps the first call's contents),
and refuse sizes beyond its array before doing any work.  Collected last so
that a failure here never hides the rest of the suite.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bnd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_6208_gb300 import binding, build
    build.build()
    binding.load()
    return binding


@pytest.mark.gpu
def test_noalloc_bounds_match_plan_bounds_twice(bnd):
    from paper_1203_6208_gb300 import inputs
    cfg = inputs.SystemConfig(n_chains=40, nb=10, c_over_cstar=2.0, seed=81)
    p = cfg.params()
    plan = bnd.Plan(p, "fp64", max_rhs=1, max_cheb=8)
    R = torch.tensor(inputs.make_chains(cfg), device="cuda")
    D = plan.alloc_D()
    plan.build_D(R, D)
    ref = torch.empty(2, dtype=torch.float64, device="cuda")
    ref_st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    plan.eig_bounds(D, 40, 0.05, 0.5, ref, ref_st)
    for _ in range(2):
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        bnd.eig_bounds_noalloc(D, plan.n3, plan.ld, 40, 0.05, 0.5, out, st)
        torch.cuda.synchronize()
        assert int(st.item()) == int(ref_st.item()) == 0
        # both run FP64 Lanczos steps with the same start vector and the same
        # multisection, whose bracket is 1e-6 of the value wide: a product
        # formed in another order may land one bracket cell away
        np.testing.assert_allclose(out.cpu().numpy(), ref.cpu().numpy(), rtol=2e-6, atol=0)


@pytest.mark.gpu
def test_noalloc_bounds_unaligned_matrix(bnd):
    """D may start on any 8-byte boundary with any leading dimension: a copy
    of the matrix one element into a buffer, with an odd leading dimension,
    gives the bounds of the aligned original."""
    from paper_1203_6208_gb300 import inputs
    cfg = inputs.SystemConfig(n_chains=20, nb=10, c_over_cstar=2.0, seed=82)
    p = cfg.params()
    plan = bnd.Plan(p, "fp64", max_rhs=1, max_cheb=8)
    D = plan.alloc_D()
    plan.build_D(torch.tensor(inputs.make_chains(cfg), device="cuda"), D)
    n3 = plan.n3
    ld = n3 + 1 if n3 % 2 == 0 else n3 + 2          # odd leading dimension
    buf = torch.zeros(1 + n3 * ld, dtype=torch.float64, device="cuda")
    buf[1:].view(n3, ld)[:, :n3] = plan.D_view(D)
    res = []
    for mat, lda in ((plan.D_view(D), plan.ld), (buf[1:], ld)):
        out = torch.empty(2, dtype=torch.float64, device="cuda")
        st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        bnd.eig_bounds_noalloc(mat, n3, lda, 30, 0.05, 0.5, out, st)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        res.append(out.cpu().numpy())
    assert buf[1:].data_ptr() % 16 == 8
    np.testing.assert_allclose(res[1], res[0], rtol=2e-6, atol=0)
    plan.close()


@pytest.mark.gpu
def test_noalloc_bounds_rejects_oversize(bnd):
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    dummy = torch.empty(8, dtype=torch.float64, device="cuda")
    with pytest.raises(bnd.BDError) as e:
        bnd.eig_bounds_noalloc(dummy, 3 * 8193, 3 * 8193, 10, 0.05, 0.5, out)
    assert e.value.status == 8 and "limit" in str(e.value)
