"""FP64 plans in launch shape 4 (BD_SHAPE_F64_DOUBLE_FLOAT): the products
D X formed in double-float on the FP32 pipe, against the FP64 oracle and
against a plain FP64 matrix product.

Error model of the shape: D entries keep 48 significant bits (hi truncated
to 24, lo the rest rounded to 24: within 2^-48), X entries 48 (rounded), the
lo x lo product is dropped, and each
32-term k tile is summed as an unnormalised FP32 pair before it is added to
the running pair with renormalisation.  Each product d x is therefore within
about 2^-46 |d x| and each sum within a small multiple of 2^-47 sum_k |d x|:
for the RPY D and Wiener columns (cancellation sum |d x| / |y| of order ten)
that is ~1e-13 of max|Y|, so the FP64 bar of the other FP64 tests (1e-11 of
max|Y| against the oracle) holds unchanged.  Arbitrary entries (zeros, signs,
all mantissa bits set, exponents from 2^-110 to 2^100) are checked element by
element against the bound 2^-40 sum_k |D_ik x_k|; entries below 2^-97 count
as zero, a change far inside that bound."""
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


def df_plan(bnd, p, R, **kw):
    plan = bnd.Plan(p, "fp64", **kw)
    plan.set_shape(bnd.BD_SHAPE_F64_DOUBLE_FLOAT)
    Rg = torch.tensor(np.ascontiguousarray(R), device="cuda")
    D = plan.alloc_D()
    plan.build_D(Rg, D)
    torch.cuda.synchronize()
    return plan, Rg, D


def product(plan, D, X):
    Xg = torch.tensor(X, device="cuda")
    Y = torch.empty_like(Xg)
    plan.apply(D, Xg, Y)
    return Y.cpu().numpy()


@pytest.mark.parametrize("n_chains,nb,m", [(5, 10, 1), (5, 10, 2), (7, 11, 3), (7, 11, 4),
                                           (30, 10, 5), (30, 10, 8), (30, 10, 16),
                                           (30, 10, 17), (70, 10, 32)])
def test_df_apply_vs_oracle(bnd, n_chains, nb, m):
    """3N = 150, 231 (ragged 32-row tiles and k tiles), 900, 2100; every
    column count class of the kernel (1, 2, 4, 8, 16, 32 columns) and the
    one-column GEMV."""
    cfg = inputs.SystemConfig(n_chains=n_chains, nb=nb, c_over_cstar=2.0, seed=61)
    p = cfg.params()
    R = inputs.make_chains(cfg)
    plan, Rg, D = df_plan(bnd, p, R, max_rhs=32)
    X = inputs.make_wiener(3 * cfg.n, m, 1.0, 62)
    Y = product(plan, D, X)
    ref = oracle.apply_D(oracle.build_D(p, R), X)
    assert relerr(Y, ref) <= TOL
    for j in range(m):
        assert relerr(Y[j], ref[j]) <= TOL
    plan.set_shape(0)                               # FP64 multiply-adds, same D
    assert relerr(Y, product(plan, D, X)) <= TOL


@pytest.mark.parametrize("m", [1, 3, 16])
def test_df_split_arbitrary_entries(bnd, m):
    """A D filled with entries that exercise the word split: zeros and
    negative zeros, all 52 mantissa bits set, exact small integers, binary
    exponents from -110 (below -97 an entry counts as zero) to +100, random
    signs; against
    numpy's FP64 product element by element."""
    cfg = inputs.SystemConfig(n_chains=7, nb=11, c_over_cstar=2.0, seed=63)
    p = cfg.params()
    R = inputs.make_chains(cfg)
    plan, Rg, D = df_plan(bnd, p, R, max_rhs=16)
    n3 = 3 * cfg.n
    rng = np.random.default_rng(64)
    A = rng.standard_normal((n3, n3)) * np.exp2(rng.integers(-110, 101, size=(n3, n3)))
    A[rng.random((n3, n3)) < 0.05] = 0.0
    A[rng.random((n3, n3)) < 0.02] = -0.0
    allbits = np.nextafter(np.exp2(rng.integers(-20, 21, size=(n3, n3)).astype(np.float64)), 0.0)
    pick = rng.random((n3, n3)) < 0.1
    A[pick] = (allbits * np.sign(rng.standard_normal((n3, n3))))[pick]
    ints = rng.integers(-1000, 1000, size=(n3, n3)).astype(np.float64)
    pick = rng.random((n3, n3)) < 0.1
    A[pick] = ints[pick]
    plan.D_view(D).copy_(torch.tensor(A, device="cuda"))
    X = inputs.make_wiener(n3, m, 1.0, 65)
    Y = product(plan, D, X)
    exact = X @ A.T                                  # m x 3N, FP64
    bound = np.abs(X) @ np.abs(A).T
    assert np.all(np.abs(Y - exact) <= 2.0 ** -40 * bound + 1e-300)


@pytest.mark.parametrize("m,nch", [(1, 20), (4, 40), (16, 12)])
def test_df_chebyshev_vs_oracle(bnd, m, nch):
    cfg = inputs.SystemConfig(n_chains=20, nb=10, c_over_cstar=2.0, seed=51)
    p = cfg.params()
    R = inputs.make_chains(cfg)
    plan, Rg, D = df_plan(bnd, p, R, max_rhs=32, max_cheb=64)
    Dr = oracle.build_D(p, R)
    lmin, lmax = oracle.exact_eigs(Dr)
    dmin, dmax = 0.9 * lmin, 1.05 * lmax
    dW = inputs.make_wiener(3 * cfg.n, m, p["dt"], 52)
    bounds = torch.tensor([dmin, dmax], dtype=torch.float64, device="cuda")
    dWg = torch.tensor(dW, device="cuda")
    dS = torch.empty_like(dWg)
    plan.chebyshev(D, bounds, nch, dWg, dS)
    dS_r, _ = oracle.cheb_sqrt(Dr, dmin, dmax, nch, dW)
    assert relerr(dS.cpu().numpy(), dS_r) <= TOL


def test_df_step_vs_oracle_and_dfma(bnd):
    """One FP64 step with fresh Lanczos bounds in shape 4 against the oracle
    step at the bounds it found, and against the same step in shape 0."""
    cfg, _ = inputs.preset("c1")
    p = cfg.params()
    R = inputs.make_chains(cfg)
    dW = inputs.make_wiener(3 * cfg.n, 2, p["dt"], cfg.seed + 1)
    res = []
    for shape in (0, 4):
        plan = bnd.Plan(p, "fp64", max_rhs=2, max_cheb=64)
        plan.set_shape(shape)
        Rg = torch.tensor(R, device="cuda")
        D = plan.alloc_D()
        DF = torch.empty(3 * cfg.n, dtype=torch.float64, device="cuda")
        dS = torch.empty(2, 3 * cfg.n, dtype=torch.float64, device="cuda")
        stats = bnd.new_stats()
        plan.step(Rg, D, torch.tensor(dW, device="cuda"), m=2, n_cheb=30, lanczos_iters=60,
                  bound_safety=0.02, dmin_fraction=0.5, DF=DF, dS=dS, stats=stats)
        st = bnd.read_stats(stats)
        assert st["status"] == 0 and st["accepted"] == 1
        res.append((st, DF.cpu().numpy(), dS.cpu().numpy(), Rg.cpu().numpy()))
        plan.close()
    (s0, DF0, dS0, R0), (s4, DF4, dS4, R4) = res
    # the Lanczos recurrences see products that differ by ~1e-13; once the
    # top Ritz value has converged, orthogonality is lost and the residual
    # term of the bound amplifies such differences (measured 8.7e-8 relative
    # on d_max after 60 steps).  Both pairs bracket the spectrum and agree
    # far inside the 2 % safety margin.
    lmin, lmax = oracle.exact_eigs(oracle.build_D(p, R))
    for st in (s0, s4):
        assert st["d_max"] >= lmax and 0 < st["d_min"] <= lmin
    assert abs(s4["d_max"] / s0["d_max"] - 1) <= 1e-6
    assert abs(s4["d_min"] / s0["d_min"] - 1) <= 1e-6
    R_ref, code, DF_r, dS_r, _ = oracle.step(p, R, dW, s4["d_min"], s4["d_max"], 30)
    assert code == 0
    assert relerr(DF4, DF_r) <= TOL
    assert relerr(dS4, dS_r) <= TOL
    assert relerr(R4, R_ref) <= TOL
    assert relerr(DF4, DF0) <= TOL


def test_df_shape_rules(bnd):
    """Shape 4 is refused on a mixed plan; an FP64 plan takes 1..3 as 0."""
    cfg = inputs.SystemConfig(n_chains=5, nb=10, c_over_cstar=2.0, seed=66)
    p = cfg.params()
    mixed = bnd.Plan(p, "mixed_f16", max_rhs=2)
    with pytest.raises(bnd.BDError):
        mixed.set_shape(bnd.BD_SHAPE_F64_DOUBLE_FLOAT)
    mixed.close()
    with pytest.raises(bnd.BDError):
        bnd.Plan(p, "fp64", max_rhs=2).set_shape(6)
    R = inputs.make_chains(cfg)
    plan, Rg, D = df_plan(bnd, p, R, max_rhs=4)
    X = inputs.make_wiener(3 * cfg.n, 4, 1.0, 67)
    Y4 = product(plan, D, X)
    plan.set_shape(bnd.BD_SHAPE_SYMMETRIC)          # ignored on FP64: multiply-adds
    Y0 = product(plan, D, X)
    plan.set_shape(0)
    assert np.array_equal(Y0, product(plan, D, X))
    assert relerr(Y4, Y0) <= TOL
