"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test names the passage it checks and the kind of mistake it catches.
None of them retypes the oracle's formula: they check invariants (alpha
independence, translation invariance, symmetry, positive definiteness,
divergence-free flow), closed forms and limits (Hasimoto's self-mobility,
free-space RPY recovery, the coincident-bead limit, C1 continuity at r = 2a,
closed-form Euler steps), library primitives (eigen-decomposition square root,
Cholesky, matmul) and published known-answer vectors (Philox).
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1203_6208_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SQRT_PI = math.sqrt(math.pi)


def mkparams(n, L, a=0.28 * SQRT_PI, alpha_factor=1.0, M=6.0, **kw):
    alpha = alpha_factor * SQRT_PI / L
    rc = M / alpha
    kc = 2 * alpha * M
    n2max = int(math.floor((kc * L / (2 * math.pi)) ** 2 + 1e-9))
    p = dict(n=n, nb=kw.pop("nb", n), L=L, a=a, alpha=alpha, rc=rc, n2max=n2max,
             overlap_corr=1, spring=0, fene_b=50.0, ev_on=0, z_star=0.0, d_star=1.0,
             r_ev=0.0, dt=1e-3)
    p.update(kw)
    return p


def omega_rpy(v, a):
    """Free-space RPY tensor, Eqs. (RPY), (b1), (b2)."""
    r = np.linalg.norm(v)
    rr = np.outer(v, v) / (r * r)
    if r >= 2 * a:
        o1 = 3 * a / (4 * r) * (1 + 2 * a * a / (3 * r * r))
        o2 = 3 * a / (4 * r) * (1 - 2 * a * a / (r * r))
    else:
        o1 = 1 - 9 * r / (32 * a)
        o2 = 3 * r / (32 * a)
    return o1 * np.eye(3) + o2 * rr


def small_system(seed=3, n=7, L=5.0, close_pair=True):
    rng = np.random.default_rng(seed)
    R = rng.uniform(0, L, size=(n, 3))
    if close_pair:
        R[1] = R[0] + np.array([0.31, -0.22, 0.17])       # |r| ~ 0.42 < 2a
        R[3] = R[2] + np.array([0.9, 0.35, -0.2])         # just above 2a
    return R


# ---------------------------------------------------------------------------
# Ewald sum (Eqs. DF, M1, M2, self term)

def test_alpha_independence():
    """Eq. (DF): the Ewald split must not change D.  Catches any wrong
    coefficient in M1, M2 or the self term, and the sign of the reciprocal
    bracket (reading R1)."""
    R = small_system()
    Ds = [oracle.build_D(mkparams(len(R), 5.0, alpha_factor=f, M=6.0), R)
          for f in (0.7, 1.0, 1.6)]
    for D in Ds[1:]:
        assert np.max(np.abs(D - Ds[0])) < 2e-12


def test_translation_invariance():
    """Shifting every bead by the same vector leaves D unchanged.  The printed
    minus sign in the reciprocal bracket of Eq. (DF) gives
    cos(k.(r_nu + r_mu)) and fails this; reading R1 passes."""
    R = small_system(seed=5)
    p = mkparams(len(R), 5.0)
    D0 = oracle.build_D(p, R)
    D1 = oracle.build_D(p, R + np.array([1.234, -0.77, 3.3]))
    assert np.max(np.abs(D1 - D0)) < 1e-12


def test_truncation_error_at_1e8_target():
    """Eqs. (rparameter, kparameter): with exp(-M^2) = 1e-8 the truncated sum
    differs from the converged (M = 6) one by a few 1e-6 relative at most:
    exp(-M^2) times the polynomial prefactors of Eq. (M1) (up to s^4 at
    s = M) summed over the many images near r_c.  Balanced real and
    reciprocal cutoffs keep it independent of alpha to within a factor ~3."""
    R = small_system(seed=11)
    D6 = oracle.build_D(mkparams(len(R), 5.0, M=6.0), R)
    for f in (0.7, 1.0, 1.5):
        D8 = oracle.build_D(mkparams(len(R), 5.0, alpha_factor=f, M=math.sqrt(math.log(1e8))), R)
        err = np.max(np.abs(D8 - D6)) / np.max(np.abs(D6))
        assert 1e-8 < err < 5e-6


def hasimoto_xi():
    with open(os.path.join(GOLDEN, "hasimoto.txt")) as f:
        for line in f:
            if line.startswith("xi"):
                return float(line.split()[1])


@pytest.mark.parametrize("L", [3.0, 7.7, 20.0])
def test_hasimoto_self_mobility(L):
    """Diagonal block = Hasimoto's periodic self-mobility
    1 - xi a/L + (4 pi/3)(a/L)^3 (the periodic Stokes solution the paper's
    Ewald sum builds on).  Pins the self term, the self-image real-space sum
    and the k-sum together."""
    xi = hasimoto_xi()
    a = 0.28 * SQRT_PI
    R = np.array([[0.1, 0.2, 0.3]])
    for f in (0.8, 1.0, 1.3):
        B = oracle.D_block(mkparams(1, L, a=a, alpha_factor=f, M=6.0), R, 0, 0)
        expect = 1 - xi * a / L + 4 * math.pi / 3 * (a / L) ** 3
        assert np.max(np.abs(B - np.diag(np.diag(B)))) < 1e-13       # isotropic
        assert abs(B[0, 0] - expect) < 1e-6 * a / L                   # 7 digits of xi
        # the implied constant is the same for every L and alpha
        xi_impl = (1 - B[0, 0] + 4 * math.pi / 3 * (a / L) ** 3) * L / a
        assert abs(xi_impl - 2.8372974794806) < 1e-10


@pytest.mark.parametrize("r_over_a", [0.6, 1.5, 2.5, 6.0])
def test_free_space_rpy_recovery(r_over_a):
    """Two beads in a growing box: D_12 - Omega(r) - (D_11 - 1) I = O(L^-3)
    for both RPY branches, Eqs. (RPY), (b1), (b2).  For r < 2a this pins the
    overlap correction M* (reading R2): the printed rr coefficient fails."""
    a = 0.5
    v = np.array([0.6, -0.3, 0.74])
    v = v / np.linalg.norm(v) * r_over_a * a
    res = []
    for L in (20.0, 40.0, 80.0):
        R = np.array([[1.0, 2.0, 3.0], [1.0, 2.0, 3.0] + v])
        p = mkparams(2, L, a=a, M=6.0)
        D12 = oracle.D_block(p, R, 0, 1)
        D11 = oracle.D_block(p, R, 0, 0)
        res.append(np.max(np.abs(D12 - omega_rpy(-v, a) - (D11[0, 0] - 1) * np.eye(3))))
    assert res[0] < 2e-3
    assert 5.0 < res[0] / res[1] < 11.0 and 5.0 < res[1] / res[2] < 11.0


def test_symmetry_and_positive_definite():
    """D is a symmetric positive-definite covariance (Eq. decomp needs B with
    B B^T = D).  The printed M* coefficient (reading R2) makes D indefinite
    for overlapping beads; the corrected one must not."""
    cfg, _ = inputs.preset("c1")
    p = cfg.params()
    R = inputs.make_chains(cfg)
    D = oracle.build_D(p, R)
    assert np.max(np.abs(D - D.T)) < 1e-14
    lmin, lmax = oracle.exact_eigs(D)
    assert lmin > 0
    oracle.cholesky(D)                      # raises if not PD
    # the system has overlapping pairs, so the check exercises M*
    d = R[:, None, :] - R[None, :, :]
    d -= p["L"] * np.round(d / p["L"])
    r = np.linalg.norm(d, axis=-1) + np.eye(len(R)) * 1e9
    assert np.sum(r < 2 * p["a"]) >= 2


def test_mstar_C1_continuity_at_2a():
    """M* vanishes to second order at r = 2a (x = 2), so D_12(r) is
    continuous with a continuous derivative across the branch switch
    (Sec. II C).  Catches the printed rr coefficient (jump 1/4)."""
    a = 0.5
    L = 6.0
    p = mkparams(2, L, a=a, M=6.0)
    e = np.array([0.48, 0.6, -0.64])
    e /= np.linalg.norm(e)

    def blk(r):
        R = np.array([[1.0, 1.0, 1.0], [1.0, 1.0, 1.0] + r * e])
        return oracle.D_block(p, R, 0, 1)

    h = 1e-4
    fl1, fl2 = blk(2 * a - h), blk(2 * a - 2 * h)
    fr1, fr2 = blk(2 * a + h), blk(2 * a + 2 * h)
    left, right = 2 * fl1 - fl2, 2 * fr1 - fr2          # one-sided limits, O(h^2)
    assert np.max(np.abs(right - left)) < 1e-7            # continuous
    sl, sr = (fl1 - fl2) / h, (fr2 - fr1) / h             # one-sided slopes, O(h)
    assert np.max(np.abs(sr - sl)) < 2e-3                 # C1
    assert np.max(np.abs(sl)) > 1e-2                      # slopes are not trivially 0


def test_coincident_limit_equals_self_block():
    """As two beads approach (r -> 0) their block D_12 tends to the diagonal
    block D_11: the overlap-corrected Ewald sum (Eq. DFmodified) makes them
    the same bead.  Pins self term + M1 + M* and the cancellation-safe
    evaluation of the close pair together."""
    a = 0.5
    p = mkparams(2, 5.0, a=a, M=6.0)
    e = np.array([0.3, -0.5, 0.81])
    e /= np.linalg.norm(e)
    R0 = np.array([[1.0, 2.0, 1.5]])
    D11 = oracle.D_block(p, np.vstack([R0, R0]), 0, 0)
    for r in (1e-2, 1e-3, 1e-4):
        R = np.vstack([R0, R0 + r * a * e])
        D12 = oracle.D_block(p, R, 0, 1)
        # Omega_B = I - (9/32)(r/a) I + (3/32)(r/a) rr: deviation linear in r
        assert np.max(np.abs(D12 - D11)) < 0.5 * r
    R = np.vstack([R0, R0])
    assert np.allclose(oracle.D_block(p, R, 0, 1), D11, atol=1e-15)


def test_divergence_free():
    """Incompressible solvent: the periodic RPY mobility is divergence-free,
    sum_j d D_ij(r) / d r_j = 0 for r != 0, on both branches.  Catches
    wrong coefficients that alpha-independence alone might let through."""
    a = 0.5
    L = 5.0
    p = mkparams(2, L, a=a, M=6.0)
    h = 1e-4
    for v in (np.array([1.3, -0.4, 0.8]), np.array([0.3, 0.2, -0.35])):
        div = np.zeros(3)
        for j in range(3):
            dv = np.zeros(3)
            dv[j] = h
            Rp = np.array([[0.0, 0.0, 0.0], v + dv])
            Rm = np.array([[0.0, 0.0, 0.0], v - dv])
            Bp = oracle.D_block(p, Rp, 1, 0)
            Bm = oracle.D_block(p, Rm, 1, 0)
            div += (Bp[:, j] - Bm[:, j]) / (2 * h)
        assert np.max(np.abs(div)) < 1e-7


def test_full_build_matches_blocks_and_rows():
    cfg, _ = inputs.preset("c1")
    p = cfg.params()
    R = inputs.make_chains(cfg)
    D = oracle.build_D(p, R)
    rows = oracle.build_D_rows(p, R, 10, 13)
    assert np.array_equal(rows, D[30:39])
    assert np.array_equal(oracle.D_block(p, R, 12, 57), D[36:39, 171:174])


# ---------------------------------------------------------------------------
# Forces (Sec. II A) and narrow-Gaussian EV (reading R6)

def ev_energy(p, R):
    """Excluded-volume energy summed over pairs and images (reading R6)."""
    L, d = p["L"], p["d_star"]
    z = p["z_star"]
    E = 0.0
    n = len(R)
    nmax = int(p["r_ev"] / L + 0.5) + 1
    rng = range(-nmax, nmax + 1)
    for i in range(n):
        for j in range(i + 1, n):
            dd = R[i] - R[j]
            dd -= L * np.round(dd / L)
            for nx in rng:
                for ny in rng:
                    for nz in rng:
                        v = dd + L * np.array([nx, ny, nz])
                        u = v @ v
                        if u <= p["r_ev"] ** 2:
                            E += z / d ** 3 * math.exp(-u / (2 * d * d))
    return E


def test_forces_hookean_fene_closed_form():
    p = mkparams(4, 10.0, nb=2)
    R = np.array([[0, 0, 0], [1.0, 2.0, 2.0], [5, 5, 5], [5.5, 5, 5]], dtype=float)
    F, bad = oracle.forces(p, R)
    assert bad == 0
    F = F.reshape(4, 3)
    assert np.allclose(F[0], [1, 2, 2]) and np.allclose(F[1], [-1, -2, -2])
    assert np.allclose(F[2], [0.5, 0, 0]) and np.allclose(F[3], [-0.5, 0, 0])
    pf = dict(p, spring=1, fene_b=10.0)
    F, bad = oracle.forces(pf, R)
    F = F.reshape(4, 3)
    assert bad == 0
    assert np.allclose(F[0], np.array([1, 2, 2]) / (1 - 9 / 10.0))
    R2 = R.copy()
    R2[1] = [3.0, 2.0, 2.0]                    # |Q|^2 = 17 > b
    _, bad = oracle.forces(pf, R2)
    assert bad == 1


def test_ev_force_is_minus_energy_gradient():
    cfg, _ = inputs.preset("c1")
    p = dict(cfg.params(), n=6, nb=6, L=4.0)
    rng = np.random.default_rng(2)
    R = rng.uniform(0, 4.0, size=(6, 3))
    p_sp = dict(p, ev_on=0)
    Fev = oracle.forces(p, R)[0] - oracle.forces(p_sp, R)[0]
    h = 1e-6
    g = np.zeros(18)
    for i in range(18):
        Rp = R.copy().reshape(-1)
        Rm = R.copy().reshape(-1)
        Rp[i] += h
        Rm[i] -= h
        g[i] = (ev_energy(p, Rp.reshape(6, 3)) - ev_energy(p, Rm.reshape(6, 3))) / (2 * h)
    assert np.max(np.abs(Fev + g)) < 1e-7 * max(1.0, np.max(np.abs(g)))
    assert abs(np.sum(Fev.reshape(6, 3), axis=0)).max() < 1e-12   # action = reaction


# ---------------------------------------------------------------------------
# Products and the Chebyshev square root (Sec. IV)

def test_apply_matches_matmul():
    rng = np.random.default_rng(0)
    D = rng.standard_normal((50, 50))
    X = rng.standard_normal((3, 50))
    assert np.allclose(oracle.apply_D(D, X), (D @ X.T).T, rtol=0, atol=1e-12)


def test_cheb_coeffs_interpolate_at_nodes():
    """Reading R5: sum_p c_p T_p(x_j) - c_0/2 reproduces sqrt at the nodes."""
    nch, dmin, dmax = 13, 0.2, 5.0
    c = oracle.cheb_coeffs(nch, dmin, dmax)
    for j in range(nch):
        t = math.pi * (j + 0.5) / nch
        x = math.cos(t)
        val = sum(c[p] * math.cos(p * math.acos(x)) for p in range(nch)) - c[0] / 2
        lam = 0.5 * (dmax - dmin) * x + 0.5 * (dmax + dmin)
        assert abs(val - math.sqrt(lam)) < 1e-13


def test_cheb_scalar_matrix():
    """D = d I: dS = f_N(d) dW, the interpolant at d, which converges to
    sqrt(d) dW geometrically in N_Ch."""
    d = 1.7
    D = d * np.eye(12)
    dW = np.random.default_rng(1).standard_normal((2, 12))
    errs = []
    for nch in (4, 8, 16, 30):
        dS, _ = oracle.cheb_sqrt(D, 1.0, 3.0, nch, dW)
        errs.append(np.max(np.abs(dS - math.sqrt(d) * dW)))
    assert errs[-1] < 1e-13 and errs[1] < errs[0] and errs[2] < errs[1]


def test_cheb_converges_to_eigen_root_and_SS_equals_D():
    """dS -> D^(1/2) dW (eigen-decomposition root) as N_Ch grows with exact
    bounds; the Chebyshev operator S satisfies S S ~ L L^T (Cholesky)."""
    cfg = inputs.SystemConfig(n_chains=2, nb=8, c_over_cstar=2.0)
    p = cfg.params()
    R = inputs.make_chains(cfg)
    D = oracle.build_D(p, R)
    lmin, lmax = oracle.exact_eigs(D)
    dW = inputs.make_wiener(D.shape[0], 2, 1e-3, 7)
    ref = (oracle.sqrt_eig(D) @ dW.T).T
    prev = None
    for nch in (10, 20, 40, 80):
        dS, Ef = oracle.cheb_sqrt(D, lmin, lmax, nch, dW)
        e = np.max(np.abs(dS - ref)) / np.max(np.abs(ref))
        if prev is not None:
            assert e < prev or e < 1e-12
        prev = e
    assert prev < 1e-10
    # S S vs Cholesky factor
    S, _ = oracle.cheb_sqrt(D, lmin, lmax, 80, np.eye(D.shape[0]))
    Lc = oracle.cholesky(D)
    assert np.max(np.abs(S @ S - Lc @ Lc.T)) < 1e-9
    assert np.max(np.abs(S - S.T)) < 1e-12


def test_fixman_estimates_closed_form():
    """Eq. (lmax-lmin-dilute) on D = a I + b 1 1^T (n even): U+ is an
    eigenvector with eigenvalue a + b n, U- sums to zero so U-.D.U- / n = a;
    then the dilute factors (2, 1/2) and Eqs. (fmax), (fmin)."""
    n, a, b = 12, 0.7, 0.05
    D = a * np.eye(n) + b * np.ones((n, n))
    dmin, dmax, lF, sF = oracle.fixman_bounds(D, 4, "dilute")
    assert abs(lF - (a + b * n)) < 1e-14 and abs(sF - a) < 1e-14
    assert abs(dmax - 2 * (a + b * n)) < 1e-14 and abs(dmin - a / 2) < 1e-14
    nb, C = 4, 8.0
    dmin, dmax, _, _ = oracle.fixman_bounds(D, nb, "semidilute", C)
    lmax = 0.35 * nb ** 0.6 * (a + b * n)
    assert abs(dmax - lmax) < 1e-14 and abs(dmin - lmax / (C * nb ** 0.6)) < 1e-14
    # D = d I: both estimates are d
    _, _, lF, sF = oracle.fixman_bounds(2.5 * np.eye(9), 3, "dilute")
    assert abs(lF - 2.5) < 1e-14 and abs(sF - 2.5) < 1e-14


def test_nch_initial_eq_nint():
    """Eq. (nint): nint(sqrt(ratio)) + 1, halves rounded up."""
    assert oracle.nch_initial(1.0, 100.0) == 11
    assert oracle.nch_initial(1.0, 6.25) == 4          # sqrt = 2.5 -> 3
    assert oracle.nch_initial(2.0, 2.0) == 2
    assert oracle.nch_initial(1.0, 6700.0) == 83       # the N = 8000 spectrum


def test_cheb_adaptive_loop():
    """Sec. IV's adaptive N_Ch: the result is the first N >= N_0 with
    E_f < tol; a loose tol stops at N_0; an unreachable one stops at the cap
    unconverged; a tight tol reproduces the eigen-decomposition root."""
    cfg = inputs.SystemConfig(n_chains=3, nb=8, c_over_cstar=2.0, seed=12)
    p = cfg.params()
    R = inputs.make_chains(cfg)
    D = oracle.build_D(p, R)
    lmin, lmax = oracle.exact_eigs(D)
    dmin, dmax = 0.9 * lmin, 1.1 * lmax
    dW = inputs.make_wiener(D.shape[0], 3, 1e-3, 13)
    n0 = oracle.nch_initial(dmin, dmax)
    _, _, n, ok = oracle.cheb_sqrt_adaptive(D, dmin, dmax, dW, 10.0, 200)
    assert ok and n == n0
    _, _, n, ok = oracle.cheb_sqrt_adaptive(D, dmin, dmax, dW, 1e-300, n0 + 3)
    assert not ok and n == n0 + 3
    dS, Ef, n, ok = oracle.cheb_sqrt_adaptive(D, dmin, dmax, dW, 1e-6, 200)
    assert ok and n > n0 and np.max(Ef) < 1e-6
    _, Ef_prev = oracle.cheb_sqrt(D, dmin, dmax, n - 1, dW)
    assert np.max(Ef_prev) >= 1e-6
    ref = (oracle.sqrt_eig(D) @ dW.T).T
    assert np.max(np.abs(dS - ref)) / np.max(np.abs(ref)) < 1e-5


def test_ef_definition():
    """E_f (Sec. IV) from the oracle equals the definition evaluated with
    the Cholesky factor: dW.D.dW = |L^T dW|^2."""
    cfg = inputs.SystemConfig(n_chains=2, nb=6, c_over_cstar=1.0)
    p = cfg.params()
    R = inputs.make_chains(cfg)
    D = oracle.build_D(p, R)
    lmin, lmax = oracle.exact_eigs(D)
    dW = inputs.make_wiener(D.shape[0], 3, 1e-3, 9)
    dS, Ef = oracle.cheb_sqrt(D, 0.9 * lmin, 1.1 * lmax, 6, dW)
    Lc = oracle.cholesky(D)
    for j in range(3):
        q = np.sum((Lc.T @ dW[j]) ** 2)
        assert abs(Ef[j] - math.sqrt(abs(dS[j] @ dS[j] - q) / q)) < 1e-12
    assert np.all(Ef > 1e-6)         # 6 terms are not converged


# ---------------------------------------------------------------------------
# Euler step, Eq. (sde)

def test_step_closed_form_with_identity_D():
    """a = 0 gives D = I exactly (every Ewald term carries a factor a), so
    Eq. (sde) reduces to r + (dt/4) F + dW/sqrt(2) (dS -> dW)."""
    cfg = inputs.SystemConfig(n_chains=3, nb=5, c_over_cstar=1.0, hstar=0.0, dt=0.01)
    p = cfg.params()
    R = inputs.make_chains(cfg)
    D = oracle.build_D(p, R)
    assert np.max(np.abs(D - np.eye(D.shape[0]))) < 1e-15
    dW = inputs.make_wiener(3 * cfg.n, 2, p["dt"], 4)
    Rn, st, DF, dS, Ef = oracle.step(p, R, dW, 0.5, 2.0, 40)
    F, _ = oracle.forces(p, R)
    assert st == 0
    expect = R.reshape(-1) + p["dt"] / 4 * F + dW[0] / math.sqrt(2)
    assert np.max(np.abs(Rn.reshape(-1) - expect)) < 1e-14


def test_step_components_consistent():
    cfg, extra = inputs.preset("c1")
    p = cfg.params()
    R = inputs.make_chains(cfg)
    D = oracle.build_D(p, R)
    lmin, lmax = oracle.exact_eigs(D)
    dW = inputs.make_wiener(3 * cfg.n, 1, p["dt"], cfg.seed + 1)
    Rn, st, DF, dS, Ef = oracle.step(p, R, dW, 0.9 * lmin, 1.1 * lmax, 20)
    F, _ = oracle.forces(p, R)
    assert st == 0
    assert np.max(np.abs(DF - D @ F)) < 1e-12 * np.max(np.abs(D @ F))
    dS2, _ = oracle.cheb_sqrt(D, 0.9 * lmin, 1.1 * lmax, 20, dW)
    assert np.array_equal(dS, dS2)


def test_fene_rejection_leaves_configuration():
    """Reading R7: a step that over-stretches a FENE spring is rejected."""
    cfg = inputs.SystemConfig(n_chains=2, nb=4, c_over_cstar=1.0, spring=1,
                              fene_b=4.0, dt=0.01)
    p = cfg.params()
    R = np.array([[0, 0, 0], [1.9, 0, 0], [2.5, 0.3, 0], [3.0, 1.0, 0.5],
                  [4, 4, 4], [4.5, 4, 4], [5, 4.5, 4], [5.5, 4.6, 4.2]], dtype=float)
    dW = np.zeros((1, 24))
    dW[0, 4] = 4.0                                  # kick bead 1 along y
    Rn, st, *_ = oracle.step(p, R, dW, 0.1, 3.0, 20)
    assert st > 0
    assert np.array_equal(Rn, R)


# ---------------------------------------------------------------------------
# Philox4x32-10 known answers

def test_philox_known_answers():
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for r in rows:
        vals = [int(x, 16) for x in r]
        assert oracle.philox4x32_10(vals[0:4], vals[4:6]) == vals[6:10]


def test_wiener_philox_moments():
    w = oracle.wiener_philox(42, 7, 200001, 1e-2)
    assert abs(np.mean(w)) < 5 * 0.1 / math.sqrt(len(w))
    assert abs(np.var(w) / 1e-2 - 1) < 0.02


# ---------------------------------------------------------------------------
# Input generator: theta statics of the seeded chains (Eqs. Re2, Rg2)

def test_seeded_chains_theta_statics():
    cfg = inputs.SystemConfig(n_chains=4000, nb=10, c_over_cstar=1.0)
    R = inputs.make_chains(cfg).reshape(4000, 10, 3)
    re2 = np.mean(np.sum((R[:, -1] - R[:, 0]) ** 2, axis=-1))
    rg2 = np.mean(np.sum((R - R.mean(axis=1, keepdims=True)) ** 2, axis=-1).mean(axis=1))
    assert abs(re2 / (3 * 9) - 1) < 0.05
    assert abs(rg2 / ((100 - 1) / 20) - 1) < 0.05


# ---------------------------------------------------------------------------
# Gradient of g . D(R) F (adjoint of the drift product)

def test_grad_DF_matches_central_differences():
    """The oracle's analytic dL/dR of L = g.D(R)F against central finite
    differences of the oracle's own D (h = 1e-6), on a system with
    overlapping pairs (M* branch) and both real and reciprocal sums; and
    dL/dF = D g."""
    R = small_system(seed=17, n=7, L=5.0)
    p = mkparams(len(R), 5.0, M=4.5)
    rng = np.random.default_rng(4)
    F = rng.standard_normal(3 * len(R))
    g = rng.standard_normal(3 * len(R))
    gR, gF = oracle.grad_DF(p, R, F, g)
    D = oracle.build_D(p, R)
    assert np.allclose(gF, D @ g, rtol=0, atol=1e-13)
    h = 1e-6
    fd = np.zeros_like(R)
    for i in range(len(R)):
        for c in range(3):
            Rp, Rm = R.copy(), R.copy()
            Rp[i, c] += h
            Rm[i, c] -= h
            fd[i, c] = (g @ oracle.build_D(p, Rp) @ F - g @ oracle.build_D(p, Rm) @ F) / (2 * h)
    assert np.max(np.abs(gR - fd)) < 2e-7 * max(1.0, np.max(np.abs(fd)))
    assert np.max(np.abs(gR.sum(axis=0))) < 1e-12     # pair forces: action = reaction


def test_cheb_adjoint_matches_central_differences():
    """Reverse pass of the Chebyshev series (bounds and N_Ch fixed): dL/ddW
    equals P(D) h (the series is symmetric in D), and dL/dR through D(R)
    matches central differences of L = h . dS(R)."""
    R = small_system(seed=23, n=6, L=5.0)
    p = mkparams(len(R), 5.0, M=4.5)
    D = oracle.build_D(p, R)
    lmin, lmax = oracle.exact_eigs(D)
    dmin, dmax, nch = 0.8 * lmin, 1.1 * lmax, 12
    rng = np.random.default_rng(8)
    dW = rng.standard_normal((2, 3 * len(R)))
    h = rng.standard_normal((2, 3 * len(R)))
    X, Y, U0 = oracle.cheb_adjoint(D, dmin, dmax, nch, dW, h)
    Ph, _ = oracle.cheb_sqrt(D, dmin, dmax, nch, h)
    assert np.max(np.abs(U0 - Ph)) < 1e-12 * np.max(np.abs(Ph))
    gR = oracle.grad_pairs(p, R, X, Y)

    def L(Rx):
        dS, _ = oracle.cheb_sqrt(oracle.build_D(p, Rx), dmin, dmax, nch, dW)
        return float(np.sum(h * dS))
    hh = 1e-6
    fd = np.zeros_like(R)
    for i in range(len(R)):
        for c in range(3):
            Rp, Rm = R.copy(), R.copy()
            Rp[i, c] += hh
            Rm[i, c] -= hh
            fd[i, c] = (L(Rp) - L(Rm)) / (2 * hh)
    assert np.max(np.abs(gR - fd)) < 2e-7 * max(1.0, np.max(np.abs(fd)))
