"""Theta-solution statics (Sec. VI, Eqs. Re2 and Rg2) from trajectories of
the batched GPU step: Hookean chains of N_b = 20 beads, N_c = 20 chains per
box, a = 0.5, dt = 0.01, three concentrations from 3e-3 c* to 3 c*.

The chains start from the exact theta equilibrium, so a correct step keeps
<Q^2> = 3 per bond, <R_e^2> = 3 (N_b - 1) and <R_g^2> = (N_b^2 - 1)/(2 N_b)
at every concentration (chains cross freely in a theta solvent).  The bond
statistic relaxes within a few time units, so a wrong noise amplitude or
drift factor shows in it after the 1500 steps here; the Euler bias at
dt = 0.01 is below 1 %.  R_e^2 and R_g^2 follow the slowest Rouse modes
(relaxation times of order 100 time units, against the 15 simulated), so
their averages stay close to those of the seeded initial ensemble, whose
sampling error is ~5 %.  Bars: <Q^2> within 3 %; <R_e^2> and <R_g^2>
within 4 standard errors (replica-to-replica scatter) and within 20 %.
"""
import numpy as np
import pytest

from paper_1203_6208_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def chain_stats(R, b, cfgs):
    """Per replica: mean bond Q^2, R_e^2 and R_g^2 over its chains."""
    out = []
    for i, c in enumerate(cfgs):
        r = R[b.r_off[i]:b.r_off[i] + b.n3[i]].view(c.n_chains, c.nb, 3)
        q2 = ((r[:, 1:] - r[:, :-1]) ** 2).sum(-1).mean()
        re2 = ((r[:, -1] - r[:, 0]) ** 2).sum(-1).mean()
        rg2 = ((r - r.mean(1, keepdim=True)) ** 2).sum(-1).mean()
        out.append(torch.stack([q2, re2, rg2]))
    return torch.stack(out)


def test_theta_statics_batched():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_6208_gb300 import binding as bnd, build
    build.build()
    bnd.load()
    nb = 20
    cfgs = inputs.theta_systems(nb=nb, concentrations=(3e-3, 0.3, 3.0), replicas=12)
    b = bnd.Batch([c.params() for c in cfgs], "mixed_f16", max_rhs=1, max_cheb=20)
    R = torch.tensor(np.concatenate([inputs.make_chains(c).reshape(-1) for c in cfgs]),
                     device="cuda")
    D = b.alloc_D()
    stats = torch.zeros(b.count * bnd.STATS_BYTES, dtype=torch.uint8, device="cuda")
    acc = torch.zeros(b.count, 3, dtype=torch.float64, device="cuda")
    nsamp = 0
    for k in range(1500):
        b.step(R, D, m=1, n_cheb=20, seed=31, stats=stats, bounds_mode=1)
        if k >= 300 and k % 20 == 0:
            acc += chain_stats(R, b, cfgs)
            nsamp += 1
    torch.cuda.synchronize()
    per_rep = (acc / nsamp).cpu().numpy()
    st = [bnd.BdStepStats.from_buffer_copy(bytes(stats[i * bnd.STATS_BYTES:(i + 1) * bnd.STATS_BYTES]
                                                 .cpu().numpy().tobytes())) for i in range(b.count)]
    assert all(x.status == 0 and x.accepted == 1 for x in st)
    ref = np.array([3.0, 3.0 * (nb - 1), (nb * nb - 1) / (2.0 * nb)])
    for ci in range(3):
        blk = per_rep[12 * ci:12 * (ci + 1)]
        mean = blk.mean(0)
        se = blk.std(0, ddof=1) / np.sqrt(len(blk))
        assert abs(mean[0] / ref[0] - 1) < 0.03, (ci, mean)
        for k in (1, 2):
            assert abs(mean[k] - ref[k]) < 4.0 * se[k], (ci, k, mean, se)
            assert abs(mean[k] / ref[k] - 1) < 0.20, (ci, k, mean)


def test_theta_relaxation_from_off_equilibrium_starts():
    """Chains started far from the theta statics relax to them: bonds
    stretched twofold (<Q^2> = 12) or compressed to 0.3 (<Q^2> = 0.27).
    A uniform rescaling of the bonds puts the same share of the excess into
    every Rouse mode, and the bond statistic follows their average, so the
    slowest mode sets the pace: for 4-bead chains its rate is
    sin^2(pi/8) = 0.15 per time unit (free draining), and 15 time units
    (1500 steps of dt = 0.01) leave ~1 % of the excess.  From there both
    starts must sit at <Q^2> = 3 (Eq. Re2 per bond: the fluctuation-
    dissipation balance of the drift D.F against the noise sqrt(D) dW); a
    wrong drift factor or noise amplitude moves that limit, from either
    side.  Dilute and semidilute boxes (0.03 and 0.3 c*) with N_Ch = 40, so
    that the Chebyshev error stays below 1 % (checked) and the limit tests
    the dynamics, not the series.  Each group's <Q^2> is held to 4 standard
    errors of its replica-to-replica scatter, as the equilibrium test above.
    <R_e^2> = 3 (N_b - 1) is reached too (within its sampling error,
    ~4 % per group of eight replicas)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_6208_gb300 import binding as bnd, build
    build.build()
    bnd.load()
    nb = 4
    cfgs = inputs.theta_systems(nb=nb, concentrations=(0.03, 0.3), replicas=8, seed=2100)
    scale = [2.0 if i % 2 == 0 else 0.3 for i in range(len(cfgs))]
    starts = []
    for c, f in zip(cfgs, scale):
        r = inputs.make_chains(c).reshape(c.n_chains, nb, 3)
        bonds = np.diff(r, axis=1) * f
        r[:, 1:] = r[:, :1] + np.cumsum(bonds, axis=1)
        starts.append(r.reshape(-1))
    b = bnd.Batch([c.params() for c in cfgs], "mixed_f16", max_rhs=1, max_cheb=40)
    R = torch.tensor(np.concatenate(starts), device="cuda")
    D = b.alloc_D()
    stats = torch.zeros(b.count * bnd.STATS_BYTES, dtype=torch.uint8, device="cuda")
    q0 = chain_stats(R, b, cfgs)[:, 0].cpu().numpy()
    acc = torch.zeros(b.count, 3, dtype=torch.float64, device="cuda")
    nsamp = 0
    for k in range(3000):
        b.step(R, D, m=1, n_cheb=40, seed=41, stats=stats, bounds_mode=1)
        if k >= 1500 and k % 10 == 0:
            acc += chain_stats(R, b, cfgs)
            nsamp += 1
    torch.cuda.synchronize()
    per = (acc / nsamp).cpu().numpy()
    q = per[:, 0]
    st = [bnd.BdStepStats.from_buffer_copy(bytes(stats[i * bnd.STATS_BYTES:(i + 1) * bnd.STATS_BYTES]
                                                 .cpu().numpy().tobytes())) for i in range(b.count)]
    assert all(x.status == 0 and x.accepted == 1 for x in st)
    assert max(x.ef_max for x in st) < 0.01, [x.ef_max for x in st]
    stretched, compressed = q[0::2], q[1::2]
    assert np.all(q0[0::2] > 8.0) and np.all(q0[1::2] < 0.5)
    # each group's mean against <Q^2> = 3 within 4 standard errors of the
    # replica-to-replica scatter (~1.4 % of the mean for eight replicas),
    # and the two groups pooled likewise
    for grp in (stretched, compressed, q):
        se = grp.std(ddof=1) / np.sqrt(len(grp))
        assert abs(grp.mean() - 3.0) < 4.0 * se, (grp, se)
    re2 = per[:, 1] / (3.0 * (nb - 1))
    assert abs(re2[0::2].mean() - 1) < 0.15 and abs(re2[1::2].mean() - 1) < 0.15, re2
