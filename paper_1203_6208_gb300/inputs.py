"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the Brownian-dynamics step itself: it only
sizes the periodic box, picks the Ewald parameters from the accuracy target,
draws bead-spring chains as Gaussian random walks and draws Wiener increments.

System recipe (the paper's systems, Sec. II A and Sec. VI):
  * N = N_c chains x N_b beads, chains contiguous in the bead index.
  * Bead radius a = sqrt(pi) h* (Sec. II A, below Eq. b2).
  * Concentration c = (c/c*) c*, c* = N_b / ((4 pi/3) (R_g^0)^3) with the
    theta-solvent R_g^0 from Eq. (Rg2): (R_g^0)^2 = (N_b^2 - 1)/(2 N_b).
    Box edge L = (N/c)^(1/3).
  * Ewald: alpha = f sqrt(pi)/L (f = 1 balances image and k counts),
    r_c = M/alpha and k_c = 2 alpha M (Eqs. rparameter, kparameter) with
    exp(-M^2) = 1e-8, i.e. M = sqrt(ln 1e8).  k-vectors k = 2 pi n/L with
    n.n <= n2max = floor((k_c L / 2 pi)^2).
  * Chains: first bead uniform in [0, L)^3, bond vectors i.i.d. N(0, 1) per
    component (unit bond variance, so <R_e^2> = 3 (N_b - 1), Eq. Re2).
    FENE systems redraw any bond with |Q|^2 >= 0.9 b.  Coordinates unwrapped.
  * Wiener increments: i.i.d. N(0, dt) per component (Sec. II A).
  * Random numbers: numpy PCG64 streams, seed = 1000 + config id for chains
    and seed + 1 for the Wiener increments.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

SQRT_PI = math.sqrt(math.pi)
M_1E8 = math.sqrt(math.log(1e8))          # exp(-M^2) = 1e-8


def c_star(nb: int) -> float:
    """Overlap concentration N_b / ((4 pi/3) R_g^3), R_g from Eq. (Rg2)."""
    rg2 = (nb * nb - 1.0) / (2.0 * nb)
    return nb / (4.0 * math.pi / 3.0 * rg2 ** 1.5)


@dataclass
class SystemConfig:
    n_chains: int
    nb: int
    c_over_cstar: float
    hstar: float = 0.28
    spring: int = 0               # 0 Hookean, 1 FENE
    fene_b: float = 50.0
    ev_on: int = 0
    z_star: float = 1.0
    overlap_corr: int = 1
    dt: float = 1e-3
    alpha_factor: float = 1.0
    M: float = M_1E8
    seed: int = 1000
    L_override: float = 0.0

    @property
    def n(self) -> int:
        return self.n_chains * self.nb

    def params(self) -> dict:
        """Plain dict understood by both the oracle and the C-ABI binding."""
        n = self.n
        if self.L_override > 0:
            L = float(self.L_override)
        else:
            c = self.c_over_cstar * c_star(self.nb)
            L = (n / c) ** (1.0 / 3.0)
        alpha = self.alpha_factor * SQRT_PI / L
        rc = self.M / alpha
        kc = 2.0 * alpha * self.M
        n2max = int(math.floor((kc * L / (2.0 * math.pi)) ** 2 + 1e-9))
        d_star = self.z_star ** 0.2
        r_ev = d_star * math.sqrt(2.0 * math.log(1e16))
        return dict(n=n, nb=self.nb, L=L, a=SQRT_PI * self.hstar, alpha=alpha, rc=rc,
                    kc=kc, n2max=n2max, overlap_corr=self.overlap_corr,
                    spring=self.spring, fene_b=self.fene_b, ev_on=self.ev_on,
                    z_star=self.z_star, d_star=d_star, r_ev=r_ev, dt=self.dt)


def make_chains(cfg: SystemConfig, seed: int | None = None) -> np.ndarray:
    """Bead positions (N, 3) float64 as seeded Gaussian random walks."""
    rng = np.random.Generator(np.random.PCG64(cfg.seed if seed is None else seed))
    p = cfg.params()
    L = p["L"]
    R = np.empty((cfg.n, 3), dtype=np.float64)
    for c in range(cfg.n_chains):
        start = rng.uniform(0.0, L, size=3)
        bonds = rng.standard_normal((cfg.nb - 1, 3))
        if cfg.spring == 1:
            for j in range(cfg.nb - 1):
                while float(bonds[j] @ bonds[j]) >= 0.9 * cfg.fene_b:
                    bonds[j] = rng.standard_normal(3)
        R[c * cfg.nb] = start
        R[c * cfg.nb + 1:(c + 1) * cfg.nb] = start + np.cumsum(bonds, axis=0)
    return R


def make_wiener(n3: int, m: int, dt: float, seed: int) -> np.ndarray:
    """(m, 3N) array; row j is Wiener column j, entries N(0, dt)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((m, n3)) * math.sqrt(dt)


# --------------------------------------------------------------------------
# The five workloads (sizes from the paper's systems; see module docstring).
PRESETS = {
    # N=100: 10 Hookean chains x 10 beads at c/c*=1, EV z*=1, N_Ch=20, m=1
    "c1": dict(cfg=SystemConfig(n_chains=10, nb=10, c_over_cstar=1.0, ev_on=1,
                                z_star=1.0, seed=1001), nch=20, m=1),
    # N=1000: 100 FENE chains x 10 beads (b=50), c/c* in {1,2,4}
    "c2": dict(cfg=SystemConfig(n_chains=100, nb=10, c_over_cstar=1.0, spring=1,
                                fene_b=50.0, ev_on=1, z_star=1.0, seed=1002),
               nch=0, m=1, tol=1e-3),
    # N=8000: 400 chains x 20 beads, theta solution (EV off, M* on), m=16
    "c4": dict(cfg=SystemConfig(n_chains=400, nb=20, c_over_cstar=4.0, ev_on=0,
                                seed=1004), nch=40, m=16),
    # N=2000: 100 chains x 20 beads, c/c*=2 (differentiable step)
    "c5": dict(cfg=SystemConfig(n_chains=100, nb=20, c_over_cstar=2.0, ev_on=0,
                                seed=1005), nch=20, m=1),
}


def preset(name: str, **overrides) -> tuple[SystemConfig, dict]:
    d = PRESETS[name]
    cfg = replace(d["cfg"], **overrides) if overrides else d["cfg"]
    extra = {k: v for k, v in d.items() if k != "cfg"}
    return cfg, extra


def batch_systems(count: int = 64, seed: int = 1003, n_min: int = 200, n_max: int = 2000):
    """Replica systems of the batched workload: N_b ~ U{10..20}, N ~ U[n_min,
    n_max] rounded to a multiple of N_b, c/c* ~ U[1, 4], Hookean theta
    chains; replica i's chains are seeded with seed * 1000 + i."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        nb = int(rng.integers(10, 21))
        n = int(rng.integers(n_min, n_max + 1))
        nc = max(1, int(round(n / nb)))
        c = float(rng.uniform(1.0, 4.0))
        out.append(SystemConfig(n_chains=nc, nb=nb, c_over_cstar=c, seed=seed * 1000 + i))
    return out


# theta-solution validation (Sec. VI): Hookean chains, a = 0.5, dt = 0.01,
# N_c = 20, concentrations from 3e-4 c* to 3 c* (box size varied)
THETA_CONCENTRATIONS = (3e-4, 3e-3, 3e-2, 0.3, 3.0)


def theta_systems(nb: int = 20, n_chains: int = 20, concentrations=THETA_CONCENTRATIONS,
                  replicas: int = 8, seed: int = 2000, alpha_factor: float = 1.5):
    """Replica systems of the theta validation workload: for each c/c*,
    `replicas` independent boxes of n_chains Hookean chains of nb beads
    (EV off, overlap-corrected RPY, a = 0.5), seeded seed * 1000 + index.
    The chains start from the exact theta equilibrium (Gaussian bonds of
    unit variance per component)."""
    out = []
    i = 0
    for c in concentrations:
        for _ in range(replicas):
            out.append(SystemConfig(n_chains=n_chains, nb=nb, c_over_cstar=float(c),
                                    hstar=0.5 / SQRT_PI, dt=0.01, ev_on=0, spring=0,
                                    alpha_factor=alpha_factor, seed=seed * 1000 + i))
            i += 1
    return out
