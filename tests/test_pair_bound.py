"""The pair estimate of lambda_min (Sec. IV bounds) on the oracle's D.

The library tightens its lower eigenvalue bound with
theta_pair = d_s - max over pairs of rho(D_{nu mu}), the smallest eigenvalue
of a pair's 6 x 6 principal submatrix.  That rests on three facts about the
Ewald-summed D, checked here on the CPU oracle:
  * every diagonal 3 x 3 block is the same multiple of the identity (the
    self term and the lattice sums are isotropic by cubic symmetry), so the
    submatrix is [[d_s I, B], [B, d_s I]] with eigenvalues d_s -+ eig(B);
  * theta_pair >= lambda_min (Cauchy interlacing), for any configuration;
  * in dense solutions with overlapping beads the lowest eigenvectors sit on
    the closest pairs, so theta_pair is within a few per cent of lambda_min.
A wrong block (a transposed index, a missing isotropic term) or a wrong sign
in the eigenvalue formula fails one of these.
"""
import numpy as np
import pytest

import oracle
from paper_1203_6208_gb300 import inputs


def pair_estimate(D, n):
    """d_s and max over nu < mu of the spectral radius of the symmetric part
    of block (nu, mu), from the 3x3 eigenvalues (numpy LAPACK)."""
    B = D.reshape(n, 3, n, 3).transpose(0, 2, 1, 3)
    iu = np.triu_indices(n, 1)
    blocks = B[iu]
    blocks = 0.5 * (blocks + blocks.transpose(0, 2, 1))
    ev = np.linalg.eigvalsh(blocks)
    return D[0, 0], np.max(np.abs(ev))


@pytest.mark.parametrize("c_over_cstar,nb,chains", [(4.0, 20, 30), (1.0, 10, 40)])
def test_diagonal_blocks_common_multiple_of_identity(c_over_cstar, nb, chains):
    cfg = inputs.SystemConfig(n_chains=chains, nb=nb, c_over_cstar=c_over_cstar, seed=91)
    p = cfg.params()
    D = oracle.build_D(p, inputs.make_chains(cfg))
    n = cfg.n
    diag = np.stack([D[3 * i:3 * i + 3, 3 * i:3 * i + 3] for i in range(n)])
    ds = diag[0, 0, 0]
    assert np.max(np.abs(diag - ds * np.eye(3))) < 1e-13 * ds


def test_pair_estimate_interlaces_and_is_tight_in_dense_solution():
    """c/c* = 4, 20-bead chains (the benchmark's solution), N = 600."""
    cfg = inputs.SystemConfig(n_chains=30, nb=20, c_over_cstar=4.0, seed=92)
    p = cfg.params()
    R = inputs.make_chains(cfg)
    D = oracle.build_D(p, R)
    lmin, _ = oracle.exact_eigs(D)
    ds, rho = pair_estimate(D, cfg.n)
    theta = ds - rho
    assert theta >= lmin * (1 - 1e-10)
    assert theta <= 1.1 * lmin
    # the bottom eigenvector is a pair mode: two beads hold almost all of it
    w, V = np.linalg.eigh(D)
    wb = (V[:, 0].reshape(cfg.n, 3) ** 2).sum(1)
    assert np.sort(wb)[-2:].sum() > 0.95


def test_pair_estimate_interlaces_in_dilute_solution():
    """Without close pairs the estimate is loose but still an upper bound
    of lambda_min, so d_min = f min(theta_Lanczos, theta_pair) stays valid."""
    cfg = inputs.SystemConfig(n_chains=10, nb=10, c_over_cstar=0.3, seed=93)
    p = cfg.params()
    D = oracle.build_D(p, inputs.make_chains(cfg))
    lmin, _ = oracle.exact_eigs(D)
    ds, rho = pair_estimate(D, cfg.n)
    assert ds - rho >= lmin * (1 - 1e-10)
