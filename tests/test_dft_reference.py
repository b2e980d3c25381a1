"""The reference of the mesh-transform parity test (numpy's FFT) against the
discrete Fourier transform written out as its definition: a dense K x K
matrix of e^{-+2 pi i jk/K} applied along each axis of small meshes.  Forward:
the half spectrum k_z <= K/2 of the unnormalised transform; inverse: the
unnormalised sum with e^{+2 pi i jk/K} over the full spectrum, which for a
Hermitian spectrum is K^3 times numpy's normalised inverse of the half."""
import numpy as np
import pytest


def dft_matrix(K, sign):
    j = np.arange(K)
    return np.exp(sign * 2j * np.pi * np.outer(j, j) / K)


def dft3(x, sign):
    K = x.shape[-1]
    F = dft_matrix(K, sign)
    for axis in (1, 2, 3):
        x = np.moveaxis(np.tensordot(x, F, axes=([axis], [1])), -1, axis)
    return x


@pytest.mark.parametrize("K", [2, 6, 10, 12, 18, 30])
def test_numpy_fft_is_the_dft(K):
    x = np.random.default_rng(K).standard_normal((2, K, K, K))
    full = dft3(x.astype(complex), -1)
    half = np.fft.rfftn(x, axes=(1, 2, 3))
    scale = np.max(np.abs(full))
    assert np.max(np.abs(half - full[..., : K // 2 + 1])) <= 1e-12 * scale
    back = dft3(full, +1)
    assert np.max(np.abs(back.imag)) <= 1e-12 * np.max(np.abs(back))
    ref = K ** 3 * np.fft.irfftn(half, s=(K, K, K), axes=(1, 2, 3))
    assert np.max(np.abs(back.real - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert np.max(np.abs(ref - K ** 3 * x)) <= 1e-12 * np.max(np.abs(ref))
