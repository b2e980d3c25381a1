"""The spectral product's mesh transforms on their own (bd_mesh_fft) against
the discrete Fourier transform's definition, taken here from numpy's FFT in
FP64: forward, out_k = sum_j x_j e^{-2 pi i j.k/K} on the half spectrum
k_z <= K/2; inverse, the Hermitian completion summed with e^{+2 pi i j.k/K}
(so inverse(forward(x)) = K^3 x).

Sizes cover every radix (4, 2, 3, 5), the most passes a K <= 512 takes
(486 = 2 3^5: six passes), the spectral workload's K = 144, the largest K
(shared memory per CTA is sized by K) and batches with a ragged last CTA.
Bars: FP64 1e-13 of max |out| (the transform's rounding error grows like
eps log K); FP32 2e-6 (measured ~5e-7 at K = 512).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = [2, 6, 8, 10, 12, 18, 30, 40, 50, 64, 90, 96, 144, 150, 250, 270]
BARS = {"fp64": 1e-13, "mixed_f16": 2e-6}


@pytest.fixture(scope="module")
def bnd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_6208_gb300 import binding, build
    build.build()
    binding.load()
    return binding


def relerr(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def forward(bnd, x, prec):
    B, K = x.shape[0], x.shape[1]
    dt = torch.float64 if prec == "fp64" else torch.float32
    xin = torch.tensor(x, dtype=dt, device="cuda")
    y = torch.empty((B, K, K, K // 2 + 1, 2), dtype=dt, device="cuda")
    bnd.mesh_fft(K, B, prec, 0, xin, y)
    y = y.cpu().numpy().astype(np.float64)
    return y[..., 0] + 1j * y[..., 1]


def inverse(bnd, c, prec):
    B, K = c.shape[0], c.shape[1]
    dt = torch.float64 if prec == "fp64" else torch.float32
    cin = torch.tensor(np.stack([c.real, c.imag], axis=-1), dtype=dt, device="cuda")
    y = torch.empty((B, K, K, K), dtype=dt, device="cuda")
    bnd.mesh_fft(K, B, prec, 1, cin, y)
    return y.cpu().numpy().astype(np.float64)


def meshes(B, K, seed, prec):
    x = np.random.default_rng(seed).standard_normal((B, K, K, K))
    # the FP32 path transforms the input as stored: compare from the same values
    return x if prec == "fp64" else x.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("prec", ["fp64", "mixed_f16"])
@pytest.mark.parametrize("K", SIZES)
def test_forward_and_inverse_match_the_dft(bnd, K, prec):
    B = 3
    x = meshes(B, K, 1000 + K, prec)
    ref = np.fft.rfftn(x, axes=(1, 2, 3))
    assert relerr(forward(bnd, x, prec), ref) <= BARS[prec]
    ref_c = ref if prec == "fp64" else ref.astype(np.complex64).astype(np.complex128)
    assert relerr(inverse(bnd, ref_c, prec), K ** 3 * np.fft.irfftn(ref_c, s=(K, K, K), axes=(1, 2, 3))) \
        <= BARS[prec]


@pytest.mark.parametrize("prec,K,B", [("mixed_f16", 486, 1), ("mixed_f16", 512, 1), ("fp64", 512, 1),
                                      ("fp64", 160, 5)])
def test_largest_meshes_and_most_passes(bnd, prec, K, B):
    x = meshes(B, K, 77 + K, prec)
    y = forward(bnd, x, prec)
    ref = np.fft.rfftn(x, axes=(1, 2, 3))
    assert relerr(y, ref) <= BARS[prec]
    del ref
    # round trip through the library's own pair: K^3 x
    back = inverse(bnd, y, prec)
    assert relerr(back, K ** 3 * x) <= 4 * BARS[prec]


def test_rejects_bad_arguments(bnd):
    x = torch.zeros(2 * 15 ** 3, dtype=torch.float64, device="cuda")
    y = torch.zeros(2 * 16 ** 3, dtype=torch.float64, device="cuda")
    for K, B in ((15, 1), (14, 1), (1024, 1), (8, 0), (8, 70000)):   # odd, factor 7, too large, B out of range
        with pytest.raises(bnd.BDError):
            bnd.mesh_fft(K, B, "fp64", 0, x, y)
    with pytest.raises(bnd.BDError):                     # overlapping buffers
        bnd.mesh_fft(8, 1, "fp64", 0, x, x)
