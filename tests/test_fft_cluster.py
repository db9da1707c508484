"""The single-pass cluster form of the batched 2D DFT (tts_fft2d for square 64, 128, 256):
against the FP64 oracle's DFT, with batches smaller and much larger than the number of
clusters resident on the GPU (the persistent loop and the prefetch of the next image),
both directions, and in place."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import tracker as O

pytestmark = pytest.mark.gpu


def check(tts, N, batch, inverse, inplace, seed):
    import torch
    rng = np.random.default_rng(seed)
    X = (rng.standard_normal((batch, N, N)) + 1j * rng.standard_normal((batch, N, N))).astype(np.complex64)
    x = torch.from_numpy(X).cuda()
    y = x if inplace else torch.empty_like(x)
    tts.tts_fft2d(x, y, inverse=inverse)
    torch.cuda.synchronize()
    got = y.cpu().numpy()
    f = O.ifft2 if inverse else O.fft2
    for b in sorted({0, batch // 2, batch - 1}):
        ref = f(X[b].astype(np.complex128))
        assert np.linalg.norm(got[b] - ref) / np.linalg.norm(ref) <= 1e-5, (N, batch, b)


@pytest.mark.parametrize("N", [64, 128, 256])
@pytest.mark.parametrize("batch", [3, 300])
def test_cluster_fft_forward(tts, N, batch):
    check(tts, N, batch, False, False, N + batch)


@pytest.mark.parametrize("N", [64, 256])
def test_cluster_fft_inverse_in_place(tts, N):
    check(tts, N, 77, True, True, 5 * N)


def test_cluster_fft_round_trip(tts):
    import torch
    rng = np.random.default_rng(9)
    X = (rng.standard_normal((40, 128, 128)) + 1j * rng.standard_normal((40, 128, 128))).astype(np.complex64)
    x = torch.from_numpy(X).cuda()
    y = torch.empty_like(x)
    z = torch.empty_like(x)
    tts.tts_fft2d(x, y)
    tts.tts_fft2d(y, z, inverse=True)
    torch.cuda.synchronize()
    assert np.linalg.norm(z.cpu().numpy() - X) / np.linalg.norm(X) <= 1e-6
