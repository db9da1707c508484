"""The square form of the batched 2D DFT (tts_fft2d for square 64 ... 384: one persistent
launch over row-band and column-band tasks, the column tasks of an image waiting on its
row tasks): against the FP64 oracle's DFT, with batches smaller and much larger than the
tasks in flight (every ordering case of the task list), both directions, in place, and an
input that is not 16-byte aligned."""
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


SIZES = [64, 96, 128, 144, 160, 192, 256, 288, 320, 384]   # line lengths T x R, R in 8 ... 24


@pytest.mark.parametrize("N", SIZES)
@pytest.mark.parametrize("batch", [3, 300])
def test_square_fft_forward(tts, N, batch):
    if N >= 320 and batch > 100:
        batch = 100
    check(tts, N, batch, False, False, N + batch)


@pytest.mark.parametrize("N", SIZES)
def test_square_fft_inverse_in_place(tts, N):
    check(tts, N, 77, True, True, 5 * N)


def test_square_fft_round_trip(tts):
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


@pytest.mark.parametrize("N,batch", [(64, 1), (128, 300), (192, 150), (256, 200), (384, 60)])
def test_square_fft_every_image(tts, N, batch):
    """Every image of a batch with many more tasks than CTAs (row and column tasks of
    different images interleaved, the intermediate images in flight in L2)."""
    import torch
    rng = np.random.default_rng(N * 7 + batch)
    X = (rng.standard_normal((batch, N, N)) + 1j * rng.standard_normal((batch, N, N))).astype(np.complex64)
    x = torch.from_numpy(X).cuda()
    y = torch.empty_like(x)
    tts.tts_fft2d(x, y)
    torch.cuda.synchronize()
    got = y.cpu().numpy().astype(np.complex128)
    F = O.dft_matrix(N)
    ref = F @ X.astype(np.complex128) @ F          # F_N X F_N for every image of the batch
    err = np.linalg.norm(got - ref, axis=(1, 2)) / np.linalg.norm(ref, axis=(1, 2))
    assert err.max() <= 1e-5, (int(err.argmax()), float(err.max()))


def test_fft_unaligned_input(tts):
    """An input that is not 16-byte aligned (8 bytes past a float2 boundary)."""
    import torch
    N, batch = 64, 5
    rng = np.random.default_rng(3)
    X = (rng.standard_normal((batch, N, N)) + 1j * rng.standard_normal((batch, N, N))).astype(np.complex64)
    buf = torch.empty(batch * N * N + 1, dtype=torch.complex64, device="cuda")
    x = buf[1:].view(batch, N, N)
    assert x.data_ptr() % 16 == 8
    x.copy_(torch.from_numpy(X).cuda())
    y = torch.empty_like(x)
    tts.tts_fft2d(x, y)
    torch.cuda.synchronize()
    got = y.cpu().numpy()
    for b in range(batch):
        ref = O.fft2(X[b].astype(np.complex128))
        assert np.linalg.norm(got[b] - ref) / np.linalg.norm(ref) <= 1e-5


@pytest.mark.parametrize("N,batch", [(128, 64), (320, 24)])
def test_autotuned_launch_shape_keeps_the_transform(tts, N, batch):
    """tts_fft2d_autotune times the square kernel's launch shapes and keeps the fastest; the
    transform under the picked shape still matches the FP64 DFT (the shape changes only the
    CTAs per SM and the row-ahead lag, not the arithmetic)."""
    import torch
    pick = tts.tts_fft2d_autotune(N, batch, reps=2)
    assert pick["ms"] > 0 and pick["ctas_per_sm"] >= 1 and pick["lag_scale"] in (0.5, 1.0, 1.5, 2.0, 3.0)
    rng = np.random.default_rng(N)
    x = (rng.standard_normal((4, N, N)) + 1j * rng.standard_normal((4, N, N))).astype(np.complex64)
    xd = torch.from_numpy(x).cuda()
    out = torch.empty_like(xd)
    tts.tts_fft2d(xd, out)
    ref = np.stack([O.fft2(a.astype(np.complex128)) for a in x])
    assert O.nrmse(out.cpu().numpy(), ref) < 1e-5
