"""The band form of the batched 2D DFT for Nx != Ny (tts_fft2d when both line lengths have a
band shape: a row-band launch and a column-band launch per group of images that fits L2):
every image against the FP64 oracle's DFT F_Nx X F_Ny, both directions, in place, batches
that span several groups, and bands that overhang the image (Ny = 120 is 7.5 bands of 16)."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import tracker as O

pytestmark = pytest.mark.gpu


def images(batch, Nx, Ny, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((batch, Nx, Ny)) + 1j * rng.standard_normal((batch, Nx, Ny))).astype(np.complex64)


def reference(X, inverse):
    Fx, Fy = O.dft_matrix(X.shape[1]), O.dft_matrix(X.shape[2])
    if inverse:
        Fx, Fy = np.conj(Fx), np.conj(Fy)
    return Fx @ X.astype(np.complex128) @ Fy


def worst(got, ref):
    return float((np.linalg.norm(got - ref, axis=(1, 2)) / np.linalg.norm(ref, axis=(1, 2))).max())


@pytest.mark.parametrize("Nx,Ny", [(192, 120), (120, 192), (96, 384), (256, 64), (160, 320), (120, 120), (240, 240),
                                   (200, 200), (216, 216), (144, 288), (200, 120)])
@pytest.mark.parametrize("inverse", [False, True])
def test_band_fft_rectangular(tts, Nx, Ny, inverse):
    import torch
    X = images(9, Nx, Ny, Nx * 3 + Ny + inverse)
    x = torch.from_numpy(X).cuda()
    y = torch.empty_like(x)
    tts.tts_fft2d(x, y, inverse=inverse)
    torch.cuda.synchronize()
    assert worst(y.cpu().numpy(), reference(X, inverse)) <= 1e-5


def test_band_fft_groups_in_place(tts):
    """300 images of 192 x 120 (184 KB each): two groups of the L2-sized split, in place."""
    import torch
    X = images(300, 192, 120, 11)
    x = torch.from_numpy(X).cuda()
    tts.tts_fft2d(x, x)
    torch.cuda.synchronize()
    assert worst(x.cpu().numpy(), reference(X, False)) <= 1e-5


def test_band_fft_round_trip(tts):
    import torch
    X = images(17, 96, 160, 5)
    x = torch.from_numpy(X).cuda()
    y, z = torch.empty_like(x), torch.empty_like(x)
    tts.tts_fft2d(x, y)
    tts.tts_fft2d(y, z, inverse=True)
    torch.cuda.synchronize()
    assert worst(z.cpu().numpy(), X.astype(np.complex128)) <= 1e-6
