"""The multi-coil tracker on the GPU (tts_set_coil_maps: Alg. 3 with C coils, §IV-B)
against the FP64 multi-coil oracle frame by frame: band-shape sizes, square and rectangular
(the fused (S1): rank-one rows generated in the row transform, rows of S stored compact),
and other sizes (explicit images, tts_fft2d, gathered rows); host rows and full device
frames; C = 1 with unit maps against the single-coil path; non-finite device frames skipped;
argument errors."""
from __future__ import annotations

import dataclasses

import numpy as np
import pytest

from oracle import multicoil as M
from oracle import tracker as O
from paper_1609_04104_gb300 import inputs
from tests.helpers import NRMSE_TOL, nrmse_per_frame

pytestmark = pytest.mark.gpu


def workload(Nx, Ny, R, T):
    return dataclasses.replace(inputs.SMALL_CINE, name=f"mc{Nx}x{Ny}", Nx=Nx, Ny=Ny, R=R, T=T, mm_iters=3,
                               rate=0.25, central_lines=4)


def run_both(tts, Nx, Ny, R, C, T, device_full=False):
    import torch
    w = workload(Nx, Ny, R, T)
    H = inputs.coil_maps(Nx, Ny, C, 1)
    Y = inputs.multicoil_kspace(w, inputs.phantom(w, T), H)          # T x C x Nx x Ny
    A0, B0 = inputs.init_factors(Nx, Ny, R, 3)
    masks = inputs.uniform_line_masks(w, T)
    ora = M.MultiCoilTracker(Nx, Ny, R, H.astype(complex), w.lambda_forget, w.mu, w.mm_iters, A=A0, B=B0)
    trk = tts.Tracker(Nx, Ny, R, w.lambda_forget, w.mu, mm_iters=w.mm_iters, central_lines=w.central_lines)
    trk.set_factors(A0, B0)
    trk.set_coil_maps(H)
    ref, out = [], []
    for t in range(T):
        rows = np.flatnonzero(masks[t])
        yr = np.ascontiguousarray(Y[t][:, rows, :])
        ref.append(ora.push_frame(yr, masks[t]))
        if device_full:
            tts.tts_push_frame(trk.h, torch.from_numpy(np.ascontiguousarray(Y[t])).cuda(),
                               torch.from_numpy(masks[t]).cuda(), full_frame=True)
        else:
            trk.push_frame(yr, masks[t])
        out.append(trk.image(t))
    trk.synchronize()
    trk.close()
    return np.array(out), np.array(ref)


@pytest.mark.parametrize("Nx,Ny,R,C", [(64, 64, 6, 4), (48, 40, 5, 3), (128, 128, 8, 8), (96, 64, 7, 3), (64, 120, 6, 2)])
def test_multicoil_matches_oracle(tts, Nx, Ny, R, C):
    out, ref = run_both(tts, Nx, Ny, R, C, 5)
    err = nrmse_per_frame(out, ref)
    assert err.max() <= NRMSE_TOL, err


def test_multicoil_full_device_frames(tts):
    out, ref = run_both(tts, 64, 48, 4, 3, 4, device_full=True)
    err = nrmse_per_frame(out, ref)
    assert err.max() <= NRMSE_TOL, err


def test_single_unit_coil_agrees_with_single_coil_path(tts):
    w = workload(64, 64, 6, 5)
    Y = inputs.kspace(w, inputs.phantom(w, w.T))
    A0, B0 = inputs.init_factors(64, 64, 6, 2)
    masks = inputs.uniform_line_masks(w, w.T)
    a = tts.Tracker(64, 64, 6, w.lambda_forget, w.mu, mm_iters=3)
    b = tts.Tracker(64, 64, 6, w.lambda_forget, w.mu, mm_iters=3)
    a.set_factors(A0, B0)
    b.set_factors(A0, B0)
    b.set_coil_maps(np.ones((1, 64, 64), np.complex64))
    for t in range(w.T):
        rows = np.flatnonzero(masks[t])
        a.push_frame(np.ascontiguousarray(Y[t][rows]), masks[t])
        b.push_frame(np.ascontiguousarray(Y[t][rows])[None], masks[t])
        xa, xb = a.image(t), b.image(t)
        assert O.nrmse(xb, xa) <= 1e-5
    b.set_coil_maps(None)   # back to the single-coil tracker
    rows = np.flatnonzero(masks[0])
    b.push_frame(np.ascontiguousarray(Y[0][rows]), masks[0])
    a.close()
    b.close()


def test_multicoil_nonfinite_device_frame_is_skipped(tts):
    import torch
    trk = tts.Tracker(32, 32, 3, 0.9, 1e-2, mm_iters=2)
    trk.set_coil_maps(inputs.coil_maps(32, 32, 2, 0))
    y = torch.zeros((2, 32, 32), dtype=torch.complex64, device="cuda")
    y[1, 0, 3] = float("nan")
    m = torch.ones(32, dtype=torch.uint8, device="cuda")
    A, B = trk.factors()
    tts.tts_push_frame(trk.h, y, m, full_frame=True)
    with pytest.raises(tts.TtsError) as ei:
        trk.synchronize()
    assert ei.value.code == tts.TTS_ENONFINITE
    A2, B2 = trk.factors()
    assert np.array_equal(A, A2) and np.array_equal(B, B2)
    trk.close()


def test_multicoil_argument_errors(tts):
    maps = inputs.coil_maps(32, 32, 2, 0)
    trk = tts.Tracker(32, 32, 3, 0.9, 1e-2, update=tts.TTS_UPDATE_JACOBI)
    with pytest.raises(tts.TtsError):
        trk.set_coil_maps(maps)
    trk.close()
    eng = tts.Engine(1 << 24, 2)
    s = eng.admit(32, 32, 3, 0.9, 1e-2)
    with pytest.raises(tts.TtsError):
        tts.tts_set_coil_maps(tts.tts_engine_handle(eng.e, s), maps)
    eng.close()
    bad = maps.copy()
    bad[0, 1, 1] = np.inf
    trk = tts.Tracker(32, 32, 3, 0.9, 1e-2)
    with pytest.raises(tts.TtsError):
        trk.set_coil_maps(bad)
    trk.close()
