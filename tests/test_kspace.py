"""The k-space interpolation tracker on the GPU (tts_config.kspace = 1, Alg. 2) against
the FP64 k-space oracle frame by frame; against the image-domain GPU tracker under the
change of variables A1 = F A, A2 = F B; its line scores on the rows of A1; argument errors."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import kspace as K
from oracle import tracker as O
from paper_1609_04104_gb300 import inputs
from tests.helpers import NRMSE_TOL, nrmse_per_frame

pytestmark = pytest.mark.gpu


def small():
    w = inputs.scaled(inputs.SMALL_CINE, T=10)
    Y = inputs.kspace(w, inputs.phantom(w, w.T))
    A0, B0 = inputs.init_factors(w.Nx, w.Ny, w.R, w.seed)
    return w, Y, A0, B0, inputs.uniform_line_masks(w, w.T)


def test_kspace_tracker_matches_oracle(tts):
    w, Y, A0, B0, M = small()
    ora = K.KspaceTracker(w.Nx, w.Ny, w.R, w.lambda_forget, w.mu, w.mm_iters, A1=A0, A2=B0)
    trk = tts.Tracker(w.Nx, w.Ny, w.R, w.lambda_forget, w.mu, mm_iters=w.mm_iters, central_lines=w.central_lines,
                      kspace=1)
    trk.set_factors(A0, B0)
    ref, out = [], []
    for t in range(w.T):
        rows = np.flatnonzero(M[t])
        ref.append(ora.push_frame(Y[t][rows], M[t]))
        trk.push_frame(np.ascontiguousarray(Y[t][rows]), M[t])
        out.append(trk.image(t))
    err = nrmse_per_frame(np.array(out), np.array(ref))
    assert err.max() <= NRMSE_TOL, err
    p = trk.line_probs()
    assert np.allclose(p, ora.line_probs(), rtol=1e-5, atol=0)
    trk.close()


def test_kspace_equals_image_domain_path(tts):
    w, Y, A0, B0, M = small()
    img = tts.Tracker(w.Nx, w.Ny, w.R, w.lambda_forget, w.mu, mm_iters=w.mm_iters, central_lines=w.central_lines)
    img.set_factors(A0, B0)
    ks = tts.Tracker(w.Nx, w.Ny, w.R, w.lambda_forget, w.mu, mm_iters=w.mm_iters, central_lines=w.central_lines,
                     kspace=1)
    ks.set_factors((O.dft_matrix(w.Nx) @ A0).astype(np.complex64), (O.dft_matrix(w.Ny) @ B0).astype(np.complex64))
    for t in range(w.T):
        rows = np.flatnonzero(M[t])
        img.push_frame(np.ascontiguousarray(Y[t][rows]), M[t])
        ks.push_frame(np.ascontiguousarray(Y[t][rows]), M[t])
        assert O.nrmse(ks.image(t), img.image(t)) <= 1e-4
    assert np.allclose(ks.line_probs(), img.line_probs(), rtol=1e-4)
    img.close()
    ks.close()


def test_kspace_informative_sequence_runs_and_draws_exact_counts(tts):
    w = inputs.scaled(inputs.CINE256, Nx=128, Ny=128, R=16, T=8)
    Y = inputs.kspace(w, inputs.phantom(w, w.T))
    trk = tts.Tracker(w.Nx, w.Ny, w.R, w.lambda_forget, w.mu, mm_iters=w.mm_iters, kspace=1)
    for t in range(w.T):
        m = np.ones(w.Nx, np.uint8) if t < w.warmup_frames else trk.next_mask(w.rate, 7)
        if t >= w.warmup_frames:
            assert m.sum() == w.k_lines
        trk.push_frame(np.ascontiguousarray(Y[t][np.flatnonzero(m)]), m)
        assert np.isfinite(trk.image(t)).all()
    trk.close()


def test_kspace_argument_errors(tts):
    with pytest.raises(tts.TtsError):
        tts.Tracker(64, 64, 4, 0.9, 1e-2, kspace=1, row_dft=1)
    trk = tts.Tracker(32, 32, 3, 0.9, 1e-2, kspace=1)
    with pytest.raises(tts.TtsError):
        trk.set_coil_maps(inputs.coil_maps(32, 32, 2, 0))
    trk.close()
    eng = tts.Engine(1 << 24, 2)
    with pytest.raises(tts.TtsError):
        eng.admit(32, 32, 3, 0.9, 1e-2, kspace=1)
    eng.close()
