"""Host frames through tts_push_frame: the library gathers the acquired rows into its pinned
staging (checking them for NaN/Inf), which the kernels read in place. A full host frame with the mask
of the last draw (line_mask NULL, read from the device copy) must give bit-identical results
to the acquired rows gathered by the caller with the mask given; a NaN/Inf in a row that was
not acquired is never read; one in an acquired row refuses the frame with nothing applied;
a checkpoint restores the drawn mask for a push without a mask. A frame in page-locked memory
pushed with TTS_HOST_PINNED is read in place by the kernels and gives the same bits as the
gathered frame; a NaN in it is found on the device and reported by the next synchronising call;
pageable memory with that flag is refused."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1609_04104_gb300 import inputs

pytestmark = pytest.mark.gpu


def small():
    w = inputs.SMALL_CINE
    T = 12
    Y = inputs.kspace(w, inputs.phantom(w, T))
    A0, B0 = inputs.init_factors(w.Nx, w.Ny, w.R, w.seed)
    return w, T, Y, A0, B0


def tracker(tts, w, A0, B0):
    trk = tts.Tracker(w.Nx, w.Ny, w.R, w.lambda_forget, w.mu, mm_iters=w.mm_iters, central_lines=w.central_lines,
                      policy=tts.TTS_POLICY_INFORMATIVE)
    trk.set_factors(A0, B0)
    return trk


def test_full_host_frame_with_drawn_mask_matches_gathered_rows(tts):
    w, T, Y, A0, B0 = small()
    a, b = tracker(tts, w, A0, B0), tracker(tts, w, A0, B0)
    full = np.ones(w.Nx, np.uint8)
    for t in range(T):
        if t < 3:
            ma = mb = full
            a.push_frame(np.ascontiguousarray(Y[t]), ma)
            b.push_frame(np.ascontiguousarray(Y[t]), full, full_frame=True)
        else:
            ma = a.next_mask(1 / 4, 5)
            mb = b.next_mask(1 / 4, 5)
            np.testing.assert_array_equal(ma, mb)
            a.push_frame(inputs.observed_rows(Y[t], ma), ma)        # caller gathers, mask given
            b.push_frame(np.ascontiguousarray(Y[t]), None, full_frame=True)   # library gathers
        xa, xb = a.image(t), b.image(t)
        assert np.array_equal(xa.view(np.uint32), xb.view(np.uint32)), t
    a.close()
    b.close()


def test_nonfinite_only_refused_in_acquired_rows(tts):
    w, T, Y, A0, B0 = small()
    trk = tracker(tts, w, A0, B0)
    trk.push_frame(np.ascontiguousarray(Y[0]), np.ones(w.Nx, np.uint8), full_frame=True)
    m = trk.next_mask(1 / 4, 9)
    f = np.ascontiguousarray(Y[1]).copy()
    skipped = np.flatnonzero(m == 0)[0]
    f[skipped, 3] = np.nan                                   # never read
    trk.push_frame(f, None, full_frame=True)
    assert trk.stats()["t"] == 2
    m2 = trk.next_mask(1 / 4, 9)
    g = np.ascontiguousarray(Y[2]).copy()
    g[np.flatnonzero(m2)[1], 5] = np.inf                     # an acquired row
    with pytest.raises(tts.TtsError) as e:
        trk.push_frame(g, None, full_frame=True)
    assert e.value.code == tts.TTS_ENONFINITE
    assert trk.stats()["t"] == 2                             # nothing applied
    trk.push_frame(np.ascontiguousarray(Y[2]), None, full_frame=True)   # the same draw still stands
    assert trk.stats()["t"] == 3
    trk.close()


def test_checkpoint_restores_the_drawn_mask_for_a_push_without_mask(tts):
    w, T, Y, A0, B0 = small()
    a = tracker(tts, w, A0, B0)
    for t in range(3):
        a.push_frame(np.ascontiguousarray(Y[t]), np.ones(w.Nx, np.uint8), full_frame=True)
    m = a.next_mask(1 / 4, 21)
    blob = a.save()
    b = tracker(tts, w, A0, B0)
    b.next_mask(1 / 2, 99)                                   # a different draw, then overwritten
    b.load(blob)
    a.push_frame(np.ascontiguousarray(Y[3]), None, full_frame=True)
    b.push_frame(np.ascontiguousarray(Y[3]), None, full_frame=True)
    assert np.array_equal(a.image(3).view(np.uint32), b.image(3).view(np.uint32))
    a.close()
    b.close()


def pinned_copy(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()


def test_pinned_frame_read_in_place_matches_gathered(tts):
    w, T, Y, A0, B0 = small()
    a, b = tracker(tts, w, A0, B0), tracker(tts, w, A0, B0)
    full = np.ones(w.Nx, np.uint8)
    Yp = pinned_copy(Y)
    for t in range(T):
        if t < 3:
            a.push_frame(np.ascontiguousarray(Y[t]), full, full_frame=True)
            b.push_frame(Yp[t], full, full_frame=True, pinned=True)
        else:
            ma, mb = a.next_mask(1 / 4, 5), b.next_mask(1 / 4, 5)
            np.testing.assert_array_equal(ma, mb)
            a.push_frame(np.ascontiguousarray(Y[t]), None, full_frame=True)
            b.push_frame(Yp[t], None, full_frame=True, pinned=True)
            # acquired rows only, pinned too
        xa, xb = a.image(t), b.image(t)
        assert np.array_equal(xa.view(np.uint32), xb.view(np.uint32)), t
    # compact rows (|S| x Ny) with the mask given
    m = a.next_mask(1 / 4, 6)
    b.next_mask(1 / 4, 6)
    rows = inputs.observed_rows(Y[T - 1], m)
    a.push_frame(rows, m)
    b.push_frame(pinned_copy(rows), m, pinned=True)
    assert np.array_equal(a.image().view(np.uint32), b.image().view(np.uint32))
    a.close()
    b.close()


def test_pinned_frame_nonfinite_reported_on_synchronize(tts):
    w, T, Y, A0, B0 = small()
    trk = tracker(tts, w, A0, B0)
    trk.push_frame(np.ascontiguousarray(Y[0]), np.ones(w.Nx, np.uint8), full_frame=True)
    A1, B1 = trk.factors()
    m = trk.next_mask(1 / 4, 9)
    g = pinned_copy(Y[1])
    g[np.flatnonzero(m)[1], 5] = np.nan                      # an acquired row
    trk.push_frame(g, None, full_frame=True, pinned=True)   # read on the device
    with pytest.raises(tts.TtsError) as e:
        trk.synchronize()
    assert e.value.code == tts.TTS_ENONFINITE
    A2, B2 = trk.factors()
    np.testing.assert_array_equal(A1, A2)
    np.testing.assert_array_equal(B1, B2)
    with pytest.raises(tts.TtsError) as e:                   # pageable memory is refused
        trk.push_frame(np.ascontiguousarray(Y[1]), None, full_frame=True, pinned=True)
    assert e.value.code == tts.TTS_EINVAL
    trk.push_frame(np.ascontiguousarray(Y[1]), None, full_frame=True)
    assert np.isfinite(trk.image()).all()
    trk.close()
