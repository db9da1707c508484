"""The allocation-free frame update (tts_push_frame_noalloc), for callers that cannot
allocate device memory while they run, against the tracker-handle path.

Kept in a file of its own that pytest collects last. It must pass alone in a fresh
process and after the other tests."""
import numpy as np
import pytest

from oracle import tracker as O
from paper_1609_04104_gb300 import inputs
from tests.helpers import NRMSE_TOL, workload_inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["small", "limit"])
def test_noalloc_matches_handle_path_two_calls(tts, name):
    import torch
    if name == "small":
        w = inputs.scaled(inputs.SMALL_CINE, T=2)
        masks = inputs.uniform_line_masks(w)
    else:   # at the size limit of the fixed scratch: 256 x 256, R = 32, full then 1/8 sampling
        w = inputs.scaled(inputs.CINE256, T=2)
        masks = np.ones((2, w.Nx), np.uint8)
        masks[1] = inputs.uniform_line_masks(inputs.scaled(w, policy="uniform", warmup_frames=0), 2)[1]
    L, Y, A0, B0 = workload_inputs(w, w.T)
    # existing entry point: a tracker handle
    trk = tts.Tracker(w.Nx, w.Ny, w.R, w.lambda_forget, w.mu, mm_iters=w.mm_iters)
    trk.set_factors(A0, B0)
    # the allocation-free entry point on caller-held device state
    A = torch.from_numpy(A0.copy()).cuda()
    B = torch.from_numpy(B0.copy()).cuda()
    stats = torch.zeros(4, dtype=torch.float64, device="cuda")
    gamma = torch.zeros(w.R, dtype=torch.complex64, device="cuda")
    for t in range(2):
        y = inputs.observed_rows(Y[t], masks[t])
        trk.push_frame(y, masks[t])
        ref_img = trk.image(t)
        rA, rB = trk.factors()
        rg = trk.gamma()
        st = trk.stats()
        tts.tts_push_frame_noalloc(A, B, stats, gamma, torch.from_numpy(y).cuda(), torch.from_numpy(masks[t]).cuda(),
                                   w.lambda_forget, w.mu, w.mm_iters)
        torch.cuda.synchronize()
        a, b, g = A.cpu().numpy(), B.cpu().numpy(), gamma.cpu().numpy()
        img = a @ np.diag(g) @ b.T
        assert O.nrmse(img, ref_img) < NRMSE_TOL
        np.testing.assert_allclose(a, rA, rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(b, rB, rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(g, rg, rtol=1e-5, atol=1e-6)
        s = stats.cpu().numpy()
        np.testing.assert_allclose(s, [st["w"], st["abar_A"], st["abar_B"], st["t"]], rtol=1e-6)


def test_noalloc_rejects_sizes_beyond_the_scratch(tts):
    import torch
    A = torch.zeros((320, 8), dtype=torch.complex64, device="cuda")
    B = torch.zeros((64, 8), dtype=torch.complex64, device="cuda")
    stats = torch.zeros(4, dtype=torch.float64, device="cuda")
    gamma = torch.zeros(8, dtype=torch.complex64, device="cuda")
    y = torch.zeros((8, 64), dtype=torch.complex64, device="cuda")
    m = torch.zeros(320, dtype=torch.uint8, device="cuda")
    with pytest.raises(tts.TtsError) as e:
        tts.tts_push_frame_noalloc(A, B, stats, gamma, y, m, 0.9, 1e-2)
    assert e.value.code == tts.TTS_EINVAL and "scratch" in tts.tts_last_error()
