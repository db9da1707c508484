"""The allocation-free frame update (tts_push_frame_noalloc) against the tracker-handle path.

It exists for callers that cannot allocate device memory while they run: code whose device
memory comes from an allocator it does not control, real-time loops sized once that must
not grow, and code that cannot take the device-wide synchronisation of cudaMalloc/cudaFree.

Kept in a file of its own that pytest collects last. It must pass alone in a fresh process
and after the other tests."""
import numpy as np
import pytest

from oracle import tracker as O
from paper_1609_04104_gb300 import inputs
from tests.helpers import NRMSE_TOL, workload_inputs

pytestmark = pytest.mark.gpu


def _state(A, B, stats, gamma):
    return A.cpu().numpy(), B.cpu().numpy(), stats.cpu().numpy(), gamma.cpu().numpy()


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
    # the allocation-free entry point on caller-held device state, every buffer made up front
    A = torch.from_numpy(A0.copy()).cuda()
    B = torch.from_numpy(B0.copy()).cuda()
    stats = torch.zeros(4, dtype=torch.float64, device="cuda")
    gamma = torch.zeros(w.R, dtype=torch.complex64, device="cuda")
    ys = [torch.from_numpy(inputs.observed_rows(Y[t], masks[t])).cuda() for t in range(2)]
    ms = [torch.from_numpy(masks[t]).cuda() for t in range(2)]
    torch.cuda.synchronize()
    alloc0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    free = []
    for t in range(2):
        y = inputs.observed_rows(Y[t], masks[t])
        trk.push_frame(y, masks[t])
        ref_img = trk.image(t)
        rA, rB = trk.factors()
        rg = trk.gamma()
        st = trk.stats()
        tts.tts_push_frame_noalloc(A, B, stats, gamma, ys[t], ms[t], w.lambda_forget, w.mu, w.mm_iters)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        a, b, s, g = _state(A, B, stats, gamma)
        img = a @ np.diag(g) @ b.T
        assert O.nrmse(img, ref_img) < NRMSE_TOL
        np.testing.assert_allclose(a, rA, rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(b, rB, rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(g, rg, rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(s, [st["w"], st["abar_A"], st["abar_B"], st["t"]], rtol=1e-6)
    # no device memory was taken by the calls: torch's allocator made no allocation, and the
    # device's free memory after the second call equals that after the first (the first
    # call on a device may load the library's kernels)
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == alloc0
    assert free[1] == free[0]


def test_noalloc_skips_a_nonfinite_frame_and_keeps_the_state(tts):
    import torch
    w = inputs.scaled(inputs.SMALL_CINE, T=2)
    masks = inputs.uniform_line_masks(w)
    L, Y, A0, B0 = workload_inputs(w, w.T)
    A = torch.from_numpy(A0.copy()).cuda()
    B = torch.from_numpy(B0.copy()).cuda()
    stats = torch.zeros(4, dtype=torch.float64, device="cuda")
    gamma = torch.zeros(w.R, dtype=torch.complex64, device="cuda")
    y0 = inputs.observed_rows(Y[0], masks[0])
    tts.tts_push_frame_noalloc(A, B, stats, gamma, torch.from_numpy(y0).cuda(), torch.from_numpy(masks[0]).cuda(),
                               w.lambda_forget, w.mu, w.mm_iters)
    torch.cuda.synchronize()
    before = _state(A, B, stats, gamma)
    y1 = inputs.observed_rows(Y[1], masks[1]).copy()
    y1[1, 3] = np.nan   # one non-finite sample, made on the host
    tts.tts_push_frame_noalloc(A, B, stats, gamma, torch.from_numpy(y1).cuda(), torch.from_numpy(masks[1]).cuda(),
                               w.lambda_forget, w.mu, w.mm_iters)
    torch.cuda.synchronize()
    after = _state(A, B, stats, gamma)
    for x, y in zip(before, after):
        assert np.array_equal(x.view(np.uint8), y.view(np.uint8))
    assert after[2][3] == 1.0   # frames processed did not advance: the frame was skipped
    # the next good frame is processed as usual
    y1[1, 3] = 0
    tts.tts_push_frame_noalloc(A, B, stats, gamma, torch.from_numpy(y1).cuda(), torch.from_numpy(masks[1]).cuda(),
                               w.lambda_forget, w.mu, w.mm_iters)
    torch.cuda.synchronize()
    assert stats.cpu().numpy()[3] == 2.0


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


def test_noalloc_rejects_mismatched_buffers_on_the_host(tts):
    """Wrong dtypes and short buffers are refused before any device call."""
    import torch
    d = "cuda"
    Nx, Ny, R = 32, 48, 4
    good = dict(A=torch.zeros((Nx, R), dtype=torch.complex64, device=d),
                B=torch.zeros((Ny, R), dtype=torch.complex64, device=d),
                stats=torch.zeros(4, dtype=torch.float64, device=d),
                gamma=torch.zeros(R, dtype=torch.complex64, device=d),
                y_rows=torch.zeros((Nx, Ny), dtype=torch.complex64, device=d),
                line_mask=torch.ones(Nx, dtype=torch.uint8, device=d))
    bad = [("stats", torch.zeros(4, dtype=torch.float32, device=d)),
           ("stats", torch.zeros(3, dtype=torch.float64, device=d)),
           ("line_mask", torch.ones(Nx - 1, dtype=torch.uint8, device=d)),
           ("line_mask", torch.ones(Nx, dtype=torch.int32, device=d)),
           ("gamma", torch.zeros(R - 1, dtype=torch.complex64, device=d)),
           ("B", torch.zeros((Ny, R + 1), dtype=torch.complex64, device=d)),
           ("A", torch.zeros((Nx, R), dtype=torch.complex128, device=d)),
           ("y_rows", torch.zeros((Nx - 1, Ny), dtype=torch.complex64, device=d))]
    for key, val in bad:
        args = dict(good)
        args[key] = val
        with pytest.raises(ValueError):
            tts.tts_push_frame_noalloc(args["A"], args["B"], args["stats"], args["gamma"], args["y_rows"],
                                       args["line_mask"], 0.9, 1e-2)
