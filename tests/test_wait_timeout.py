"""Failure detection of the bounded device waits, run out on purpose without faulting or
hanging the GPU: one awaited arrival is withheld (a host-set test hook), every wait of the
launch is limited to about 1 ms of SM clock, and the kernel must give up, record the error
status the host reads, and return. The next ordinary call must succeed and match the FP64
oracle.

- the square band-task FFT: the row tasks of one image publish nothing, so the column tasks
  of that image run their wait out;
- the tensor-core DFT: one producer's bulk copy and arrival for a K' chunk are withheld, so
  the MMA issuer's wait on that stage runs out (the other producers' waits follow, every
  producer first waits for its own copies in flight, and TMEM is freed);
- the tracker with the tensor-core row transform: the frame whose transform gave up is
  skipped, tts_synchronize reports TTS_ETIMEOUT, and the next frames match the oracle run
  that skipped the same frame."""
import time

import numpy as np
import pytest

from oracle import tracker as O
from paper_1609_04104_gb300 import inputs
from tests.helpers import NRMSE_TOL, workload_inputs

pytestmark = pytest.mark.gpu

WAIT = 2_000_000   # SM clocks, about 1 ms


def cn(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


def _dft_ref(x):
    return np.stack([O.fft2(a.astype(np.complex128)) for a in x])


@pytest.mark.parametrize("N,batch,image", [(256, 6, 2), (128, 4, 0), (64, 9, 8)])
def test_square_fft_wait_runs_out_then_next_call_ok(tts, N, batch, image):
    import torch
    x = torch.from_numpy(cn(np.random.default_rng(N), batch, N, N)).cuda()
    out = torch.empty_like(x)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    t0 = time.perf_counter()
    tts.tts_test_withheld_wait(0, x, out, None, image, WAIT, status)
    torch.cuda.synchronize()
    assert time.perf_counter() - t0 < 10.0
    assert int(status.item()) == 1, "the withheld image's column tasks did not report their wait"
    tts.tts_fft2d(x, out)   # ordinary call on the same buffers and device
    torch.cuda.synchronize()
    assert O.nrmse(out.cpu().numpy(), _dft_ref(x.cpu().numpy())) < 1e-5


@pytest.mark.parametrize("N,batch,chunk", [(128, 2, 3), (256, 1, 0), (64, 3, 7)])
def test_tensor_core_dft_wait_runs_out_then_next_call_ok(tts, N, batch, chunk):
    import torch
    x = torch.from_numpy(cn(np.random.default_rng(N + 1), batch, N, N)).cuda()
    out, tmp = torch.empty_like(x), torch.empty_like(x)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    t0 = time.perf_counter()
    tts.tts_test_withheld_wait(1, x, out, tmp, chunk, WAIT, status)
    torch.cuda.synchronize()
    assert time.perf_counter() - t0 < 10.0
    assert int(status.item()) == 1, "the MMA issuer's wait on the withheld stage did not report"
    status.zero_()
    tts.tts_dft2d_gemm(x, out, tmp, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert O.nrmse(out.cpu().numpy(), _dft_ref(x.cpu().numpy())) < 1e-4


def test_tracker_frame_skipped_when_row_transform_gives_up(tts):
    w = inputs.scaled(inputs.SMALL_CINE, T=6)
    L, Y, A0, B0 = workload_inputs(w, w.T)
    masks = inputs.uniform_line_masks(w)
    trk = tts.Tracker(w.Nx, w.Ny, w.R, w.lambda_forget, w.mu, mm_iters=w.mm_iters, row_dft=tts.TTS_ROWDFT_BF16X3)
    trk.set_factors(A0, B0)
    ora = O.Tracker(w.Nx, w.Ny, w.R, w.lambda_forget, w.mu, w.mm_iters, A=A0, B=B0)
    skip = 2
    for t in range(w.T):
        y = inputs.observed_rows(Y[t], masks[t])
        if t == skip:
            before = (trk.factors(), trk.gamma(), trk.stats())
            tts.tts_test_withhold_row_transform(trk.h, 1, WAIT)
            trk.push_frame(y, masks[t])
            with pytest.raises(tts.TtsError) as e:
                trk.synchronize()
            assert e.value.code == tts.TTS_ETIMEOUT
            after = (trk.factors(), trk.gamma(), trk.stats())
            for a, b in zip(before[0], after[0]):
                assert np.array_equal(a, b)
            assert np.array_equal(before[1], after[1])
            # the surrogate statistics are untouched (t counts the pushes, this one included)
            assert all(before[2][k] == after[2][k] for k in ("abar_A", "abar_B", "w"))
            continue   # the oracle skips the same frame
        trk.push_frame(y, masks[t])
        trk.synchronize()
        ref = ora.push_frame(y, masks[t])
        assert O.nrmse(trk.image(t), ref) < NRMSE_TOL, t
    trk.close()
