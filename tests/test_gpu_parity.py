"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same seeded
inputs. Image bound: per-frame NRMSE <= 1e-4 (FP32 path vs FP64 oracle). FP64 ridge
solve: gamma within 1e-10 relative when both sides solve the same system."""
import numpy as np
import pytest

from oracle import tracker as O
from paper_1609_04104_gb300 import inputs
from tests.helpers import NRMSE_TOL, nrmse_per_frame, run_gpu, run_oracle, workload_inputs

pytestmark = pytest.mark.gpu


def cn(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


# ----------------------------------------------------------------------------------
# batched 2D DFT
# ----------------------------------------------------------------------------------
@pytest.mark.parametrize("batch,Nx,Ny", [(1, 1, 1), (3, 6, 10), (2, 15, 9), (4, 64, 64), (2, 160, 192),
                                         (1, 256, 256), (1, 320, 384), (1, 512, 512), (5, 384, 128)])
@pytest.mark.parametrize("inverse", [False, True])
def test_fft2d_matches_oracle_dft(tts, batch, Nx, Ny, inverse):
    import torch
    rng = np.random.default_rng(Nx * 7 + Ny)
    x = cn(rng, batch, Nx, Ny).astype(np.complex64)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    tts.tts_fft2d(xd, yd, inverse=inverse)
    y = yd.cpu().numpy()
    for b in range(batch):
        ref = O.ifft2(x[b].astype(np.complex128)) if inverse else O.fft2(x[b].astype(np.complex128))
        assert O.nrmse(y[b], ref) < 1e-5
        assert np.max(np.abs(y[b] - ref)) < 1e-5 * max(1.0, np.max(np.abs(ref))) * np.sqrt(Nx * Ny) ** 0.5
    # in place
    tts.tts_fft2d(xd, xd, inverse=inverse)
    np.testing.assert_array_equal(xd.cpu().numpy(), y)


# ----------------------------------------------------------------------------------
# line draws: bit-exact given identical probabilities
# ----------------------------------------------------------------------------------
def _prob_cases():
    rng = np.random.default_rng(42)
    cases = []
    for Nx in (1, 8, 13, 64, 200, 256, 384, 512):
        p = rng.uniform(0, 1, Nx) ** 4
        p /= p.sum()
        cases.append(p)
    p = 1.0 / (1.0 + np.minimum(np.arange(64), 64 - np.arange(64)))
    cases.append(p / p.sum())
    k = np.array([0, 3, 0, 1, 0, 0, 4, 2, 0, 0] * 4, float)     # tiny integer weights
    cases.append(k * 2.0 ** -52)
    z = np.zeros(32); z[10] = z[20] = 0.5                         # forces the fallback fill
    cases.append(z)
    return cases


@pytest.mark.parametrize("ci", range(11))
def test_line_draws_bit_exact(tts, ci):
    p = _prob_cases()[ci]
    Nx = len(p)
    for seed, ctr in ((0, 0), (7, 123), (2 ** 40 + 5, 2 ** 41 + 3), (99, (5 << 40) | 17)):
        for k_lines in sorted({1, min(Nx, 4), max(1, Nx // 8), max(1, Nx // 4), Nx, Nx + 3}):
            for central in sorted({0, min(8, Nx), min(3, Nx)}):
                for wr in (False, True):
                    ref = O.sample_lines_from_probs(p, k_lines, central, seed, ctr, wr)
                    got = tts.tts_sample_lines_from_probs(p, k_lines, central, seed, ctr, wr)
                    np.testing.assert_array_equal(got, ref, err_msg=f"Nx={Nx} k={k_lines} c={central} "
                                                                     f"seed={seed} ctr={ctr} wr={wr}")


def test_line_draws_device_pointers(tts):
    import torch
    p = _prob_cases()[5]
    ref = O.sample_lines_from_probs(p, 32, 8, 3, 77)
    pd = torch.from_numpy(p).cuda()
    out = torch.zeros(len(p), dtype=torch.uint8, device="cuda")
    tts.tts_sample_lines_from_probs(pd, 32, 8, 3, 77, False, out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), ref)


# ----------------------------------------------------------------------------------
# scores (probabilities) of the current subspace
# ----------------------------------------------------------------------------------
@pytest.mark.parametrize("Nx,Ny,R", [(64, 64, 8), (256, 256, 32), (192, 160, 48), (60, 45, 5), (384, 384, 64),
                                    (120, 96, 16), (160, 128, 24), (216, 144, 16), (200, 64, 8)])
def test_informative_probs_match_oracle(tts, Nx, Ny, R):
    rng = np.random.default_rng(Nx + R)
    A = cn(rng, Nx, R).astype(np.complex64)
    A[:, 0] *= 5.0
    B = cn(rng, Ny, R).astype(np.complex64)
    if R > 2:
        A[:, 2] = 0                                   # a zero column scores uniformly
    trk = tts.Tracker(Nx, Ny, R, 0.9, 1e-2)
    trk.set_factors(A, B)
    p = trk.line_probs()
    ref = O.informative_line_probs(A.astype(np.complex128), Ny)
    np.testing.assert_allclose(p, ref, rtol=2e-5, atol=0)
    assert abs(p.sum() - 1.0) < 1e-5
    # the fused score + draw equals the oracle's draw on the device's own scores
    m = trk.next_mask(1 / 8, 11)
    ref_m = O.sample_lines_from_probs(p, max(8, int(np.floor(Nx / 8 + 0.5))), 8, 11, O.line_draw_counter(0))
    np.testing.assert_array_equal(m, ref_m)


@pytest.mark.parametrize("policy,alpha", [(0, -1.0), (1, -1.0), (1, -0.5)])
def test_fixed_policy_probs(tts, policy, alpha):
    Nx = 96
    trk = tts.Tracker(Nx, 32, 4, 0.9, 1e-2, policy=policy, vd_alpha=alpha)
    p = trk.line_probs()
    ref = O.uniform_line_probs(Nx) if policy == 0 else O.vardens_line_probs(Nx, alpha)
    np.testing.assert_allclose(p, ref, rtol=1e-14)
    m = trk.next_mask(0.25, 5)
    np.testing.assert_array_equal(m, O.sample_lines_from_probs(p, 24, 8, 5, O.line_draw_counter(0)))


# ----------------------------------------------------------------------------------
# tracker trajectories
# ----------------------------------------------------------------------------------
SMALL = inputs.SMALL_CINE


@pytest.mark.parametrize("launch,C", [(0, 1), (0, 2), (0, 4), (0, 8), (1, 8), (1, 3)])
def test_small_cine_free_running(tts, launch, C):
    """64x64, R=8, 5 MM iterations, lambda 0.9, 25 % uniform lines: all 50 frames."""
    w = SMALL
    L, Y, A0, B0 = workload_inputs(w, w.T)
    masks = inputs.uniform_line_masks(w)
    ref, _, _ = run_oracle(w, w.T, Y, A0, B0, masks=masks)
    trk, got = run_gpu(tts, w, w.T, Y, A0, B0, masks, launch=launch, cluster_ctas=C)
    err = nrmse_per_frame(got, ref)
    assert err.max() < NRMSE_TOL, err
    st = trk.stats()
    tr = O.Tracker(w.Nx, w.Ny, w.R, w.lambda_forget, w.mu, w.mm_iters, A=A0, B=B0)
    for t in range(w.T):
        tr.push_frame(inputs.observed_rows(Y[t], masks[t]), masks[t])
    assert st["t"] == w.T
    np.testing.assert_allclose([st["abar_A"], st["abar_B"], st["w"]], [tr.abar_A, tr.abar_B, tr.w], rtol=1e-4)


def test_small_cine_jacobi(tts):
    w = inputs.scaled(SMALL, T=20)
    L, Y, A0, B0 = workload_inputs(w, w.T)
    masks = inputs.uniform_line_masks(w)
    ref, _, _ = run_oracle(w, w.T, Y, A0, B0, masks=masks, update="jacobi")
    _, got = run_gpu(tts, w, w.T, Y, A0, B0, masks, update=1)
    assert nrmse_per_frame(got, ref).max() < NRMSE_TOL


@pytest.mark.parametrize("Nx,Ny,R", [(128, 128, 16), (64, 192, 12)])
def test_band_row_transform_lengths(tts, Nx, Ny, R):
    """Line lengths whose acquired rows the frame kernel transforms with the register
    four-step FFT (Ny = 128: eight threads a row; 192: sixteen; 256 is the cine workload),
    fully sampled and undersampled frames, against the FP64 oracle."""
    w = inputs.Workload(name="band", Nx=Nx, Ny=Ny, R=R, T=5, n_ellipses=4, sigma=0.01, lambda_forget=0.9,
                        mu=1e-2, mm_iters=2, policy="uniform", rate=0.25, central_lines=8, seed=5)
    L, Y, A0, B0 = workload_inputs(w, w.T)
    masks = inputs.uniform_line_masks(w)
    masks[0] = 1
    ref, _, _ = run_oracle(w, w.T, Y, A0, B0, masks=masks)
    _, got = run_gpu(tts, w, w.T, Y, A0, B0, masks)
    assert nrmse_per_frame(got, ref).max() < NRMSE_TOL


@pytest.mark.parametrize("Nx,Ny,R,K,C", [(60, 45, 5, 2, 4), (30, 50, 1, 3, 2), (64, 32, 33, 2, 8),
                                         (48, 40, 48, 1, 16), (40, 24, 64, 2, 5), (16, 16, 3, 4, 16)])
def test_ragged_shapes(tts, Nx, Ny, R, K, C):
    """Non-square grids, R across the 32-lane boundary, cluster sizes that do not divide
    the rows, a single acquired line, and full sampling."""
    rng = np.random.default_rng(Nx * Ny + R)
    w = inputs.Workload(name="ragged", Nx=Nx, Ny=Ny, R=R, T=6, n_ellipses=4, sigma=0.01, lambda_forget=0.85,
                        mu=1e-2, mm_iters=K, policy="uniform", rate=0.3, central_lines=min(8, Nx), seed=3)
    L, Y, A0, B0 = workload_inputs(w, w.T)
    masks = inputs.uniform_line_masks(w)
    masks[1] = 0
    masks[1, rng.integers(Nx)] = 1                       # one line
    masks[2] = 1                                          # all lines
    ref, _, _ = run_oracle(w, w.T, Y, A0, B0, masks=masks)
    _, got = run_gpu(tts, w, w.T, Y, A0, B0, masks, cluster_ctas=C)
    assert nrmse_per_frame(got, ref).max() < NRMSE_TOL


def test_cine256_informative_full_size(tts):
    """256x256, R=32, K=3, lambda 0.95, 5 fully sampled frames then informative lines at
    1/8 (the oracle's own draws, fed to both sides); default fused launch, as timed."""
    w = inputs.CINE256
    T = 14
    L, Y, A0, B0 = workload_inputs(w, T)
    ref, masks, _ = run_oracle(w, T, Y, A0, B0)
    assert all(int(m.sum()) == w.k_lines for m in masks[w.warmup_frames:])
    _, got = run_gpu(tts, w, T, Y, A0, B0, masks)
    err = nrmse_per_frame(got, ref)
    assert err.max() < NRMSE_TOL, err


def test_teacher_forced_frame_from_oracle_state(tts):
    """Each frame starts the GPU from the oracle's state (factors and statistics):
    isolates the per-frame error from trajectory drift."""
    w = inputs.scaled(inputs.CINE256, T=9)
    L, Y, A0, B0 = workload_inputs(w, w.T)
    ref, masks, states = run_oracle(w, w.T, Y, A0, B0)
    trk = tts.Tracker(w.Nx, w.Ny, w.R, w.lambda_forget, w.mu, mm_iters=w.mm_iters)
    for t in (0, 5, 8):
        st = states[t]
        trk.set_factors(st["A"].astype(np.complex64), st["B"].astype(np.complex64))
        trk.set_stats(st["abar_A"], st["abar_B"], st["w"], t)
        trk.push_frame(inputs.observed_rows(Y[t], masks[t]), masks[t])
        assert O.nrmse(trk.image(t), ref[t]) < NRMSE_TOL / 10


def test_ridge_solve_fp64(tts):
    """Given the same factors, one MM iteration's gamma matches the oracle's FP64 ridge
    solve of the same system to the accuracy of the FP32 Gram entries."""
    rng = np.random.default_rng(12)
    Nx, Ny, R = 32, 24, 6
    A = cn(rng, Nx, R).astype(np.complex64)
    B = cn(rng, Ny, R).astype(np.complex64)
    mask = np.zeros(Nx, np.uint8); mask[[0, 1, 5, 9, 30, 31]] = 1
    Yf = O.fft2(cn(rng, Nx, Ny))
    rows = np.flatnonzero(mask)
    trk = tts.Tracker(Nx, Ny, R, 1.0, 0.3, mm_iters=1)
    trk.set_factors(A, B)
    trk.push_frame(Yf[rows].astype(np.complex64), mask)
    g = trk.gamma()
    Phi = O.phi_matrix(A.astype(np.complex128), B.astype(np.complex128), rows)
    ref = O.ridge_gamma(Phi, Yf[rows].astype(np.complex64).astype(np.complex128).reshape(-1), 0.3)
    assert np.linalg.norm(g - ref) / np.linalg.norm(ref) < 1e-5


# ----------------------------------------------------------------------------------
# API behaviour
# ----------------------------------------------------------------------------------
def test_image_range_and_errors(tts):
    trk = tts.Tracker(32, 32, 4, 0.9, 1e-2)
    with pytest.raises(tts.TtsError) as e:
        trk.image(0)
    assert e.value.code == tts.TTS_ERANGE
    y = np.zeros((4, 32), np.complex64)
    m = np.zeros(32, np.uint8); m[:4] = 1
    trk.push_frame(y, m)
    trk.image(0)
    with pytest.raises(tts.TtsError) as e:
        trk.image(1)
    assert e.value.code == tts.TTS_ERANGE
    with pytest.raises(tts.TtsError) as e:
        trk.push_frame(y, np.zeros(32, np.uint8))
    assert e.value.code == tts.TTS_EINVAL
    with pytest.raises(tts.TtsError) as e:
        trk.next_mask(0.0, 1)
    assert e.value.code == tts.TTS_EINVAL
    trk2 = tts.Tracker(32, 32, 4, 0.9, 1e-2)
    with pytest.raises(tts.TtsError) as e:
        trk2.push_frame(y, None)
    assert e.value.code == tts.TTS_ESTATE


def test_nonfinite_frame_rejected_host_and_device(tts):
    import torch
    rng = np.random.default_rng(1)
    trk = tts.Tracker(32, 32, 4, 0.9, 1e-2)
    m = np.zeros(32, np.uint8); m[[0, 3, 7, 31]] = 1
    y = cn(rng, 4, 32).astype(np.complex64)
    trk.push_frame(y, m)
    A1, B1 = trk.factors()
    bad = y.copy(); bad[2, 5] = np.nan
    with pytest.raises(tts.TtsError) as e:
        trk.push_frame(bad, m)
    assert e.value.code == tts.TTS_ENONFINITE
    # device pointers: the device skips the frame and reports it on synchronize
    tts.tts_push_frame(trk.h, torch.from_numpy(bad).cuda(), torch.from_numpy(m).cuda())
    with pytest.raises(tts.TtsError) as e:
        trk.synchronize()
    assert e.value.code == tts.TTS_ENONFINITE
    A2, B2 = trk.factors()
    np.testing.assert_array_equal(A1, A2)
    np.testing.assert_array_equal(B1, B2)
    trk.synchronize()                                  # reported once
    # the tracker keeps working
    trk.push_frame(y, m)
    assert np.isfinite(trk.image()).all()


def test_device_pointer_push_equals_host_push(tts):
    import torch
    w = inputs.scaled(SMALL, T=6)
    L, Y, A0, B0 = workload_inputs(w, w.T)
    masks = inputs.uniform_line_masks(w)
    _, ref = run_gpu(tts, w, w.T, Y, A0, B0, masks)
    trk = tts.Tracker(w.Nx, w.Ny, w.R, w.lambda_forget, w.mu, mm_iters=w.mm_iters)
    trk.set_factors(A0, B0)
    out = torch.empty((w.Nx, w.Ny), dtype=torch.complex64, device="cuda")
    for t in range(w.T):
        yd = torch.from_numpy(inputs.observed_rows(Y[t], masks[t])).cuda()
        md = torch.from_numpy(masks[t]).cuda()
        tts.tts_push_frame(trk.h, yd, md)
        tts.tts_image(trk.h, t, out)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), ref[t])


def test_save_load_resume_bit_identical(tts):
    w = inputs.scaled(SMALL, T=10)
    L, Y, A0, B0 = workload_inputs(w, w.T)
    masks = inputs.uniform_line_masks(w)
    _, ref = run_gpu(tts, w, w.T, Y, A0, B0, masks)
    a = tts.Tracker(w.Nx, w.Ny, w.R, w.lambda_forget, w.mu, mm_iters=w.mm_iters)
    a.set_factors(A0, B0)
    for t in range(5):
        a.push_frame(inputs.observed_rows(Y[t], masks[t]), masks[t])
    blob = a.save()
    b = tts.Tracker(w.Nx, w.Ny, w.R, w.lambda_forget, w.mu, mm_iters=w.mm_iters)
    b.load(blob)
    for t in range(5, w.T):
        b.push_frame(inputs.observed_rows(Y[t], masks[t]), masks[t])
        np.testing.assert_array_equal(b.image(t), ref[t])


def test_streams_isolated_alone_and_interleaved(tts):
    """Two trackers interleaved on their own streams give the same images as each alone."""
    ws = [inputs.scaled(SMALL, T=8, seed=1), inputs.scaled(SMALL, T=8, seed=2, Nx=48, Ny=40, R=5)]
    data = []
    for w in ws:
        L, Y, A0, B0 = workload_inputs(w, w.T)
        masks = inputs.uniform_line_masks(w)
        _, alone = run_gpu(tts, w, w.T, Y, A0, B0, masks)
        data.append((w, Y, A0, B0, masks, alone))
    trks = []
    for k, (w, Y, A0, B0, masks, _) in enumerate(data):
        t_ = tts.Tracker(w.Nx, w.Ny, w.R, w.lambda_forget, w.mu, mm_iters=w.mm_iters, stream_id=k)
        t_.set_factors(A0, B0)
        trks.append(t_)
    for t in range(8):
        for k, (w, Y, A0, B0, masks, alone) in enumerate(data):
            trks[k].push_frame(inputs.observed_rows(Y[t], masks[t]), masks[t])
        for k, (w, Y, A0, B0, masks, alone) in enumerate(data):
            np.testing.assert_array_equal(trks[k].image(t), alone[t])


@pytest.mark.parametrize("R,cond", [(1, 1.0), (8, 1e3), (32, 1e5), (33, 1e4), (48, 1e6), (64, 1e4)])
def test_ridge_ldl_fp64_matches_oracle(tts, R, cond):
    """The device FP64 LDL^H solve of a given system matches the oracle's FP64 Cholesky
    solve to 1e-10 relative (both solve the same G, h)."""
    rng = np.random.default_rng(R)
    Qm, _ = np.linalg.qr(cn(rng, R, R))
    ev = np.geomspace(1.0, 1.0 / cond, R)
    G = (Qm * ev) @ Qm.conj().T
    G = 0.5 * (G + G.conj().T)
    h = cn(rng, R)
    g = tts.tts_ridge_solve(G, h)
    ref = O.cholesky_solve(G, h)
    assert np.linalg.norm(g - ref) / np.linalg.norm(ref) < 1e-10 * max(1.0, cond / 1e4)


def test_full_frame_push_equals_row_push(tts):
    import torch
    w = inputs.scaled(SMALL, T=5)
    L, Y, A0, B0 = workload_inputs(w, w.T)
    masks = inputs.uniform_line_masks(w)
    _, ref = run_gpu(tts, w, w.T, Y, A0, B0, masks)
    for device in (False, True):
        trk = tts.Tracker(w.Nx, w.Ny, w.R, w.lambda_forget, w.mu, mm_iters=w.mm_iters)
        trk.set_factors(A0, B0)
        for t in range(w.T):
            if device:
                tts.tts_push_frame(trk.h, torch.from_numpy(Y[t]).cuda(), torch.from_numpy(masks[t]).cuda(),
                                   full_frame=True)
            else:
                tts.tts_push_frame(trk.h, np.ascontiguousarray(Y[t]), masks[t], full_frame=True)
            np.testing.assert_array_equal(trk.image(t), ref[t])


def test_frame_without_lines_device_mask(tts):
    """A device line mask may select no line (a host mask with none is refused with
    TTS_EINVAL): the frame then runs with |S| = 0, so gamma_t = 0, the image is exactly zero
    and the factors take the data-free MM step; the frames after it stay within the image
    bound of the oracle run through the same masks."""
    import torch
    w = inputs.scaled(SMALL, T=8)
    L, Y, A0, B0 = workload_inputs(w, w.T)
    masks = inputs.uniform_line_masks(w)[: w.T].copy()
    masks[3] = 0
    ref, _, _ = run_oracle(w, w.T, Y, A0, B0, masks=masks)
    trk = tts.Tracker(w.Nx, w.Ny, w.R, w.lambda_forget, w.mu, mm_iters=w.mm_iters, central_lines=w.central_lines)
    trk.set_factors(A0, B0)
    out = torch.empty((w.Nx, w.Ny), dtype=torch.complex64, device="cuda")
    got = []
    for t in range(w.T):
        rows = inputs.observed_rows(Y[t], masks[t])
        if len(rows) == 0:
            rows = np.zeros((1, w.Ny), np.complex64)         # never read
        yd = torch.from_numpy(np.ascontiguousarray(rows, np.complex64)).cuda()
        md = torch.from_numpy(masks[t]).cuda()
        tts.tts_push_frame(trk.h, yd, md)
        tts.tts_image(trk.h, t, out)
        torch.cuda.synchronize()
        got.append(out.cpu().numpy())
        if t == 3:
            assert np.all(trk.gamma() == 0)
    got = np.array(got)
    assert np.all(ref[3] == 0) and np.all(got[3] == 0)
    keep = [t for t in range(w.T) if t != 3]
    assert nrmse_per_frame(got[keep], ref[keep]).max() < NRMSE_TOL
    with pytest.raises(tts.TtsError) as e:
        trk.push_frame(np.zeros((0, w.Ny), np.complex64), masks[3])
    assert e.value.code == tts.TTS_EINVAL
    trk.close()


@pytest.mark.parametrize("Nx,Ny,R,K,C,T", [(512, 32, 64, 2, 8, 3), (32, 512, 64, 2, 16, 3), (512, 512, 8, 1, 16, 3)])
def test_maximum_sizes(tts, Nx, Ny, R, K, C, T):
    """The largest layouts: Nx or Ny = 512 (the maximum line length) with R = 64 (the
    maximum rank), 128 acquired lines (several chunks of m), and a 512 x 512 frame on a
    16-CTA cluster."""
    w = inputs.Workload(name="maximum", Nx=Nx, Ny=Ny, R=R, T=T, n_ellipses=4, sigma=0.01, lambda_forget=0.9,
                        mu=1e-2, mm_iters=K, policy="uniform", rate=0.25, central_lines=8, seed=5)
    L, Y, A0, B0 = workload_inputs(w, w.T)
    masks = inputs.uniform_line_masks(w)
    ref, _, _ = run_oracle(w, w.T, Y, A0, B0, masks=masks)
    trk, got = run_gpu(tts, w, w.T, Y, A0, B0, masks, cluster_ctas=C)
    assert tts.tts_get_config(trk.h).cluster_ctas == C
    assert nrmse_per_frame(got, ref).max() < NRMSE_TOL
