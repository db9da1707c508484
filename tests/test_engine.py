"""The multi-stream engine (tts_engine_*): every stream's frames, images and line draws in
a batched step equal those of the same stream's handle run alone, whatever else is in
the step (continuous batching: streams join late, leave, and skip steps); admission by
arena footprint; argument errors. Parity with the FP64 oracle for a stream in a mix."""
from __future__ import annotations

import dataclasses

import numpy as np
import pytest

from paper_1609_04104_gb300 import inputs
from tests.helpers import NRMSE_TOL, nrmse_per_frame, run_oracle

pytestmark = pytest.mark.gpu

# (Nx, Ny, R, K, rate): uneven sizes, ranks (small and large per-thread output counts),
# iteration counts and rates in one mix
# (384 x 384, R 48 does not fit clusters of 4 CTAs: it runs in a second launch group of 8)
MIX = [(64, 64, 8, 5, 0.25), (96, 80, 16, 3, 1 / 6), (128, 128, 48, 3, 1 / 8), (80, 96, 32, 2, 0.25),
       (48, 64, 4, 4, 0.25), (160, 128, 24, 3, 1 / 8), (384, 384, 48, 2, 1 / 8)]
T = 7


def mix_workloads():
    out = []
    for k, (Nx, Ny, R, K, rate) in enumerate(MIX):
        out.append(dataclasses.replace(inputs.CINE256, name=f"mix{k}", Nx=Nx, Ny=Ny, R=R, T=T, mm_iters=K,
                                       rate=rate, warmup_frames=2, seed=11 + k))
    return out


def stream_kspace(w):
    return inputs.kspace(w, inputs.phantom(w, T))


def cfg_of(w, k):
    return dict(mm_iters=w.mm_iters, central_lines=w.central_lines, init_seed=w.seed, stream_id=k)


def run_alone(tts, w, k, Y, frames, C):
    """The stream alone through its own handle (clusters of C CTAs): push, image, next
    mask per frame."""
    trk = tts.Tracker(w.Nx, w.Ny, w.R, w.lambda_forget, w.mu, cluster_ctas=C, **cfg_of(w, k))
    imgs, masks = [], []
    m = drawn = np.ones(w.Nx, np.uint8)
    for t in range(frames):
        if t >= w.warmup_frames:
            m = drawn
        trk.push_frame(inputs.observed_rows(Y[t], m), m)
        imgs.append(trk.image(t))
        drawn = trk.next_mask(w.rate, 1000 + k)
        masks.append(drawn.copy())
    A, B = trk.factors()
    trk.close()
    return np.array(imgs), np.array(masks), A, B


def schedule():
    """Which streams take part in each engine step: stream 3 joins at step 2, stream 1
    sits out step 3, stream 5 joins at step 1 and leaves after 4 frames."""
    plan = []
    for s in range(T + 2):
        part = []
        for k in range(len(MIX)):
            if k == 3 and s < 2:
                continue
            if k == 1 and s == 3:
                continue
            if k == 5 and not (1 <= s < 5):
                continue
            part.append(k)
        plan.append(part)
    return plan


def run_engine(tts, ws, Ys, graph=True, device_inputs=False):
    import torch
    eng = tts.Engine(1 << 30, 16, graph=graph)
    slots, t_of, cs = {}, {}, {}
    imgs = {k: [] for k in range(len(ws))}
    masks = {k: [] for k in range(len(ws))}
    drawn = {}
    for s, part in enumerate(schedule()):
        part = [k for k in part if t_of.get(k, 0) < T]
        for k in part:
            if k not in slots:
                w = ws[k]
                slots[k] = eng.admit(w.Nx, w.Ny, w.R, w.lambda_forget, w.mu, **cfg_of(w, k))
                cs[k] = eng.cluster_ctas(slots[k])
                t_of[k] = 0
        if not part:
            continue
        frames, ms = [], []
        for k in part:
            w, t = ws[k], t_of[k]
            m = np.ones(w.Nx, np.uint8) if t < w.warmup_frames else drawn[k]
            rows = inputs.observed_rows(Ys[k][t], m)
            if device_inputs:
                frames.append(torch.from_numpy(rows).cuda())
                ms.append(torch.from_numpy(m).cuda())
            else:
                frames.append(rows)
                ms.append(m)
        eng.step([slots[k] for k in part], frames, [ws[k].rate for k in part], [1000 + k for k in part], masks=ms)
        for k in part:
            imgs[k].append(eng.image(slots[k]))
            drawn[k] = eng.mask(slots[k])
            masks[k].append(drawn[k].copy())
            t_of[k] += 1
        if 5 in slots and t_of[5] == 4:
            eng.release(slots.pop(5))
    facs = {k: eng.factors(slots[k]) for k in slots}
    info = eng.info()
    eng.close()
    return ({k: np.array(v) for k, v in imgs.items()}, {k: np.array(v) for k, v in masks.items()}, facs, info,
            cs)


@pytest.fixture(scope="module")
def mix():
    ws = mix_workloads()
    return ws, [stream_kspace(w) for w in ws]


@pytest.fixture(scope="module")
def engine_run(tts, mix):
    ws, Ys = mix
    return run_engine(tts, ws, Ys, graph=True)


def test_engine_equals_alone(tts, mix, engine_run):
    ws, Ys = mix
    imgs, masks, facs, info, cs = engine_run
    assert info["active"] == len(MIX) - 1 and info["steps"] >= T
    assert info["cluster_ctas"] == 4 and info["groups"] == 2
    assert cs[6] == 8 and all(cs[k] == 4 for k in range(6))
    for k, w in enumerate(ws):
        n = len(imgs[k])
        assert n == (4 if k == 5 else T)
        ai, am, A, B = run_alone(tts, w, k, Ys[k], n, cs[k])
        assert np.array_equal(imgs[k].view(np.uint32), ai.view(np.uint32)), f"stream {k}: images differ"
        assert np.array_equal(masks[k], am), f"stream {k}: drawn masks differ"
        if k in facs:
            assert np.array_equal(facs[k][0].view(np.uint32), A.view(np.uint32))
            assert np.array_equal(facs[k][1].view(np.uint32), B.view(np.uint32))
        assert np.all(am.sum(axis=1) == w.k_lines)


def test_engine_graph_and_direct_launch_agree(tts, mix, engine_run):
    ws, Ys = mix
    imgs, masks = engine_run[0], engine_run[1]
    imgs2, masks2 = run_engine(tts, ws, Ys, graph=False, device_inputs=True)[:2]
    for k in range(len(ws)):
        assert np.array_equal(imgs[k].view(np.uint32), imgs2[k].view(np.uint32))
        assert np.array_equal(masks[k], masks2[k])


def test_engine_stream_matches_oracle(tts):
    """The small cine (64 x 64, R 8, K 5, fixed uniform masks) as one stream in a mix with
    two larger streams; its images against the FP64 oracle frame by frame."""
    w = inputs.scaled(inputs.SMALL_CINE, T=10)
    L = inputs.phantom(w, w.T)
    Y = inputs.kspace(w, L)
    A0, B0 = inputs.init_factors(w.Nx, w.Ny, w.R, w.seed)
    M = inputs.uniform_line_masks(w, w.T)
    ref, _, _ = run_oracle(w, w.T, Y, A0, B0, masks=M)
    others = [dataclasses.replace(inputs.CINE256, name="o1", Nx=128, Ny=160, R=32, T=w.T, warmup_frames=w.T),
              dataclasses.replace(inputs.CINE256, name="o2", Nx=192, Ny=192, R=48, T=w.T, warmup_frames=w.T)]
    Yo = [stream_kspace(dataclasses.replace(o, T=T))[:1] for o in others]
    eng = tts.Engine(1 << 30, 4)
    s0 = eng.admit(w.Nx, w.Ny, w.R, w.lambda_forget, w.mu, mm_iters=w.mm_iters, central_lines=w.central_lines,
                   policy=tts.TTS_POLICY_UNIFORM)
    tts.tts_set_factors(tts.tts_engine_handle(eng.e, s0), A0, B0)
    so = [eng.admit(o.Nx, o.Ny, o.R, o.lambda_forget, o.mu, mm_iters=o.mm_iters, stream_id=7 + i)
          for i, o in enumerate(others)]
    out = []
    for t in range(w.T):
        full = [np.ones(o.Nx, np.uint8) for o in others]
        eng.step([s0] + so, [inputs.observed_rows(Y[t], M[t])] + [Yo[i][0] for i in range(2)],
                 [w.rate, 0.125, 0.125], [1, 2, 3], masks=[M[t]] + full)
        out.append(eng.image(s0))
    eng.close()
    err = nrmse_per_frame(np.array(out), ref)
    assert err.max() <= NRMSE_TOL, err


def test_engine_admission_by_footprint(tts):
    cfg = tts.tts_config_init(256, 256, 32, 0.95, 1e-2, mm_iters=3)
    f = tts.tts_stream_footprint(cfg)
    cfg4 = tts.tts_config_init(256, 256, 32, 0.95, 1e-2, mm_iters=3, cluster_ctas=4)
    cfg8 = tts.tts_config_init(256, 256, 32, 0.95, 1e-2, mm_iters=3, cluster_ctas=8)
    assert f == tts.tts_stream_footprint(cfg4) < tts.tts_stream_footprint(cfg8)   # partial sums per CTA
    assert f >= 8 * 256 * 256 * 3   # frame staging, Yt and image planes at least
    eng = tts.Engine(2 * f + 65536, 8)
    a = eng.admit(256, 256, 32, 0.95, 1e-2, mm_iters=3)
    b = eng.admit(256, 256, 32, 0.95, 1e-2, mm_iters=3)
    info = eng.info()
    assert info["arena_used"] == 2 * f and info["active"] == 2
    with pytest.raises(tts.TtsError) as ei:
        eng.admit(256, 256, 32, 0.95, 1e-2, mm_iters=3)
    assert ei.value.code == tts.TTS_EBUSY
    small = eng.admit(16, 16, 2, 0.95, 1e-2)   # a small stream still fits in what is left
    eng.release(a)
    c = eng.admit(256, 256, 32, 0.95, 1e-2, mm_iters=3)
    assert c == a
    eng.release(small)
    eng.release(b)
    eng.release(c)
    info = eng.info()
    assert info["arena_used"] == 0 and info["active"] == 0
    assert info["arena_largest_free"] == info["arena_bytes"]   # freed blocks coalesce
    eng.close()
    eng = tts.Engine(1 << 26, 2)
    eng.admit(32, 32, 4, 0.9, 1e-2)
    eng.admit(32, 32, 4, 0.9, 1e-2)
    with pytest.raises(tts.TtsError) as ei:
        eng.admit(32, 32, 4, 0.9, 1e-2)
    assert ei.value.code == tts.TTS_EBUSY
    eng.close()


def test_engine_errors_leave_streams_unchanged(tts):
    eng = tts.Engine(1 << 26, 4)
    s0 = eng.admit(32, 32, 4, 0.9, 1e-2, policy=tts.TTS_POLICY_UNIFORM)
    s1 = eng.admit(48, 32, 4, 0.9, 1e-2, policy=tts.TTS_POLICY_UNIFORM)
    rng = np.random.default_rng(3)
    y0 = (rng.standard_normal((32, 32)) + 1j * rng.standard_normal((32, 32))).astype(np.complex64)
    y1 = (rng.standard_normal((48, 32)) + 1j * rng.standard_normal((48, 32))).astype(np.complex64)
    m0, m1 = np.ones(32, np.uint8), np.ones(48, np.uint8)

    def code(**kw):
        args = dict(slots=[s0, s1], frames=[y0, y1], rates=[0.5, 0.5], seeds=[1, 2], masks=[m0, m1])
        args.update(kw)
        with pytest.raises(tts.TtsError) as ei:
            eng.step(**args)
        return ei.value.code

    assert code(slots=[s0, s0], frames=[y0, y0], masks=[m0, m0]) == tts.TTS_EINVAL
    assert code(rates=[0.0, 0.5]) == tts.TTS_EINVAL
    assert code(slots=[s0, 3]) == tts.TTS_EINVAL
    assert code(masks=[None, None]) == tts.TTS_ESTATE          # no mask drawn yet
    bad = y1.copy()
    bad[5, 7] = np.nan
    assert code(frames=[y0, bad]) == tts.TTS_ENONFINITE
    for s in (s0, s1):
        assert tts.tts_get_stats(tts.tts_engine_handle(eng.e, s))["t"] == 0
    with pytest.raises(tts.TtsError) as ei:
        eng.image(s0)
    assert ei.value.code == tts.TTS_ERANGE
    eng.step([s0, s1], [y0, y1], [0.5, 0.5], [1, 2], masks=[m0, m1])
    for s, Nx in ((s0, 32), (s1, 48)):
        assert tts.tts_get_stats(tts.tts_engine_handle(eng.e, s))["t"] == 1
        assert eng.mask(s).sum() == (16 if Nx == 32 else 24)
    eng.synchronize()
    eng.close()


def test_engine_autotune(tts):
    cfgs = [tts.tts_config_init(Nx, Ny, R, 0.95, 1e-2, mm_iters=3, stream_id=k)
            for k, (Nx, Ny, R) in enumerate([(128, 128, 16), (192, 160, 32), (256, 256, 48), (320, 320, 48)] * 4)]
    best, ms = tts.tts_engine_autotune(cfgs, steps=3)
    assert best in (1, 2, 4, 8, 16) and ms[best] is not None
    timed = {c: v for c, v in ms.items() if v is not None}
    assert ms[best] == min(timed.values()) and len(timed) >= 3
    with pytest.raises(tts.TtsError):
        tts.tts_engine_autotune([], steps=1)
