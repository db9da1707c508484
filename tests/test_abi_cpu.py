"""Host-side checks that need no GPU: the library builds/loads and exports every entry
point of include/tts.h, argument validation, no CPU fallback, and the input recipe."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1609_04104_gb300 import build, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "tts.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tts_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    path = build.build()
    return ctypes.CDLL(path)


def test_library_exports_every_declared_entry_point(lib):
    names = header_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    from paper_1609_04104_gb300 import tts
    assert sorted(tts.EXPORTS) == names


def test_binding_constants_match_the_header():
    """Every TTS_* constant of include/tts.h (#define or enum) has the same value in the
    Python binding, so flags and limits passed through it mean what the library reads."""
    from paper_1609_04104_gb300 import tts
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "tts.h")).read(), flags=re.S)
    consts = {}
    for name, expr in re.findall(r"#define\s+(TTS_[A-Z0-9_]+)\s+([^\n]+)", src):
        expr = expr.strip()
        m = re.fullmatch(r"\(?\s*(\d+)u?\s*(?:<<\s*(\d+))?\s*\)?", expr)
        if m:
            consts[name] = int(m.group(1)) << int(m.group(2) or 0)
    for name, val in re.findall(r"\b(TTS_[A-Z0-9_]+)\s*=\s*(-?\d+)", src):
        consts[name] = int(val)
    assert len(consts) >= 30
    for name, val in consts.items():
        assert getattr(tts, name) == val, name


def test_config_validation_runs_before_any_cuda_call():
    from paper_1609_04104_gb300 import tts
    for bad in (dict(Nx=7), dict(Nx=0), dict(Ny=600), dict(R=0), dict(R=65), dict(lambda_forget=0.0),
                dict(lambda_forget=1.5), dict(mu=0.0), dict(mm_iters=0), dict(central_lines=99),
                dict(policy=7), dict(update=3), dict(launch=4), dict(cluster_ctas=17)):
        kw = dict(Nx=64, Ny=64, R=8, lambda_forget=0.9, mu=1e-2)
        kw.update(bad)
        cfg = tts.tts_config_init(kw.pop("Nx"), kw.pop("Ny"), kw.pop("R"), kw.pop("lambda_forget"), kw.pop("mu"))
        for k, v in bad.items():
            setattr(cfg, k, v)
        with pytest.raises(tts.TtsError) as e:
            tts.tts_create_ex(cfg)
        assert e.value.code == tts.TTS_EINVAL, bad


def test_no_cpu_fallback_without_a_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1609_04104_gb300 import tts
    with pytest.raises(tts.TtsError) as e:
        tts.tts_create(64, 64, 8, 0.9, 1e-2)
    assert e.value.code == tts.TTS_ECUDA
    assert "no CPU fallback" in tts.tts_last_error() or "CUDA" in tts.tts_last_error()
    with pytest.raises(tts.TtsError) as e:
        tts.tts_engine_create(1 << 24, 4)
    assert e.value.code == tts.TTS_ECUDA
    cfg = tts.tts_config_init(64, 64, 8, 0.9, 1e-2)
    with pytest.raises(tts.TtsError) as e:
        tts.tts_engine_autotune([cfg], steps=1)
    assert e.value.code in (tts.TTS_ECUDA, tts.TTS_EINVAL)


def test_input_recipe_shapes_and_masks():
    w = inputs.scaled(inputs.CINE256, T=7)
    L = inputs.phantom(w)
    assert L.shape == (7, 256, 256) and L.dtype == np.complex64
    assert np.all(L.imag == 0) and 0 < L.real.max() < 12
    Y = inputs.kspace(w, L)
    # the noise is the only difference between Y and the exact transform
    d = Y - np.fft.fft2(L, norm="ortho")
    assert abs(np.std(d) - w.sigma) < 0.05 * w.sigma
    m = inputs.uniform_line_masks(inputs.SMALL_CINE)
    assert m.shape == (50, 64) and np.all(m.sum(1) == 16)
    assert np.all(m[:, inputs.central_set(64, 8)] == 1)
    assert inputs.CINE256.k_lines == 32 and inputs.SMALL_CINE.k_lines == 16
    A, B = inputs.init_factors(256, 192, 32)
    assert A.shape == (256, 32) and B.shape == (192, 32)
    assert abs(np.mean(np.abs(A) ** 2) - 1 / 256) < 0.1 / 256


def test_transform_and_sampler_arguments_checked_before_any_cuda_call(lib):
    """Argument errors of the standalone entry points come back as TTS_EINVAL (-1) with a
    message, before the library touches the device (fake, never dereferenced addresses)."""
    P = ctypes.c_void_p
    lib.tts_fft2d.argtypes = [P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P]
    lib.tts_dft2d_gemm.argtypes = [P, P, P] + [ctypes.c_int] * 5 + [P, P]
    lib.tts_sample_lines_from_probs.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                                ctypes.c_uint64, ctypes.c_int, P, ctypes.c_int]
    lib.tts_last_error.restype = ctypes.c_char_p
    a, b, c = P(0x10000), P(0x20000), P(0x30000)
    assert lib.tts_fft2d(None, b, 1, 64, 64, 0, None) == -1
    assert lib.tts_fft2d(a, b, 1, 7, 64, 0, None) == -1            # prime factor 7
    assert lib.tts_fft2d(a, b, 1, 64, 1024, 0, None) == -1          # beyond 512
    assert lib.tts_fft2d(a, b, -1, 64, 64, 0, None) == -1
    assert lib.tts_dft2d_gemm(a, b, c, 1, 48, 64, 0, 0, None, None) == -1   # 48: not a multiple of 32
    assert lib.tts_dft2d_gemm(a, b, a, 1, 64, 64, 0, 0, None, None) == -1   # tmp aliases in
    assert lib.tts_dft2d_gemm(P(0x10008), b, c, 1, 64, 64, 0, 0, None, None) == -1   # 8 bytes off 16
    assert b"aligned" in lib.tts_last_error()
    assert lib.tts_dft2d_gemm(a, b, c, 1, 64, 64, 0, 5, None, None) == -1   # unknown precision
    p = (ctypes.c_double * 8)(*([0.125] * 8))
    out = (ctypes.c_uint8 * 8)()
    assert lib.tts_sample_lines_from_probs(None, 8, 2, 0, 1, 0, 0, out, 0) == -1
    assert lib.tts_sample_lines_from_probs(p, 0, 2, 0, 1, 0, 0, out, 0) == -1
    assert lib.tts_sample_lines_from_probs(p, 8, 2, 9, 1, 0, 0, out, 0) == -1   # central > Nx
    bad = (ctypes.c_double * 8)(*([0.125] * 7 + [float("nan")]))
    assert lib.tts_sample_lines_from_probs(bad, 8, 2, 0, 1, 0, 0, out, 0) == -1


def _footprint(tts, Nx, Ny, R, C):
    cfg = tts.tts_config_init(Nx, Ny, R, 0.95, 1e-2)
    cfg.cluster_ctas = C
    return tts.tts_stream_footprint(cfg)


def test_stream_footprint_is_host_arithmetic_and_grows_with_the_cluster():
    """tts_stream_footprint needs no device. It covers the resident state of a stream (A, B,
    their anchors and the three Nx x Ny planes: staged rows, transformed rows, image), and
    the per-CTA partial sums make it grow by exactly C x (Nx R complex + Nx R + 2 R^2 float-float
    complex + R float) between cluster sizes. A layout that does not fit clusters of the size asked is
    refused with TTS_EINVAL; 0 means the engine default (4 CTAs)."""
    from paper_1609_04104_gb300 import tts
    for Nx, Ny, R in [(64, 64, 8), (256, 256, 32), (128, 96, 16), (192, 120, 24)]:
        f = {C: _footprint(tts, Nx, Ny, R, C) for C in (2, 4, 8, 16)}
        assert f[4] == _footprint(tts, Nx, Ny, R, 0)
        assert f[2] >= 8 * (2 * (Nx + Ny) * R + 3 * Nx * Ny)
        # partials: Ahat (complex), P (float-float complex), ||a||^2 (float), B^H B and
        # Ahat^H Ahat (float-float complex)
        per_cta = 8 * Nx * R + 16 * Nx * R + 4 * R + 2 * 16 * R * R
        for a, b in [(2, 4), (4, 8), (8, 16)]:
            assert abs((f[b] - f[a]) - (b - a) * per_cta) <= 4 * 256, (Nx, Ny, R, a, b)
    with pytest.raises(tts.TtsError) as e:
        _footprint(tts, 384, 384, 64, 4)
    assert e.value.code == tts.TTS_EINVAL
    assert _footprint(tts, 384, 384, 64, 16) > _footprint(tts, 256, 256, 32, 16)
