"""Python binding of the tracker's C ABI (include/tts.h), argument marshalling only.

Every function here has the name of the C entry point it calls; all arithmetic runs in
the CUDA kernels of libtts.so. Arrays are passed either as numpy arrays (host memory)
or as torch CUDA tensors (device memory, TTS_DEVICE_PTRS). There is no CPU fallback:
loading fails loudly when the library or a CUDA device is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtts.so")

TTS_OK = 0
TTS_EINVAL, TTS_ENOMEM, TTS_ECUDA, TTS_ERANGE, TTS_ENONFINITE, TTS_ETIMEOUT, TTS_ESTATE = -1, -2, -3, -4, -5, -6, -7
TTS_EBUSY = -8
TTS_ENGINE_GRAPH = 1
TTS_ENGINE_MAX_SLOTS = 4096
TTS_DFT_BF16X3, TTS_DFT_BF16 = 0, 1
TTS_ROWDFT_FFT, TTS_ROWDFT_BF16X3, TTS_ROWDFT_BF16 = 0, 1, 2
TTS_DEVICE_PTRS = 1
TTS_FULL_FRAME = 2
TTS_HOST_PINNED = 4
TTS_MAX_COILS = 64
TTS_NOALLOC_MAX_N = 256
TTS_NOALLOC_MAX_R = 32
TTS_NOALLOC_SCRATCH_BYTES = 4 << 20
TTS_POLICY_UNIFORM, TTS_POLICY_VARDENS, TTS_POLICY_INFORMATIVE = 0, 1, 2
TTS_UPDATE_GAUSS_SEIDEL, TTS_UPDATE_JACOBI = 0, 1
TTS_LAUNCH_FUSED, TTS_LAUNCH_PHASES = 0, 1
TTS_RIDGE_FF_ALL, TTS_RIDGE_FF_LAST = 0, 1

EXPORTS = [
    "tts_config_init", "tts_create", "tts_create_ex", "tts_destroy", "tts_set_factors", "tts_get_factors",
    "tts_get_stats", "tts_set_stats", "tts_get_gamma", "tts_get_gamma_fp64", "tts_get_ridge_operands",
    "tts_get_config", "tts_push_frame", "tts_image", "tts_next_mask",
    "tts_line_probs", "tts_sample_lines_from_probs", "tts_save", "tts_load", "tts_synchronize",
    "tts_launches_per_frame", "tts_ridge_solve", "tts_fft2d", "tts_push_frame_noalloc",
    "tts_stream_footprint", "tts_engine_create", "tts_engine_destroy", "tts_engine_admit", "tts_engine_release",
    "tts_engine_handle", "tts_engine_step", "tts_engine_image", "tts_engine_mask", "tts_engine_synchronize",
    "tts_engine_info", "tts_engine_autotune", "tts_dft2d_gemm", "tts_set_coil_maps", "tts_fp32_fma_rate",
    "tts_test_withheld_wait", "tts_test_withhold_row_transform", "tts_fft2d_autotune", "tts_last_error",
]


class TtsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"tts error {code}: {msg}")
        self.code = code


class tts_config(ctypes.Structure):
    _fields_ = [
        ("Nx", ctypes.c_int), ("Ny", ctypes.c_int), ("R", ctypes.c_int),
        ("lambda_forget", ctypes.c_double), ("mu", ctypes.c_double),
        ("mm_iters", ctypes.c_int), ("central_lines", ctypes.c_int), ("policy", ctypes.c_int),
        ("vd_alpha", ctypes.c_double), ("with_replacement", ctypes.c_int), ("update", ctypes.c_int),
        ("launch", ctypes.c_int), ("cluster_ctas", ctypes.c_int), ("init_seed", ctypes.c_uint64),
        ("stream_id", ctypes.c_uint32), ("cuda_stream", ctypes.c_void_p), ("row_dft", ctypes.c_int),
        ("kspace", ctypes.c_int), ("ridge_precision", ctypes.c_int),
    ]


class tts_frame_args(ctypes.Structure):
    _fields_ = [
        ("Nx", ctypes.c_int), ("Ny", ctypes.c_int), ("R", ctypes.c_int),
        ("lambda_forget", ctypes.c_double), ("mu", ctypes.c_double),
        ("mm_iters", ctypes.c_int), ("update", ctypes.c_int),
        ("A", ctypes.c_void_p), ("B", ctypes.c_void_p), ("stats", ctypes.c_void_p), ("gamma", ctypes.c_void_p),
        ("y_rows", ctypes.c_void_p), ("line_mask", ctypes.c_void_p), ("flags", ctypes.c_int),
    ]


class tts_engine_stats(ctypes.Structure):
    _fields_ = [
        ("arena_bytes", ctypes.c_size_t), ("arena_used", ctypes.c_size_t), ("arena_largest_free", ctypes.c_size_t),
        ("active", ctypes.c_int), ("max_slots", ctypes.c_int), ("cluster_ctas", ctypes.c_int),
        ("groups", ctypes.c_int), ("resident_clusters", ctypes.c_int), ("steps", ctypes.c_int64),
    ]


_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libtts.so (building it first if it is missing) and declare the signatures."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        from . import build as _build
        _build.build()
    lib = ctypes.CDLL(path)
    P, I, D, U64, U32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32
    H = ctypes.c_void_p
    sig = {
        "tts_config_init": (None, [ctypes.POINTER(tts_config), I, I, I, D, D]),
        "tts_create": (I, [I, I, I, D, D, ctypes.POINTER(H)]),
        "tts_create_ex": (I, [ctypes.POINTER(tts_config), ctypes.POINTER(H)]),
        "tts_destroy": (None, [H]),
        "tts_set_factors": (I, [H, P, P, I]),
        "tts_get_factors": (I, [H, P, P, I]),
        "tts_get_stats": (I, [H, ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(D),
                              ctypes.POINTER(ctypes.c_int64)]),
        "tts_set_stats": (I, [H, D, D, D, ctypes.c_int64]),
        "tts_get_gamma": (I, [H, P]),
        "tts_get_gamma_fp64": (I, [H, P]),
        "tts_get_ridge_operands": (I, [H, P, P, P, ctypes.POINTER(I)]),
        "tts_get_config": (I, [H, ctypes.POINTER(tts_config)]),
        "tts_push_frame": (I, [H, P, P, I]),
        "tts_image": (I, [H, ctypes.c_int64, P, I]),
        "tts_next_mask": (I, [H, D, U64, P, I]),
        "tts_line_probs": (I, [H, P, I]),
        "tts_sample_lines_from_probs": (I, [P, I, I, I, U64, U64, I, P, I]),
        "tts_save": (I, [H, P, ctypes.POINTER(ctypes.c_size_t)]),
        "tts_load": (I, [H, P, ctypes.c_size_t]),
        "tts_synchronize": (I, [H]),
        "tts_launches_per_frame": (I, [H]),
        "tts_ridge_solve": (I, [P, P, I, P]),
        "tts_fft2d": (I, [P, P, I, I, I, I, P]),
        "tts_push_frame_noalloc": (I, [ctypes.POINTER(tts_frame_args), P]),
        "tts_dft2d_gemm": (I, [P, P, P, I, I, I, I, I, P, P]),
        "tts_set_coil_maps": (I, [H, P, I, I]),
        "tts_stream_footprint": (I, [ctypes.POINTER(tts_config), ctypes.POINTER(ctypes.c_size_t)]),
        "tts_engine_create": (I, [ctypes.c_size_t, I, I, I, P, ctypes.POINTER(H)]),
        "tts_engine_destroy": (None, [H]),
        "tts_engine_admit": (I, [H, ctypes.POINTER(tts_config), ctypes.POINTER(I)]),
        "tts_engine_release": (I, [H, I]),
        "tts_engine_handle": (I, [H, I, ctypes.POINTER(H)]),
        "tts_engine_step": (I, [H, I, P, P, P, P, P, I]),
        "tts_engine_image": (I, [H, I, P, I]),
        "tts_engine_mask": (I, [H, I, P, I]),
        "tts_engine_synchronize": (I, [H]),
        "tts_engine_info": (I, [H, ctypes.POINTER(tts_engine_stats)]),
        "tts_engine_autotune": (I, [ctypes.POINTER(tts_config), I, I, ctypes.POINTER(I), P]),
        "tts_fp32_fma_rate": (I, [I, I, ctypes.POINTER(D), ctypes.POINTER(D)]),
        "tts_test_withheld_wait": (I, [I, P, P, P, I, I, I, ctypes.c_longlong, P, P]),
        "tts_test_withhold_row_transform": (I, [H, I, ctypes.c_longlong]),
        "tts_fft2d_autotune": (I, [I, I, I, I, ctypes.POINTER(D), ctypes.POINTER(I), ctypes.POINTER(D)]),
        "tts_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(rc: int) -> int:
    if rc < 0:
        raise TtsError(rc, tts_last_error())
    return rc


def tts_last_error() -> str:
    return load().tts_last_error().decode(errors="replace")


# --- pointer helpers --------------------------------------------------------------

def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype=None):
    """(address, device_flag) of a numpy array (host) or torch CUDA tensor (device)."""
    if x is None:
        return None, 0
    if _is_torch(x):
        if not x.is_cuda or not x.is_contiguous():
            raise ValueError("torch tensors must be contiguous CUDA tensors")
        return x.data_ptr(), TTS_DEVICE_PTRS
    if not isinstance(x, np.ndarray) or not x.flags.c_contiguous:
        raise ValueError("host arrays must be C-contiguous numpy arrays")
    if dtype is not None and x.dtype != dtype:
        raise ValueError(f"expected dtype {dtype}, got {x.dtype}")
    return x.ctypes.data, 0


def _flags(*flags):
    fs = {f for f in flags if f is not None}
    if len(fs) > 1:
        raise ValueError("mix of host and device buffers in one call")
    return fs.pop() if fs else 0


# --- the C entry points -------------------------------------------------------------

def tts_config_init(Nx, Ny, R, lambda_forget, mu, **overrides) -> tts_config:
    cfg = tts_config()
    load().tts_config_init(ctypes.byref(cfg), Nx, Ny, R, lambda_forget, mu)
    for k, v in overrides.items():
        if k == "cuda_stream" and v is not None and not isinstance(v, int):
            v = v.cuda_stream  # torch.cuda.Stream
        setattr(cfg, k, v)
    return cfg


def tts_create(Nx, Ny, R, lambda_forget, mu) -> int:
    h = ctypes.c_void_p()
    _check(load().tts_create(Nx, Ny, R, lambda_forget, mu, ctypes.byref(h)))
    return h.value


def tts_create_ex(cfg: tts_config) -> int:
    h = ctypes.c_void_p()
    _check(load().tts_create_ex(ctypes.byref(cfg), ctypes.byref(h)))
    return h.value


def tts_destroy(h) -> None:
    load().tts_destroy(h)


def tts_set_factors(h, A, B) -> None:
    pa, fa = _ptr(A, np.complex64)
    pb, fb = _ptr(B, np.complex64)
    _check(load().tts_set_factors(h, pa, pb, _flags(fa, fb)))


def tts_get_factors(h, A, B) -> None:
    pa, fa = _ptr(A, np.complex64)
    pb, fb = _ptr(B, np.complex64)
    _check(load().tts_get_factors(h, pa, pb, _flags(fa, fb)))


def tts_get_stats(h) -> dict:
    a, b, w, t = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    _check(load().tts_get_stats(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(w), ctypes.byref(t)))
    return dict(abar_A=a.value, abar_B=b.value, w=w.value, t=t.value)


def tts_set_stats(h, abar_A, abar_B, w, t) -> None:
    _check(load().tts_set_stats(h, abar_A, abar_B, w, t))


def tts_get_gamma(h, R) -> np.ndarray:
    g = np.zeros(R, np.complex64)
    _check(load().tts_get_gamma(h, g.ctypes.data))
    return g


def tts_get_gamma_fp64(h, R) -> np.ndarray:
    g = np.zeros(2 * R, np.float64)
    _check(load().tts_get_gamma_fp64(h, g.ctypes.data))
    return g[0::2] + 1j * g[1::2]


def tts_get_ridge_operands(h, Nx, Ny, R):
    """(Ahat_S, Yt, rows) of the most recent frame's first ridge step (test hook)."""
    A = np.zeros((Nx, R), np.complex64)
    Y = np.zeros((Nx, Ny), np.complex64)
    rows = np.zeros(Nx, np.int32)
    n = ctypes.c_int(0)
    _check(load().tts_get_ridge_operands(h, A.ctypes.data, Y.ctypes.data, rows.ctypes.data, ctypes.byref(n)))
    s = n.value
    return A[:s].copy(), Y[:s].copy(), rows[:s].copy()


def tts_get_config(h) -> tts_config:
    cfg = tts_config()
    _check(load().tts_get_config(h, ctypes.byref(cfg)))
    return cfg


def tts_set_coil_maps(h, maps) -> None:
    """Coil sensitivities (C x Nx x Ny complex64, numpy or CUDA tensor); None = single coil."""
    if maps is None:
        _check(load().tts_set_coil_maps(h, None, 0, 0))
        return
    pm, fm = _ptr(maps, np.complex64)
    _check(load().tts_set_coil_maps(h, pm, maps.shape[0], fm))


def tts_push_frame(h, y_rows, line_mask=None, full_frame=False, pinned=False) -> None:
    py, fy = _ptr(y_rows, np.complex64)
    pm, fm = _ptr(line_mask, np.uint8)
    flags = _flags(fy, fm if line_mask is not None else None)
    flags |= (TTS_FULL_FRAME if full_frame else 0) | (TTS_HOST_PINNED if pinned and not fy else 0)
    _check(load().tts_push_frame(h, py, pm, flags))


def tts_image(h, t, out) -> None:
    po, fo = _ptr(out, np.complex64)
    _check(load().tts_image(h, t, po, fo))


def tts_next_mask(h, rate, seed, out) -> None:
    po, fo = _ptr(out, np.uint8)
    _check(load().tts_next_mask(h, rate, seed, po, fo))


def tts_line_probs(h, out) -> None:
    po, fo = _ptr(out, np.float64)
    _check(load().tts_line_probs(h, po, fo))


def tts_sample_lines_from_probs(p, k_lines, central, seed, ctr, with_replacement=False, out=None):
    Nx = p.shape[0]
    if out is None:
        out = np.zeros(Nx, np.uint8)
    pp, fp = _ptr(p, np.float64)
    po, fo = _ptr(out, np.uint8)
    _check(load().tts_sample_lines_from_probs(pp, Nx, k_lines, central, seed, ctr, int(with_replacement), po,
                                              _flags(fp, fo)))
    return out


def tts_save(h) -> bytes:
    n = ctypes.c_size_t(0)
    _check(load().tts_save(h, None, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(load().tts_save(h, buf, ctypes.byref(n)))
    return buf.raw[: n.value]


def tts_load(h, blob: bytes) -> None:
    _check(load().tts_load(h, blob, len(blob)))


def tts_synchronize(h) -> None:
    _check(load().tts_synchronize(h))


def tts_launches_per_frame(h) -> int:
    return _check(load().tts_launches_per_frame(h))


def tts_ridge_solve(G: np.ndarray, h: np.ndarray) -> np.ndarray:
    """Solve of G gamma = h to FP64 accuracy on the device (G Hermitian positive definite)."""
    G = np.ascontiguousarray(G, np.complex128)
    h = np.ascontiguousarray(h, np.complex128)
    g = np.zeros(h.shape[0], np.complex128)
    _check(load().tts_ridge_solve(G.ctypes.data, h.ctypes.data, h.shape[0], g.ctypes.data))
    return g


def tts_fft2d(x, out, inverse=False, stream=None) -> None:
    """Batched unitary 2D DFT of torch CUDA tensors of shape (batch, Nx, Ny), complex64."""
    if x.dim() == 2:
        batch, (Nx, Ny) = 1, x.shape
    else:
        batch, Nx, Ny = x.shape
    s = 0 if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    _check(load().tts_fft2d(x.data_ptr(), out.data_ptr(), batch, Nx, Ny, int(inverse), s))


def tts_dft2d_gemm(x, out, tmp, inverse=False, precision=TTS_DFT_BF16X3, status=None, stream=None) -> None:
    """Unitary 2D DFT of torch CUDA tensors (batch, Nx, Ny) complex64 on the tensor cores."""
    if x.dim() == 2:
        batch, (Nx, Ny) = 1, x.shape
    else:
        batch, Nx, Ny = x.shape
    s = 0 if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    st = None if status is None else status.data_ptr()
    _check(load().tts_dft2d_gemm(x.data_ptr(), out.data_ptr(), tmp.data_ptr(), batch, Nx, Ny, int(inverse),
                                 precision, st, s))


def tts_push_frame_noalloc(A, B, stats, gamma, y_rows, line_mask, lambda_forget, mu, mm_iters=1,
                           update=TTS_UPDATE_GAUSS_SEIDEL, full_frame=False, stream=None) -> None:
    """Frame update on caller-held device state (torch CUDA tensors) that allocates
    nothing: A (Nx x R), B (Ny x R), gamma (R) complex64; stats (4) float64 holding
    w, abar_A, abar_B, frames; y_rows (the acquired rows, |S| x Ny, or with full_frame the
    whole Nx x Ny frame) complex64 and line_mask (Nx) uint8 as for tts_push_frame. Runs on
    `stream`, by default torch's current stream. The library reads and writes these
    buffers by their sizes, so every dtype and size is checked here first."""
    import torch
    for t in (A, B, stats, gamma, y_rows, line_mask):
        if not _is_torch(t) or not t.is_cuda or not t.is_contiguous():
            raise ValueError("tts_push_frame_noalloc takes contiguous CUDA tensors")
    c64 = torch.complex64
    if A.dtype != c64 or B.dtype != c64 or gamma.dtype != c64 or y_rows.dtype != c64:
        raise ValueError("A, B, gamma and y_rows must be complex64")
    if stats.dtype != torch.float64 or stats.numel() < 4:
        raise ValueError("stats must be float64 with at least 4 elements")
    if line_mask.dtype != torch.uint8:
        raise ValueError("line_mask must be uint8")
    if A.dim() != 2 or B.dim() != 2 or A.shape[1] != B.shape[1]:
        raise ValueError("A (Nx x R) and B (Ny x R) must be matrices with the same number of columns")
    Nx, Ny, R = A.shape[0], B.shape[0], A.shape[1]
    if gamma.numel() < R:
        raise ValueError(f"gamma needs at least R = {R} elements")
    if line_mask.numel() < Nx:
        raise ValueError(f"line_mask needs at least Nx = {Nx} elements")
    rows = Nx if full_frame else int(np.count_nonzero(line_mask[:Nx].cpu().numpy()))   # host copy: no device allocation
    if y_rows.numel() < rows * Ny:
        raise ValueError(f"y_rows needs at least {rows} x {Ny} elements")
    args = tts_frame_args(Nx, Ny, R, lambda_forget, mu, mm_iters, update,
                          A.data_ptr(), B.data_ptr(), stats.data_ptr(), gamma.data_ptr(), y_rows.data_ptr(),
                          line_mask.data_ptr(), TTS_FULL_FRAME if full_frame else 0)
    if stream is None:
        s = torch.cuda.current_stream(A.device).cuda_stream
    else:
        s = stream if isinstance(stream, int) else stream.cuda_stream
    _check(load().tts_push_frame_noalloc(ctypes.byref(args), s))


def tts_fp32_fma_rate(iters=200000, reps=3) -> tuple[float, float]:
    """(TFLOP/s, best ms) of the device's FP32 FMA throughput (calibration kernel)."""
    tf, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(load().tts_fp32_fma_rate(iters, reps, ctypes.byref(tf), ctypes.byref(ms)))
    return tf.value, ms.value


def tts_fft2d_autotune(N, batch, inverse=False, reps=3) -> dict:
    """Times tts_fft2d's launch shapes for square N x N and keeps the fastest (tts.h)."""
    ms, per_sm, lag = ctypes.c_double(0.0), ctypes.c_int(0), ctypes.c_double(0.0)
    _check(load().tts_fft2d_autotune(N, batch, int(inverse), reps, ctypes.byref(ms), ctypes.byref(per_sm),
                                     ctypes.byref(lag)))
    return {"ms": ms.value, "ctas_per_sm": per_sm.value, "lag_scale": lag.value}


def tts_test_withheld_wait(kind, x, out, tmp, index, wait_cycles, status, stream=None) -> None:
    """Test hook: a square FFT (kind 0) or tensor-core DFT (kind 1) of torch CUDA tensors
    (batch, N, N) complex64 with one awaited arrival withheld (tts.h)."""
    batch, N = x.shape[0], x.shape[1]
    s = 0 if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    _check(load().tts_test_withheld_wait(kind, x.data_ptr(), out.data_ptr(), None if tmp is None else tmp.data_ptr(),
                                         batch, N, index, wait_cycles, status.data_ptr(), s))


def tts_test_withhold_row_transform(h, chunk, wait_cycles) -> None:
    _check(load().tts_test_withhold_row_transform(h, chunk, wait_cycles))


def tts_stream_footprint(cfg: tts_config) -> int:
    n = ctypes.c_size_t(0)
    _check(load().tts_stream_footprint(ctypes.byref(cfg), ctypes.byref(n)))
    return n.value


def tts_engine_create(arena_bytes, max_slots, cluster_ctas=0, flags=TTS_ENGINE_GRAPH, stream=None) -> int:
    e = ctypes.c_void_p()
    s = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    _check(load().tts_engine_create(arena_bytes, max_slots, cluster_ctas, flags, s, ctypes.byref(e)))
    return e.value


def tts_engine_destroy(e) -> None:
    load().tts_engine_destroy(e)


def tts_engine_admit(e, cfg: tts_config) -> int:
    slot = ctypes.c_int(-1)
    _check(load().tts_engine_admit(e, ctypes.byref(cfg), ctypes.byref(slot)))
    return slot.value


def tts_engine_release(e, slot) -> None:
    _check(load().tts_engine_release(e, slot))


def tts_engine_handle(e, slot) -> int:
    h = ctypes.c_void_p()
    _check(load().tts_engine_handle(e, slot, ctypes.byref(h)))
    return h.value


def tts_engine_step(e, slots, frames, rates, seeds, masks=None, full_frame=False) -> None:
    """One frame for each listed slot: frames[k] (numpy host arrays or torch CUDA tensors,
    all of one kind), masks None or a list (entries None = the drawn mask)."""
    n = len(slots)
    if not (len(frames) == len(rates) == len(seeds) == n) or (masks is not None and len(masks) != n):
        raise ValueError("slots, frames, rates, seeds (and masks) must have one entry per slot")
    if n == 0:
        _check(load().tts_engine_step(e, 0, None, None, None, None, None, 0))
        return
    ptrs, kinds = [], set()
    for f in frames:
        p, k = _ptr(f, np.complex64)
        ptrs.append(p)
        kinds.add(k)
    mptrs = None
    if masks is not None:
        mptrs = []
        for m in masks:
            p, k = _ptr(m, np.uint8)
            mptrs.append(p or 0)
            if m is not None:
                kinds.add(k)
    if len(kinds) > 1:
        raise ValueError("mix of host and device buffers in one call")
    flags = kinds.pop() | (TTS_FULL_FRAME if full_frame else 0)
    c_slots = (ctypes.c_int * n)(*slots)
    c_frames = (ctypes.c_void_p * n)(*ptrs)
    c_masks = (ctypes.c_void_p * n)(*mptrs) if mptrs is not None else None
    c_rates = (ctypes.c_double * n)(*rates)
    c_seeds = (ctypes.c_uint64 * n)(*seeds)
    _check(load().tts_engine_step(e, n, c_slots, c_frames, c_masks, c_rates, c_seeds, flags))


def tts_engine_image(e, slot, out) -> None:
    po, fo = _ptr(out, np.complex64)
    _check(load().tts_engine_image(e, slot, po, fo))


def tts_engine_mask(e, slot, out) -> None:
    po, fo = _ptr(out, np.uint8)
    _check(load().tts_engine_mask(e, slot, po, fo))


def tts_engine_synchronize(e) -> None:
    _check(load().tts_engine_synchronize(e))


def tts_engine_info(e) -> dict:
    st = tts_engine_stats()
    _check(load().tts_engine_info(e, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in tts_engine_stats._fields_}


def tts_engine_autotune(cfgs, steps=5):
    """(best cluster size, {C: ms per step or None}) for a list of tts_config."""
    n = len(cfgs)
    arr = (tts_config * n)(*cfgs)
    best = ctypes.c_int(0)
    ms = (ctypes.c_double * 5)()
    _check(load().tts_engine_autotune(arr, n, steps, ctypes.byref(best), ms))
    return best.value, {c: (ms[i] if ms[i] >= 0 else None) for i, c in enumerate((1, 2, 4, 8, 16))}


class Engine:
    """Convenience owner of one engine (same calls as the C ABI)."""

    def __init__(self, arena_bytes, max_slots, cluster_ctas=0, graph=True, stream=None):
        self.e = tts_engine_create(arena_bytes, max_slots, cluster_ctas, TTS_ENGINE_GRAPH if graph else 0, stream)
        self.shapes = {}

    def close(self):
        if self.e:
            tts_engine_destroy(self.e)
            self.e = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def admit(self, Nx, Ny, R, lambda_forget, mu, **cfg) -> int:
        slot = tts_engine_admit(self.e, tts_config_init(Nx, Ny, R, lambda_forget, mu, **cfg))
        self.shapes[slot] = (Nx, Ny, R)
        return slot

    def release(self, slot):
        tts_engine_release(self.e, slot)
        self.shapes.pop(slot, None)

    def step(self, slots, frames, rates, seeds, masks=None, full_frame=False):
        tts_engine_step(self.e, slots, frames, rates, seeds, masks, full_frame)

    def image(self, slot, out=None):
        if out is None:
            Nx, Ny, _ = self.shapes[slot]
            out = np.zeros((Nx, Ny), np.complex64)
        tts_engine_image(self.e, slot, out)
        return out

    def mask(self, slot, out=None):
        if out is None:
            out = np.zeros(self.shapes[slot][0], np.uint8)
        tts_engine_mask(self.e, slot, out)
        return out

    def cluster_ctas(self, slot) -> int:
        return tts_get_config(tts_engine_handle(self.e, slot)).cluster_ctas

    def factors(self, slot):
        Nx, Ny, R = self.shapes[slot]
        A = np.zeros((Nx, R), np.complex64)
        B = np.zeros((Ny, R), np.complex64)
        tts_get_factors(tts_engine_handle(self.e, slot), A, B)
        return A, B

    def synchronize(self):
        tts_engine_synchronize(self.e)

    def info(self) -> dict:
        return tts_engine_info(self.e)


class Tracker:
    """Convenience owner of one tracker handle (same calls as the C ABI)."""

    def __init__(self, Nx, Ny, R, lambda_forget, mu, **cfg):
        self.Nx, self.Ny, self.R = Nx, Ny, R
        self.cfg = tts_config_init(Nx, Ny, R, lambda_forget, mu, **cfg)
        self.h = tts_create_ex(self.cfg)

    def close(self):
        if self.h:
            tts_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_factors(self, A, B):
        tts_set_factors(self.h, np.ascontiguousarray(A, np.complex64) if isinstance(A, np.ndarray) else A,
                        np.ascontiguousarray(B, np.complex64) if isinstance(B, np.ndarray) else B)

    def factors(self):
        A = np.zeros((self.Nx, self.R), np.complex64)
        B = np.zeros((self.Ny, self.R), np.complex64)
        tts_get_factors(self.h, A, B)
        return A, B

    def stats(self):
        return tts_get_stats(self.h)

    def set_stats(self, abar_A, abar_B, w, t):
        tts_set_stats(self.h, abar_A, abar_B, w, t)

    def gamma(self):
        return tts_get_gamma(self.h, self.R)

    def gamma_fp64(self):
        return tts_get_gamma_fp64(self.h, self.R)

    def ridge_operands(self):
        return tts_get_ridge_operands(self.h, self.Nx, self.Ny, self.R)

    def set_coil_maps(self, maps):
        tts_set_coil_maps(self.h, np.ascontiguousarray(maps, np.complex64) if isinstance(maps, np.ndarray) else maps)

    def push_frame(self, y_rows, line_mask=None, full_frame=False, pinned=False):
        """pinned: y_rows is a numpy view of page-locked memory that stays unchanged until the
        frame has been processed; the kernels read it in place (TTS_HOST_PINNED)."""
        if isinstance(y_rows, np.ndarray) and not pinned:
            y_rows = np.ascontiguousarray(y_rows, np.complex64)
        if isinstance(line_mask, np.ndarray):
            line_mask = np.ascontiguousarray(line_mask, np.uint8)
        tts_push_frame(self.h, y_rows, line_mask, full_frame, pinned)

    def image(self, t=None, out=None):
        if t is None:
            t = self.stats()["t"] - 1
        if out is None:
            out = np.zeros((self.Nx, self.Ny), np.complex64)
        tts_image(self.h, t, out)
        return out

    def next_mask(self, rate, seed, out=None):
        if out is None:
            out = np.zeros(self.Nx, np.uint8)
        tts_next_mask(self.h, rate, seed, out)
        return out

    def line_probs(self):
        p = np.zeros(self.Nx, np.float64)
        tts_line_probs(self.h, p)
        return p

    def save(self) -> bytes:
        return tts_save(self.h)

    def load(self, blob: bytes):
        tts_load(self.h, blob)

    def synchronize(self):
        tts_synchronize(self.h)
