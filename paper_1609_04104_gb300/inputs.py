"""Seeded synthetic inputs for the tracker: cine phantoms, k-space frames, line masks,
initial factors.

This module holds no arithmetic of the tracking method. It only synthesises what a
scanner and an initialiser would hand the tracker:

* a ground-truth image sequence L_t (ellipse phantom, real intensities stored as
  complex64), standing in for the paper's cardiac cine data (§VI, datasets D1/D2),
  which are not available;
* k-space frames Y_t = DFT2(L_t) + v with complex Gaussian noise v ~ CN(0, sigma^2)
  (the single-coil model of §IV). The forward transform is numpy's FFT with
  orthonormal scaling, a library routine used here only to synthesise data;
* Cartesian line masks for the fixed policies the workloads prescribe
  (central lines + uniformly random lines, or fully sampled warm-up frames);
* i.i.d. CN(0, 1/N) initial factors ("initialize at random", Alg. 3).

Both the CUDA path and the FP64 oracle consume exactly the arrays produced here.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Workload:
    """One tracker workload: phantom recipe, sampling recipe and tracker parameters."""

    name: str
    Nx: int                 # phase-encode axis (rows, index i)
    Ny: int                 # readout axis (columns, index j)
    R: int                  # PARAFAC rank
    T: int                  # frames
    n_ellipses: int
    sigma: float            # k-space noise std per complex sample
    lambda_forget: float
    mu: float
    mm_iters: int
    policy: str             # "uniform" (fixed masks from this module) | "informative"
    rate: float             # fraction of phase-encode lines per frame
    central_lines: int = 8
    warmup_frames: int = 0  # leading fully-sampled frames (warm start, §VI)
    mod_ellipses: int = 2   # ellipses whose semi-axes breathe
    mod_period: float = 20.0
    mod_amp: float = 0.15
    drift_px_per_frame: float = 0.0   # peak speed of the rigid phase-encode shift
    drift_period: float = 80.0
    seed: int = 0

    @property
    def k_lines(self) -> int:
        return max(self.central_lines, int(math.floor(self.rate * self.Nx + 0.5)))


# Small cine: 64x64, R=8, T=50, 6 ellipses, 8 central + uniform lines to 25 %.
SMALL_CINE = Workload(
    name="cine64_r8", Nx=64, Ny=64, R=8, T=50, n_ellipses=6, sigma=0.01,
    lambda_forget=0.9, mu=1e-2, mm_iters=5, policy="uniform", rate=0.25, seed=0)

# Cine size: 256x256, R=32, T=200, 12 ellipses + respiratory drift, informative
# sampling at 1/8 (32 of 256 lines, 8 central), first 5 frames fully sampled.
CINE256 = Workload(
    name="cine256_r32_informative", Nx=256, Ny=256, R=32, T=200, n_ellipses=12,
    sigma=0.01, lambda_forget=0.95, mu=1e-2, mm_iters=3, policy="informative",
    rate=1.0 / 8.0, warmup_frames=5, drift_px_per_frame=0.5, drift_period=80.0, seed=0)

# Precision-variant size: 192x192, R=32, same phantom family as CINE256.
CINE192 = dataclasses.replace(CINE256, name="cine192_r32_informative", Nx=192, Ny=192)

WORKLOADS = {w.name: w for w in (SMALL_CINE, CINE256, CINE192)}


def scaled(w: Workload, **kw) -> Workload:
    """A copy of `w` with some fields replaced (smaller T for tests, other sizes...)."""
    return dataclasses.replace(w, **kw)


@dataclasses.dataclass(frozen=True)
class Ellipse:
    cx: float
    cy: float
    a: float        # semi-axis along the rotated x axis (normalised units)
    b: float
    theta: float
    intensity: float
    breathes: bool


def ellipses(w: Workload) -> list[Ellipse]:
    """Ellipse 0 is a fixed 'body' (semi-axes 0.85, 0.75); the others have centres
    uniform in the disc r <= 0.6, semi-axes U(0.08, 0.35), angle U(0, pi); all have
    intensity U(0.2, 1). Ellipses 1..mod_ellipses breathe."""
    rng = np.random.default_rng([w.seed, 0xE11])
    out = [Ellipse(0.0, 0.0, 0.85, 0.75, 0.0, float(rng.uniform(0.2, 1.0)), False)]
    for e in range(1, w.n_ellipses):
        r = 0.6 * math.sqrt(float(rng.uniform()))
        phi = float(rng.uniform(0.0, 2.0 * math.pi))
        out.append(Ellipse(
            cx=r * math.cos(phi), cy=r * math.sin(phi),
            a=float(rng.uniform(0.08, 0.35)), b=float(rng.uniform(0.08, 0.35)),
            theta=float(rng.uniform(0.0, math.pi)),
            intensity=float(rng.uniform(0.2, 1.0)),
            breathes=(1 <= e <= w.mod_ellipses)))
    return out


def phantom_frame(w: Workload, t: int, ells: list[Ellipse] | None = None) -> np.ndarray:
    """Ground-truth image L_t (Nx x Ny, float64), rasterised at pixel centres on
    [-1, 1]^2. Row index i runs along the phase-encode axis (normalised coordinate u),
    column index j along readout (v)."""
    ells = ellipses(w) if ells is None else ells
    u = -1.0 + (2.0 * np.arange(w.Nx) + 1.0) / w.Nx
    v = -1.0 + (2.0 * np.arange(w.Ny) + 1.0) / w.Ny
    U, V = np.meshgrid(u, v, indexing="ij")
    shift_px = 0.0
    if w.drift_px_per_frame:
        amp = w.drift_px_per_frame * w.drift_period / (2.0 * math.pi)
        shift_px = amp * math.sin(2.0 * math.pi * t / w.drift_period)
    du = shift_px * 2.0 / w.Nx
    img = np.zeros((w.Nx, w.Ny))
    scale = 1.0 + w.mod_amp * math.sin(2.0 * math.pi * t / w.mod_period)
    for e in ells:
        a, b = (e.a * scale, e.b * scale) if e.breathes else (e.a, e.b)
        x = U - (e.cx + du)
        y = V - e.cy
        c, s = math.cos(e.theta), math.sin(e.theta)
        xr = c * x + s * y
        yr = -s * x + c * y
        img += e.intensity * ((xr / a) ** 2 + (yr / b) ** 2 <= 1.0)
    return img


def phantom(w: Workload, T: int | None = None) -> np.ndarray:
    """All ground-truth frames, shape (T, Nx, Ny), complex64."""
    T = w.T if T is None else T
    ells = ellipses(w)
    return np.stack([phantom_frame(w, t, ells) for t in range(T)]).astype(np.complex64)


def kspace(w: Workload, frames: np.ndarray) -> np.ndarray:
    """Fully sampled noisy k-space Y_t = DFT2(L_t) + v, v ~ CN(0, sigma^2)
    (real and imaginary parts each N(0, sigma^2/2)); complex64, shape (T, Nx, Ny).
    DC sits at index (0, 0) (no fftshift)."""
    rng = np.random.default_rng([w.seed, 0x5A])
    Y = np.fft.fft2(frames.astype(np.complex128), axes=(-2, -1), norm="ortho")
    s = w.sigma / math.sqrt(2.0)
    Y = Y + s * (rng.standard_normal(Y.shape) + 1j * rng.standard_normal(Y.shape))
    return Y.astype(np.complex64)


def central_set(Nx: int, central: int) -> np.ndarray:
    """Indices {-c/2, ..., c/2-1} mod Nx of the always-acquired central lines."""
    c = min(central, Nx)
    return np.array(sorted(((k - c // 2) % Nx) for k in range(c)), dtype=np.int64)


def uniform_line_masks(w: Workload, T: int | None = None) -> np.ndarray:
    """Fixed Cartesian masks: the central lines plus lines drawn uniformly without
    replacement up to k_lines in total; the first warmup_frames are fully sampled.
    Shape (T, Nx), uint8."""
    T = w.T if T is None else T
    rng = np.random.default_rng([w.seed, 0x3A5C])
    masks = np.zeros((T, w.Nx), np.uint8)
    cen = central_set(w.Nx, w.central_lines)
    rest = np.setdiff1d(np.arange(w.Nx), cen)
    for t in range(T):
        if t < w.warmup_frames:
            masks[t] = 1
            continue
        masks[t, cen] = 1
        extra = w.k_lines - len(cen)
        if extra > 0:
            masks[t, rng.choice(rest, size=extra, replace=False)] = 1
    return masks


def init_factors(Nx: int, Ny: int, R: int, seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Initial spatial factors A (Nx x R) and B (Ny x R), i.i.d. CN(0, 1/N); complex64."""
    rng = np.random.default_rng([seed, 0xFAC])

    def cn(n, r):
        s = 1.0 / math.sqrt(2.0 * n)
        return (s * (rng.standard_normal((n, r)) + 1j * rng.standard_normal((n, r)))).astype(np.complex64)

    return cn(Nx, R), cn(Ny, R)


def observed_rows(Y_t: np.ndarray, mask: np.ndarray) -> np.ndarray:
    """The acquired rows of one k-space frame, in increasing row order (|S| x Ny)."""
    return np.ascontiguousarray(Y_t[np.flatnonzero(mask)])


# ---- many streams ------------------------------------------------------------------

UNEVEN_SIZES = (128, 160, 192, 256, 320)
UNEVEN_RANKS = (16, 32, 48)
UNEVEN_RATES = (1.0 / 4.0, 1.0 / 6.0, 1.0 / 8.0)


def uneven_streams(n: int = 64, T: int = 100, seed: int = 0) -> list[Workload]:
    """Independent cine slices of uneven size: (Nx, Ny) drawn independently from
    {128, 160, 192, 256, 320}, R from {16, 32, 48}, sampling rate from {1/4, 1/6, 1/8};
    CINE256's phantom family, tracker parameters and warm start; stream k has seed k."""
    rng = np.random.default_rng([seed, 0xBA7C])
    out = []
    for k in range(n):
        Nx, Ny = (int(v) for v in rng.choice(UNEVEN_SIZES, size=2))
        R = int(rng.choice(UNEVEN_RANKS))
        rate = float(UNEVEN_RATES[int(rng.integers(len(UNEVEN_RATES)))])
        out.append(dataclasses.replace(CINE256, name=f"stream{k}_{Nx}x{Ny}_r{R}", Nx=Nx, Ny=Ny, R=R, T=T,
                                       rate=rate, seed=seed * 100003 + k))
    return out


# 5-smooth square sizes in [128, 384] (radices of the transforms stay in {2, 3, 5})
SERVING_SIZES = (128, 144, 160, 180, 192, 200, 216, 240, 250, 256, 270, 288, 300, 320, 360, 384)


@dataclasses.dataclass(frozen=True)
class Arrival:
    """One serving request: a cine stream that opens at `t_open` seconds and sends
    `frames` frames at `fps` frames per second."""

    t_open: float
    fps: float
    frames: int
    work: Workload


def serving_arrivals(n: int = 256, rate_per_s: float = 4.0, lifetime: int = 300, seed: int = 0,
                     preload: bool = False) -> list[Arrival]:
    """Poisson arrivals (mean `rate_per_s` new streams per second; all at t = 0 when
    `preload`), each stream 20-50 frames/s for `lifetime` frames, square 5-smooth
    matrix 128-384, R in {16, 24, 32, 40, 48}, informative sampling at 1/8."""
    rng = np.random.default_rng([seed, 0x5E7E])
    t = 0.0
    out = []
    for k in range(n):
        if not preload:
            t += float(rng.exponential(1.0 / rate_per_s))
        N = int(rng.choice(SERVING_SIZES))
        R = int(rng.choice((16, 24, 32, 40, 48)))
        fps = float(rng.uniform(20.0, 50.0))
        w = dataclasses.replace(CINE256, name=f"serve{k}_{N}_r{R}", Nx=N, Ny=N, R=R, T=lifetime,
                                rate=1.0 / 8.0, seed=seed * 100003 + k)
        out.append(Arrival(t_open=t, fps=fps, frames=lifetime, work=w))
    return out


# ---- several receive coils ----------------------------------------------------------

def coil_maps(Nx: int, Ny: int, C: int, seed: int = 0) -> np.ndarray:
    """Synthetic coil sensitivities H_c (C x Nx x Ny, complex64): coil c sits at angle
    2 pi c / C on a circle of radius 1.3 around the field of view [-1, 1]^2, with a
    Gaussian magnitude profile (width 0.9) and a smooth linear phase of random slope;
    the maps are normalised so that sum_c |H_c|^2 = 1 at every pixel (SENSE-style)."""
    rng = np.random.default_rng([seed, 0xC011])
    x = (np.arange(Nx) + 0.5) / Nx * 2.0 - 1.0
    y = (np.arange(Ny) + 0.5) / Ny * 2.0 - 1.0
    X, Yg = np.meshgrid(x, y, indexing="ij")
    maps = []
    for c in range(C):
        th = 2.0 * math.pi * c / C
        cx, cy = 1.3 * math.cos(th), 1.3 * math.sin(th)
        mag = np.exp(-((X - cx) ** 2 + (Yg - cy) ** 2) / (2.0 * 0.9 ** 2))
        kx, ky = rng.uniform(-1.5, 1.5, size=2)
        maps.append(mag * np.exp(1j * (kx * X + ky * Yg + rng.uniform(0, 2 * math.pi))))
    H = np.stack(maps)
    H /= np.sqrt(np.sum(np.abs(H) ** 2, axis=0, keepdims=True))
    return H.astype(np.complex64)


def multicoil_kspace(w: Workload, frames: np.ndarray, H: np.ndarray) -> np.ndarray:
    """Each coil's fully sampled noisy k-space, Y_c,t = DFT2(H_c .* L_t) + v with
    v ~ CN(0, sigma^2); complex64, shape (T, C, Nx, Ny)."""
    rng = np.random.default_rng([w.seed, 0x5B])
    img = H[None, :, :, :].astype(np.complex128) * frames[:, None, :, :].astype(np.complex128)
    Y = np.fft.fft2(img, axes=(-2, -1), norm="ortho")
    s = w.sigma / math.sqrt(2.0)
    Y = Y + s * (rng.standard_normal(Y.shape) + 1j * rng.standard_normal(Y.shape))
    return Y.astype(np.complex64)
