"""The seeded synthetic inputs against the recipe they state (no GPU): the many-stream and
serving workloads draw from the stated sets, the serving arrivals are a Poisson process of the
stated rate, the coil maps are SENSE-normalised, the cine-256 phantom drifts along the
phase-encode axis at the stated peak speed and its ellipses breathe with the stated period,
and every generator is a function of its seed alone."""
from __future__ import annotations

import math

import numpy as np
import pytest

from paper_1609_04104_gb300 import inputs


def test_uneven_streams_draw_from_the_stated_sets():
    ws = inputs.uneven_streams(64, T=100, seed=0)
    assert len(ws) == 64
    for w in ws:
        assert w.Nx in inputs.UNEVEN_SIZES and w.Ny in inputs.UNEVEN_SIZES
        assert w.R in inputs.UNEVEN_RANKS and w.rate in inputs.UNEVEN_RATES
        assert w.T == 100 and w.lambda_forget == inputs.CINE256.lambda_forget
        assert w.mm_iters == inputs.CINE256.mm_iters
    assert len({w.seed for w in ws}) == 64
    assert len({(w.Nx, w.Ny) for w in ws}) > 10          # uneven, independently drawn
    again = inputs.uneven_streams(64, T=100, seed=0)
    assert [(w.Nx, w.Ny, w.R, w.rate, w.seed) for w in ws] == [(w.Nx, w.Ny, w.R, w.rate, w.seed) for w in again]


def test_serving_arrivals_are_a_poisson_process_of_the_stated_rate():
    arr = inputs.serving_arrivals(4000, rate_per_s=4.0, lifetime=300, seed=3)
    t = np.array([a.t_open for a in arr])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    # exponential gaps: mean 1/rate and standard deviation equal to the mean (5-sigma bands)
    assert abs(gaps.mean() - 0.25) < 5 * 0.25 / math.sqrt(len(gaps))
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1
    for a in arr[:256]:
        assert a.work.Nx == a.work.Ny and a.work.Nx in inputs.SERVING_SIZES
        assert a.work.R in (16, 24, 32, 40, 48) and 20.0 <= a.fps <= 50.0
        assert a.frames == 300 and a.work.rate == 1.0 / 8.0
    pre = inputs.serving_arrivals(256, preload=True)
    assert all(a.t_open == 0.0 for a in pre)


@pytest.mark.parametrize("C", [1, 4, 16])
def test_coil_maps_are_sense_normalised(C):
    H = inputs.coil_maps(48, 40, C, seed=2)
    assert H.shape == (C, 48, 40) and H.dtype == np.complex64
    np.testing.assert_allclose(np.sum(np.abs(H.astype(np.complex128)) ** 2, axis=0), 1.0, atol=1e-6)
    if C > 1:   # the coils see different parts of the field of view
        mags = np.abs(H).reshape(C, -1)
        assert np.all(mags.max(axis=1) > 1.5 * mags.min(axis=1))


def test_cine256_drifts_at_the_stated_peak_speed():
    """The rigid shift d(t) = (v T / 2 pi) sin(2 pi t / T) along the phase-encode axis has
    peak speed v = 0.5 px/frame at t = 0; the body's centre of mass follows it."""
    w = inputs.scaled(inputs.CINE256, n_ellipses=1)      # the body ellipse alone
    def com(t):
        img = inputs.phantom_frame(w, t)
        i = np.arange(w.Nx)[:, None]
        return float((img * i).sum() / img.sum())
    v = w.drift_px_per_frame
    amp = v * w.drift_period / (2 * math.pi)
    for t in (0, 10, 20, 40, 60):
        assert abs((com(t) - com(0)) - amp * math.sin(2 * math.pi * t / w.drift_period)) < 0.15
    assert abs((com(1) - com(0)) - v) < 0.15


def test_breathing_ellipses_follow_the_stated_modulation():
    """Ellipses 1 and 2 scale their semi-axes by 1 + 0.15 sin(2 pi t / 20); the others stay."""
    w = inputs.SMALL_CINE
    ells = inputs.ellipses(w)
    assert [e.breathes for e in ells[:4]] == [False, True, True, False]
    one = [e if i == 1 else inputs.Ellipse(e.cx, e.cy, e.a, e.b, e.theta, 0.0, e.breathes)
           for i, e in enumerate(ells)]
    big = inputs.scaled(w, Nx=256, Ny=256)
    area0 = inputs.phantom_frame(big, 0, one).sum() / ells[1].intensity
    area5 = inputs.phantom_frame(big, 5, one).sum() / ells[1].intensity     # sin = 1
    assert abs(area5 / area0 - 1.15 ** 2) < 0.03


def test_kspace_noise_has_the_stated_level_and_generators_are_seeded():
    w = inputs.scaled(inputs.SMALL_CINE, T=4)
    L = inputs.phantom(w)
    Y = inputs.kspace(w, L)
    d = Y - np.fft.fft2(L, norm="ortho")
    assert abs(np.std(d) - w.sigma) < 0.05 * w.sigma
    assert abs(np.mean(d)) < 5 * w.sigma / math.sqrt(d.size)
    np.testing.assert_array_equal(Y, inputs.kspace(w, L))
    A1, B1 = inputs.init_factors(64, 48, 8, seed=9)
    A2, B2 = inputs.init_factors(64, 48, 8, seed=9)
    np.testing.assert_array_equal(A1, A2)
    np.testing.assert_array_equal(B1, B2)
    # initial factors CN(0, 1/N)
    assert abs(np.mean(np.abs(inputs.init_factors(512, 512, 64, 1)[0]) ** 2) * 512 - 1.0) < 0.05
