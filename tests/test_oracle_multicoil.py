"""Pins of the multi-coil oracle (Alg. 3 with C coils, §IV-B) against facts other than its
own formulas: the single-coil tracker (C = 1, H = 1), the image-domain gradient of the
data fit by finite differences (Theta), factor gradients by finite differences, the
majoriser inequality in both blocks, Phi against a brute-force DFT, monotone MM, and exact
recovery of noiseless multi-coil data."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import multicoil as M
from oracle import tracker as O
from paper_1609_04104_gb300 import inputs


def cn(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)


def test_single_coil_all_ones_is_the_single_coil_tracker():
    rng = np.random.default_rng(1)
    Nx, Ny, R = 10, 8, 3
    A0, B0 = 0.4 * cn(rng, Nx, R), 0.4 * cn(rng, Ny, R)
    a = O.Tracker(Nx, Ny, R, 0.9, 1e-2, 3, A=A0, B=B0)
    b = M.MultiCoilTracker(Nx, Ny, R, np.ones((1, Nx, Ny)), 0.9, 1e-2, 3, A=A0, B=B0)
    for t in range(5):
        mask = np.zeros(Nx, np.uint8)
        mask[rng.choice(Nx, 4, replace=False)] = 1
        Y = O.fft2(cn(rng, Nx, 2) @ cn(rng, 2, Ny))
        rows = np.flatnonzero(mask)
        xa = a.push_frame(Y[rows], mask)
        xb = b.push_frame(Y[rows][None], mask)
        assert np.allclose(xa, xb, rtol=0, atol=1e-12 * np.abs(xa).max())


def test_theta_is_the_negative_image_gradient_of_the_data_fit():
    """The gradient of 1/2 sum_c ||P_Omega(Y_c - F(H_c .* L))||^2 in the real coordinates of
    the image L (packed as d/dRe + i d/dIm) at L = X is -Theta, by central differences in
    every pixel."""
    rng = np.random.default_rng(2)
    Nx, Ny, C = 5, 4, 3
    H = cn(rng, C, Nx, Ny)
    rows = np.array([0, 2, 3])
    Y = np.zeros((C, Nx, Ny), complex)
    Y[:, rows, :] = cn(rng, C, len(rows), Ny)
    X = cn(rng, Nx, Ny)

    def f(L):
        E = np.zeros_like(Y)
        for c in range(C):
            E[c][rows] = Y[c][rows] - O.fft2(H[c] * L)[rows]
        return 0.5 * float(np.vdot(E, E).real)

    E = np.zeros_like(Y)
    for c in range(C):
        E[c][rows] = Y[c][rows] - O.fft2(H[c] * X)[rows]
    Theta = M.mc_theta(E, H)
    h = 1e-6
    G = np.zeros((Nx, Ny), complex)
    for i in range(Nx):
        for j in range(Ny):
            d = np.zeros((Nx, Ny), complex)
            d[i, j] = h
            gr = (f(X + d) - f(X - d)) / (2 * h)
            gi = (f(X + 1j * d) - f(X - 1j * d)) / (2 * h)
            G[i, j] = gr + 1j * gi
    assert np.allclose(G, -Theta, atol=1e-7)


@pytest.mark.parametrize("block", ["A", "B"])
def test_factor_gradients_by_finite_differences(block):
    rng = np.random.default_rng(3)
    Nx, Ny, R, C = 5, 4, 2, 3
    H = cn(rng, C, Nx, Ny)
    rows = np.array([1, 2, 4])
    Y = np.zeros((C, Nx, Ny), complex)
    Y[:, rows, :] = cn(rng, C, len(rows), Ny)
    A, B, g = cn(rng, Nx, R), cn(rng, Ny, R), cn(rng, R)
    mu, rho = 0.1, 0.05
    X = A if block == "A" else B
    grad = (M.mc_gradient_A if block == "A" else M.mc_gradient_B)(A, B, g, H, Y, rows, rho)

    def J(Z):
        return M.mc_objective_J(Z if block == "A" else A, B if block == "A" else Z, g, H, Y, rows, mu, rho)

    h = 1e-6
    num = np.zeros_like(X)
    for idx in np.ndindex(X.shape):
        d = np.zeros_like(X)
        d[idx] = h
        num[idx] = (J(X + d) - J(X - d)) / (2 * h) + 1j * (J(X + 1j * d) - J(X - 1j * d)) / (2 * h)
    # the real-coordinate gradient packed as d/dRe + i d/dIm, as for the single coil
    assert np.allclose(num, grad, atol=1e-6)


def test_majoriser_bounds_the_data_fit():
    rng = np.random.default_rng(4)
    Nx, Ny, R, C = 6, 5, 3, 4
    H = np.asarray(inputs.coil_maps(Nx, Ny, C, 1), complex)
    rows = np.array([0, 1, 3, 5])
    Y = np.zeros((C, Nx, Ny), complex)
    Y[:, rows, :] = cn(rng, C, len(rows), Ny)
    A, B, g = cn(rng, Nx, R), cn(rng, Ny, R), 2 * cn(rng, R)
    rho = 0.0
    hmax = M.h_max(H)
    alpha = M.mc_lipschitz_A(B, g, rho, hmax)
    f0 = M.mc_objective_J(A, B, g, H, Y, rows, 0.0, rho)
    gA = M.mc_gradient_A(A, B, g, H, Y, rows, rho)
    for _ in range(20):
        D = cn(rng, Nx, R) * rng.uniform(0.01, 3.0)
        f1 = M.mc_objective_J(A + D, B, g, H, Y, rows, 0.0, rho)
        assert f1 <= f0 + float(np.vdot(gA, D).real) + 0.5 * alpha * float(np.vdot(D, D).real) + 1e-9


def test_majoriser_bounds_the_data_fit_in_b():
    """The B block's weight h_max sum_r |gamma_r|^2 ||a_r||^2 + rho majorises the data fit
    along any direction of B (the mirror of the A-block pin)."""
    rng = np.random.default_rng(6)
    Nx, Ny, R, C = 5, 6, 3, 3
    H = np.asarray(inputs.coil_maps(Nx, Ny, C, 2), complex)
    rows = np.array([0, 2, 3])
    Y = np.zeros((C, Nx, Ny), complex)
    Y[:, rows, :] = cn(rng, C, len(rows), Ny)
    A, B, g = cn(rng, Nx, R), cn(rng, Ny, R), 2 * cn(rng, R)
    rho = 0.0
    alpha = M.mc_lipschitz_B(A, g, rho, M.h_max(H))
    f0 = M.mc_objective_J(A, B, g, H, Y, rows, 0.0, rho)
    gB = M.mc_gradient_B(A, B, g, H, Y, rows, rho)
    for _ in range(20):
        D = cn(rng, Ny, R) * rng.uniform(0.01, 3.0)
        f1 = M.mc_objective_J(A, B + D, g, H, Y, rows, 0.0, rho)
        assert f1 <= f0 + float(np.vdot(gB, D).real) + 0.5 * alpha * float(np.vdot(D, D).real) + 1e-9


def test_phi_against_a_brute_force_dft():
    """Column r of Phi stacks, coil by coil, the acquired rows of the unitary 2D DFT of
    H_c .* a_r b_r^T written as the quadruple sum over (n, m) (O(N^4), no matrix product
    and no library transform); and mc_data stacks the acquired rows in the same order."""
    rng = np.random.default_rng(8)
    Nx, Ny, R, C = 4, 3, 2, 2
    H = cn(rng, C, Nx, Ny)
    A, B = cn(rng, Nx, R), cn(rng, Ny, R)
    rows = np.array([1, 3])

    def dft2_brute(X):
        out = np.zeros_like(X)
        for k in range(Nx):
            for l in range(Ny):
                acc = 0j
                for n in range(Nx):
                    for m in range(Ny):
                        acc += X[n, m] * np.exp(-2j * np.pi * (k * n / Nx + l * m / Ny))
                out[k, l] = acc / np.sqrt(Nx * Ny)
        return out

    Phi = M.mc_phi(A, B, H, rows)
    assert Phi.shape == (C * len(rows) * Ny, R)
    for r in range(R):
        col = np.concatenate([dft2_brute(H[c] * np.outer(A[:, r], B[:, r]))[rows, :].reshape(-1) for c in range(C)])
        np.testing.assert_allclose(Phi[:, r], col, rtol=0, atol=1e-12)
    Yf = cn(rng, C, Nx, Ny)
    np.testing.assert_array_equal(M.mc_data(Yf, rows), np.concatenate([Yf[c][rows, :].reshape(-1) for c in range(C)]))


def test_normalised_coil_maps():
    H = inputs.coil_maps(24, 20, 6, 0)
    s = np.sum(np.abs(H.astype(complex)) ** 2, axis=0)
    assert np.allclose(s, 1.0, atol=1e-6)
    assert abs(M.h_max(H.astype(complex)) - 1.0) < 1e-6


def test_mm_objective_monotone_per_substep():
    rng = np.random.default_rng(6)
    Nx, Ny, R, C = 10, 8, 3, 3
    H = np.asarray(inputs.coil_maps(Nx, Ny, C, 2), complex)
    tr = M.MultiCoilTracker(Nx, Ny, R, H, 0.9, 1e-2, 3, A=0.3 * cn(rng, Nx, R), B=0.3 * cn(rng, Ny, R))
    for t in range(6):
        mask = np.zeros(Nx, np.uint8)
        mask[rng.choice(Nx, 4, replace=False)] = 1
        rows = np.flatnonzero(mask)
        X = cn(rng, Nx, 2) @ cn(rng, 2, Ny)
        Yc = np.stack([O.fft2(H[c] * X)[rows] for c in range(C)])
        tr.push_frame(Yc, mask, record=True)
        vals = [v for _, v in tr.trace]
        assert len(vals) == 1 + 3 * 3
        for a, b in zip(vals, vals[1:]):
            assert b <= a + 1e-12 * abs(a), (t, vals)


def test_exact_recovery_noiseless_multicoil():
    rng = np.random.default_rng(5)
    Nx, Ny, R, C = 8, 6, 2, 3
    H = np.asarray(inputs.coil_maps(Nx, Ny, C, 3), complex)
    As, Bs = cn(rng, Nx, R), cn(rng, Ny, R)
    tr = M.MultiCoilTracker(Nx, Ny, R, H, 0.5, 1e-12, 20, A=0.3 * cn(rng, Nx, R), B=0.3 * cn(rng, Ny, R))
    full = np.ones(Nx, np.uint8)
    for t in range(200):
        X = As @ np.diag(cn(rng, R)) @ Bs.T
        x = tr.push_frame(np.stack([O.fft2(H[c] * X) for c in range(C)]), full)
    assert O.nrmse(x, X) < 1e-8


def test_frame_without_lines_is_the_data_free_step():
    """No acquired line in any coil: the data term is empty, so gamma = 0, the image is zero,
    and what is left of each block's objective, lf abar / 2 ||X - X[t-1]||^2 + rho / 2 ||X||^2,
    is minimised by X[t-1] lf abar / (lf abar + rho), whatever the coil maps."""
    rng = np.random.default_rng(17)
    Nx, Ny, R, C, lf, mu = 10, 8, 3, 4, 0.85, 0.03
    H = cn(rng, C, Nx, Ny)
    tr = M.MultiCoilTracker(Nx, Ny, R, H, lf, mu, 2, A=0.4 * cn(rng, Nx, R), B=0.4 * cn(rng, Ny, R))
    for t in range(3):
        mask = np.zeros(Nx, np.uint8)
        mask[rng.choice(Nx, 4, replace=False)] = 1
        Y = cn(rng, C, Nx, Ny)
        tr.push_frame(Y[:, np.flatnonzero(mask), :], mask)
    A1, B1, aA, aB, w = tr.A.copy(), tr.B.copy(), tr.abar_A, tr.abar_B, tr.w
    x = tr.push_frame(np.zeros((C, 0, Ny)), np.zeros(Nx, np.uint8))
    rho = mu / (lf * w + 1.0)
    assert np.all(x == 0) and np.all(tr.gamma == 0)
    np.testing.assert_allclose(tr.A, A1 * (lf * aA / (lf * aA + rho)), rtol=1e-13, atol=0)
    np.testing.assert_allclose(tr.B, B1 * (lf * aB / (lf * aB + rho)), rtol=1e-13, atol=0)
    assert tr.abar_A == pytest.approx(lf * aA + rho, rel=1e-15)
    assert tr.abar_B == pytest.approx(lf * aB + rho, rel=1e-15)
