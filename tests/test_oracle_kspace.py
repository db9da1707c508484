"""Pins of the k-space interpolation oracle (Alg. 2, §IV-A): its images equal those of the
image-domain tracker started from the transformed factors (the two share no transform
code: the k-space tracker never applies a DFT inside its iterations); finite-difference
gradients; monotone MM; the paper's Alg. 2 row update for one Jacobi iteration; scores."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import kspace as K
from oracle import tracker as O


def cn(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)


@pytest.mark.parametrize("update", ["gauss_seidel", "jacobi"])
def test_equals_image_domain_tracker_under_the_change_of_variables(update):
    rng = np.random.default_rng(11)
    Nx, Ny, R = 10, 8, 3
    A, B = 0.4 * cn(rng, Nx, R), 0.4 * cn(rng, Ny, R)
    img = O.Tracker(Nx, Ny, R, 0.9, 1e-2, 3, update=update, A=A, B=B)
    ks = K.KspaceTracker(Nx, Ny, R, 0.9, 1e-2, 3, update=update,
                         A1=O.dft_matrix(Nx) @ A, A2=O.dft_matrix(Ny) @ B)
    for t in range(6):
        mask = np.zeros(Nx, np.uint8)
        mask[rng.choice(Nx, 4, replace=False)] = 1
        rows = np.flatnonzero(mask)
        Y = O.fft2(cn(rng, Nx, 2) @ cn(rng, 2, Ny))
        xi = img.push_frame(Y[rows], mask)
        xk = ks.push_frame(Y[rows], mask)
        assert np.allclose(xk, xi, atol=1e-11 * np.abs(xi).max())
        assert np.allclose(ks.line_probs(), img.line_probs(), atol=1e-13)


def test_gradients_by_finite_differences():
    rng = np.random.default_rng(12)
    Nx, Ny, R = 5, 4, 2
    P, Q, g = cn(rng, Nx, R), cn(rng, Ny, R), cn(rng, R)
    rows = np.array([0, 3])
    Y = O.zero_filled(cn(rng, 2, Ny), rows, Nx)
    mu, rho = 0.2, 0.05
    for which in ("A1", "A2"):
        X = P if which == "A1" else Q
        grad = (K.ks_gradient_A1 if which == "A1" else K.ks_gradient_A2)(P, Q, g, Y, rows, rho)

        def J(Z):
            return K.ks_objective_J(Z if which == "A1" else P, Q if which == "A1" else Z, g, Y, rows, mu, rho)

        eps = 1e-6
        for idx in np.ndindex(X.shape):
            d = np.zeros_like(X)
            d[idx] = eps
            num = (J(X + d) - J(X - d)) / (2 * eps) + 1j * (J(X + 1j * d) - J(X - 1j * d)) / (2 * eps)
            assert abs(num - grad[idx]) < 1e-6 * max(1.0, abs(grad[idx]))


def test_rows_outside_omega_keep_their_data_term_zero():
    """Only the rows of A1 that meet Omega see the data term: the other rows move by the
    penalty and the surrogate pull only (Alg. 2 updates the i-th row when datum (i, j) arrives)."""
    rng = np.random.default_rng(13)
    Nx, Ny, R = 8, 5, 2
    P, Q, g = cn(rng, Nx, R), cn(rng, Ny, R), cn(rng, R)
    rows = np.array([1, 4, 6])
    Y = O.zero_filled(cn(rng, 3, Ny), rows, Nx)
    rho = 0.3
    G = K.ks_gradient_A1(P, Q, g, Y, rows, rho)
    others = np.setdiff1d(np.arange(Nx), rows)
    assert np.allclose(G[others], rho * P[others], atol=1e-14)


def test_mm_objective_monotone_per_substep():
    rng = np.random.default_rng(14)
    Nx, Ny, R = 12, 9, 3
    ks = K.KspaceTracker(Nx, Ny, R, 0.9, 1e-2, 3, A1=cn(rng, Nx, R), A2=cn(rng, Ny, R))
    for t in range(6):
        mask = np.zeros(Nx, np.uint8)
        mask[rng.choice(Nx, 5, replace=False)] = 1
        Y = cn(rng, Nx, 2) @ cn(rng, 2, Ny)
        ks.push_frame(Y[np.flatnonzero(mask)], mask, record=True)
        vals = [v for _, v in ks.trace]
        for a, b in zip(vals, vals[1:]):
            assert b <= a + 1e-12 * abs(a)


def test_one_jacobi_iteration_is_papers_row_update():
    """K = 1, lambda_forget = 1, Jacobi: a_r^(1) <- (1 - mu_t lambda / t) a_r^(1)
    + mu_t gamma_r^* sum_{(i,j) in Omega} e_ij conj(a_{j,r}^(2)) e_i with mu_t = 1 / abar_t
    (Alg. 2 (S2)); likewise a^(2)."""
    rng = np.random.default_rng(15)
    Nx, Ny, R = 6, 5, 2
    P, Q = cn(rng, Nx, R), cn(rng, Ny, R)
    lam = 0.3
    ks = K.KspaceTracker(Nx, Ny, R, 1.0, lam, 1, update="jacobi", A1=P, A2=Q)
    mask = np.array([1, 0, 1, 0, 1, 1], np.uint8)
    rows = np.flatnonzero(mask)
    Yf = cn(rng, Nx, Ny)
    ks.push_frame(Yf[rows], mask)
    g = O.ridge_gamma(K.ks_phi(P, Q, rows), Yf[rows].reshape(-1), lam)
    E = K.ks_residual(P, Q, g, O.zero_filled(Yf[rows], rows, Nx), rows)
    abarA, abarB = O.lipschitz_A(Q, g, lam), O.lipschitz_B(P, g, lam)
    for r in range(R):
        a = (1 - lam / abarA) * P[:, r] + (1 / abarA) * np.conj(g[r]) * (E @ np.conj(Q[:, r]))
        b = (1 - lam / abarB) * Q[:, r] + (1 / abarB) * np.conj(g[r]) * (E.T @ np.conj(P[:, r]))
        np.testing.assert_allclose(ks.A1[:, r], a, atol=1e-12)
        np.testing.assert_allclose(ks.A2[:, r], b, atol=1e-12)


def test_scores_on_k_space_rows():
    A1 = np.zeros((16, 2), complex)
    A1[3, 0] = 1.0
    p = K.ks_line_probs(A1, 8)
    assert abs(p.sum() - 1.0) < 1e-14
    assert p[3] > p[4] and np.allclose(np.delete(p, 3), p[0])


@pytest.mark.parametrize("update", ["gauss_seidel", "jacobi"])
def test_frame_without_lines_is_the_data_free_step(update):
    """No acquired line: gamma = 0, the interpolated frame and its image are zero, and the
    k-space factors take the data-free step A[t-1] lf abar / (lf abar + rho) (the minimiser of
    the forgotten surrogates plus the factor penalty)."""
    rng = np.random.default_rng(23)
    Nx, Ny, R, lf, mu = 10, 8, 3, 0.9, 0.02
    tr = K.KspaceTracker(Nx, Ny, R, lf, mu, 2, update=update, A1=0.4 * cn(rng, Nx, R), A2=0.4 * cn(rng, Ny, R))
    for t in range(3):
        mask = np.zeros(Nx, np.uint8)
        mask[rng.choice(Nx, 4, replace=False)] = 1
        Y = O.fft2(cn(rng, Nx, 2) @ cn(rng, 2, Ny))
        tr.push_frame(Y[np.flatnonzero(mask)], mask)
    P1, Q1, aA, aB, w = tr.A1.copy(), tr.A2.copy(), tr.abar_A, tr.abar_B, tr.w
    x = tr.push_frame(np.zeros((0, Ny)), np.zeros(Nx, np.uint8))
    rho = mu / (lf * w + 1.0)
    assert np.all(x == 0) and np.all(tr.gamma == 0)
    np.testing.assert_allclose(tr.A1, P1 * (lf * aA / (lf * aA + rho)), rtol=1e-13, atol=0)
    np.testing.assert_allclose(tr.A2, Q1 * (lf * aB / (lf * aB + rho)), rtol=1e-13, atol=0)
