"""FP64 CPU oracle of the k-space interpolation tracker: Alg. 2 of the paper (§IV-A).

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
and reference legs may import this module. The product library never does, and this
module imports nothing from it.

The k-space frame X_t is modelled directly as trilinear, x^{(i,j)} = <alpha_i, beta_j,
gamma_t> with alpha_i, beta_j the rows of the k-space factors A1 (Nx x R), A2 (Ny x R), and
observed on Omega_t (§IV-A, the sketch e_i e_j^T). Alg. 2 then reads:
  (S1) Phi_{l, r} = A1[i, r] A2[j, r] for l = (i, j) in Omega; gamma solves the ridge problem;
  (S2) each factor row that meets Omega moves along sum over Omega of the residual times
       the other factor's conjugate row: grad_A1 = rho A1 - E conj(A2) diag(conj gamma)
       and grad_A2 = rho A2 - E^T conj(A1) diag(conj gamma), E the residual on Omega.
The image is F^{-1}(A1 diag(gamma) A2^T) (the paper keeps its magnitude). The readings of
tracker.py (forgetting, Gauss-Seidel MM iterations, surrogate minimiser, alpha from the
other factor's column norms) apply unchanged. Because F is unitary, this is the image-domain
tracker under the change of variables A1 = F_Nx A, A2 = F_Ny B.
"""
from __future__ import annotations

import numpy as np

from . import tracker as T


def ks_phi(A1: np.ndarray, A2: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """Phi of Alg. 2 (S1): row l = (i, j) in Omega (rows x [Ny], row by row) holds
    A1[i, r] A2[j, r]. Shape (|S| Ny) x R (no rows when S is empty)."""
    rows = np.asarray(rows, dtype=np.int64)
    Ny, R = A2.shape
    return (A1[rows][:, None, :] * A2[None, :, :]).reshape(len(rows) * Ny, R)


def ks_residual(A1, A2, gamma, Y, rows) -> np.ndarray:
    """E = P_Omega(Y - A1 diag(gamma) A2^T), zero off Omega: the residual of the trilinear
    k-space model of §IV-A on the sampled entries."""
    X = A1 @ np.diag(gamma) @ A2.T
    E = np.zeros_like(Y)
    E[rows, :] = Y[rows, :] - X[rows, :]
    return E


def ks_objective_J(A1, A2, gamma, Y, rows, mu, rho) -> float:
    """f_t of §III-A for the k-space model of §IV-A (Alg. 2): data fit on Omega, ridge on
    gamma, factor penalty rho / 2 on A1 and A2."""
    E = ks_residual(A1, A2, gamma, Y, rows)
    return 0.5 * float(np.vdot(E, E).real) + 0.5 * mu * float(np.vdot(gamma, gamma).real) \
        + 0.5 * rho * float(np.vdot(A1, A1).real + np.vdot(A2, A2).real)


def ks_gradient_A1(A1, A2, gamma, Y, rows, rho) -> np.ndarray:
    """Gradient of f_t in A1 (Alg. 2 (S2), the row updates of §IV-A)."""
    E = ks_residual(A1, A2, gamma, Y, rows)
    return rho * A1 - E @ np.conj(A2) @ np.diag(np.conj(gamma))


def ks_gradient_A2(A1, A2, gamma, Y, rows, rho) -> np.ndarray:
    """Gradient of f_t in A2 (Alg. 2 (S2), the row updates of §IV-A)."""
    E = ks_residual(A1, A2, gamma, Y, rows)
    return rho * A2 - E.T @ np.conj(A1) @ np.diag(np.conj(gamma))


class KspaceTracker:
    """Online k-space interpolation tracker (Alg. 2 with the readings above)."""

    def __init__(self, Nx, Ny, R, lambda_forget, mu, mm_iters=1, update="gauss_seidel", A1=None, A2=None):
        self.Nx, self.Ny, self.R = Nx, Ny, R
        self.lf, self.mu, self.K = float(lambda_forget), float(mu), int(mm_iters)
        if update not in ("gauss_seidel", "jacobi"):
            raise ValueError(update)
        self.update = update
        self.A1 = np.zeros((Nx, R), np.complex128) if A1 is None else np.array(A1, np.complex128)
        self.A2 = np.zeros((Ny, R), np.complex128) if A2 is None else np.array(A2, np.complex128)
        self.abar_A = self.abar_B = self.w = 0.0
        self.t = 0
        self.gamma = np.zeros(R, np.complex128)
        self.trace = []

    def push_frame(self, y_rows: np.ndarray, mask: np.ndarray, record=False) -> np.ndarray:
        """Frame t: y_rows (|S| x Ny) the acquired k-space rows in increasing row order.
        Returns the image F^{-1}(A1[t] diag(gamma_t) A2[t]^T) (Alg. 2, §IV-A)."""
        rows = np.flatnonzero(np.asarray(mask))
        Y = T.zero_filled(np.asarray(y_rows, np.complex128), rows, self.Nx)
        y = Y[rows, :].reshape(-1)
        lf, mu = self.lf, self.mu
        self.w = lf * self.w + 1.0
        rho = mu / self.w
        P0, Q0 = self.A1.copy(), self.A2.copy()
        P, Q, gamma = self.A1, self.A2, self.gamma
        alpha_A = alpha_B = rho
        self.trace = []

        def H(P_, Q_, g_):
            return ks_objective_J(P_, Q_, g_, Y, rows, mu, rho) \
                + 0.5 * lf * self.abar_A * float(np.vdot(P_ - P0, P_ - P0).real) \
                + 0.5 * lf * self.abar_B * float(np.vdot(Q_ - Q0, Q_ - Q0).real)

        if record:
            self.trace.append(("start", H(P, Q, gamma)))
        for _ in range(self.K):
            gamma = T.ridge_gamma(ks_phi(P, Q, rows), y, mu)                    # (S1)
            if record:
                self.trace.append(("gamma", H(P, Q, gamma)))
            if self.update == "gauss_seidel":                                    # (S2)
                alpha_A = T.lipschitz_A(Q, gamma, rho)
                P = T.mm_step(P, P0, ks_gradient_A1(P, Q, gamma, Y, rows, rho), alpha_A, self.abar_A, lf)
                if record:
                    self.trace.append(("A", H(P, Q, gamma)))
                alpha_B = T.lipschitz_B(P, gamma, rho)
                Q = T.mm_step(Q, Q0, ks_gradient_A2(P, Q, gamma, Y, rows, rho), alpha_B, self.abar_B, lf)
                if record:
                    self.trace.append(("B", H(P, Q, gamma)))
            else:
                alpha_A = T.lipschitz_A(Q, gamma, rho)
                alpha_B = T.lipschitz_B(P, gamma, rho)
                gP = ks_gradient_A1(P, Q, gamma, Y, rows, rho)
                gQ = ks_gradient_A2(P, Q, gamma, Y, rows, rho)
                P, Q = (T.mm_step(P, P0, gP, alpha_A, self.abar_A, lf), T.mm_step(Q, Q0, gQ, alpha_B, self.abar_B, lf))
                if record:
                    self.trace.append(("AB", H(P, Q, gamma)))
        self.abar_A = lf * self.abar_A + alpha_A
        self.abar_B = lf * self.abar_B + alpha_B
        self.A1, self.A2, self.gamma = P, Q, gamma
        self.t += 1
        return self.image()

    def kspace(self) -> np.ndarray:
        """The interpolated k-space frame X_t = A1[t] diag(gamma_t) A2[t]^T (§IV-A)."""
        return self.A1 @ np.diag(self.gamma) @ self.A2.T

    def image(self) -> np.ndarray:
        """F^{-1}(X_t) (§IV-A); the paper's image is its magnitude."""
        return T.ifft2(self.kspace())

    def line_probs(self) -> np.ndarray:
        """Line scores of §V-B (eq. score) on the k-space factor A1, marginalised (§VI-C)."""
        return ks_line_probs(self.A1, self.Ny)

    def next_mask(self, k_lines: int, central: int, seed: int, stream_id: int = 0,
                  with_replacement: bool = False) -> np.ndarray:
        """The lines of the next frame drawn from line_probs (Alg. 4)."""
        ctr = T.line_draw_counter(self.t, stream_id)
        return T.sample_lines_from_probs(self.line_probs(), k_lines, central, seed, ctr, with_replacement)


def ks_line_probs(A1: np.ndarray, Ny: int) -> np.ndarray:
    """The informative line scores of §V-B marginalised over readout (§VI-C) on the
    k-space factor itself (Alg. 2 keeps its factor in k-space): s_i = (Ny ||abar_i||^2 + R)
    / (R (Nx + Ny)) with abar the rows of the column-normalised A1; a zero column scores
    uniformly."""
    Nx, R = A1.shape
    norms2 = np.sum(np.abs(A1) ** 2, axis=0)
    Abar2 = np.empty((Nx, R))
    for r in range(R):
        Abar2[:, r] = np.abs(A1[:, r]) ** 2 / norms2[r] if norms2[r] > 0.0 else 1.0 / Nx
    return (Ny * np.sum(Abar2, axis=1) + R) / (R * (Nx + Ny))
