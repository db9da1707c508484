"""FP64 CPU oracle of the multi-coil (tomographic parallel MRI) tracker: Alg. 3 of the
paper with C coils of known sensitivity (§IV-B, "Tomographic parallel MRI").

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
and reference legs may import this module. The product library never does, and this
module imports nothing from it.

Data model (§IV-B): coil c sees y_c^{(i,j)} = [F(H_c .* L_t)]_{ij} + v, (i, j) in Omega_t,
with H_c the Nx x Ny complex sensitivity of coil c. Alg. 3 then reads:
  (S1) Phi stacks the coils' masked 2D DFTs of the sensitivity-weighted rank-one images,
       column r = [vec_Omega F(H_1 .* a_r b_r^T); ...; vec_Omega F(H_C .* a_r b_r^T)],
       and gamma solves the ridge problem on the stacked data y = [y_1; ...; y_C];
  (S2) the gradient uses Theta = sum_c conj(H_c) .* F^{-1}(Xi_c) with Xi_c the coil's
       residual on Omega, zero elsewhere: grad_A = rho A - Theta conj(B) diag(conj gamma),
       grad_B = rho B - Theta^T conj(A) diag(conj gamma).
The readings of tracker.py (forgetting, several Gauss-Seidel MM iterations, the surrogate
minimiser) carry over. The one change is the majoriser weight of a factor block: the map
A -> {P_Omega F(H_c .* (A D B^T))}_c has squared norm at most
h_max ||D B^T||_F^2 with h_max = max_ij sum_c |H_c[i,j]|^2 (F unitary, P_Omega a
projection), so alpha_A = h_max sum_r |gamma_r|^2 ||b_r||^2 + rho (likewise alpha_B with
||a_r||). With C = 1 and H_1 = all-ones this is exactly the single-coil tracker.
"""
from __future__ import annotations

import numpy as np

from . import tracker as T


def mc_phi(A: np.ndarray, B: np.ndarray, H: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """Phi of Alg. 3 (S1) with coils: column r stacks vec_Omega F(H_c .* a_r b_r^T) over
    c = 1..C, Omega = rows x [Ny] vectorised row by row. Shape (C |S| Ny) x R."""
    C = H.shape[0]
    R = A.shape[1]
    cols = []
    for r in range(R):
        img = np.outer(A[:, r], B[:, r])
        cols.append(np.concatenate([T.fft2(H[c] * img)[rows, :].reshape(-1) for c in range(C)]))
    return np.stack(cols, axis=1)


def mc_data(Y: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """The stacked observations y = [y_1; ...; y_C] of the coils (§IV-B data model) from
    zero-filled coil frames Y (C x Nx x Ny)."""
    return np.concatenate([Y[c][rows, :].reshape(-1) for c in range(Y.shape[0])])


def mc_residual(A, B, gamma, H, Y, rows) -> np.ndarray:
    """Xi_c = P_Omega(Y_c - F(H_c .* (A diag(gamma) B^T))), zero off Omega; C x Nx x Ny: each
    coil's k-space residual of Alg. 3 (S2) (§IV-B)."""
    X = A @ np.diag(gamma) @ B.T
    E = np.zeros_like(Y)
    for c in range(H.shape[0]):
        E[c][rows, :] = Y[c][rows, :] - T.fft2(H[c] * X)[rows, :]
    return E


def mc_theta(E: np.ndarray, H: np.ndarray) -> np.ndarray:
    """Theta = sum_c conj(H_c) .* F^{-1}(Xi_c) (Alg. 3 (S2))."""
    return sum(np.conj(H[c]) * T.ifft2(E[c]) for c in range(H.shape[0]))


def mc_objective_J(A, B, gamma, H, Y, rows, mu, rho) -> float:
    """J = 1/2 sum_c ||P_Omega(y_c - F(H_c .* (A diag gamma B^T)))||^2 + mu/2 ||gamma||^2
    + rho/2 (||A||^2 + ||B||^2): f_t of §III-A for the coil model of §IV-B."""
    E = mc_residual(A, B, gamma, H, Y, rows)
    return 0.5 * float(np.vdot(E, E).real) + 0.5 * mu * float(np.vdot(gamma, gamma).real) \
        + 0.5 * rho * float(np.vdot(A, A).real + np.vdot(B, B).real)


def mc_gradient_A(A, B, gamma, H, Y, rows, rho) -> np.ndarray:
    """grad_A = rho A - Theta conj(B) diag(conj gamma), Theta from every coil (Alg. 3 (S2))."""
    Theta = mc_theta(mc_residual(A, B, gamma, H, Y, rows), H)
    return rho * A - Theta @ np.conj(B) @ np.diag(np.conj(gamma))


def mc_gradient_B(A, B, gamma, H, Y, rows, rho) -> np.ndarray:
    """grad_B = rho B - Theta^T conj(A) diag(conj gamma) (Alg. 3 (S2))."""
    Theta = mc_theta(mc_residual(A, B, gamma, H, Y, rows), H)
    return rho * B - Theta.T @ np.conj(A) @ np.diag(np.conj(gamma))


def h_max(H: np.ndarray) -> float:
    """max over pixels of sum_c |H_c|^2: the factor by which the coil operator can scale the
    majoriser of a factor block (the reading stated in this module's header)."""
    return float(np.max(np.sum(np.abs(H) ** 2, axis=0)))


def mc_lipschitz_A(B, gamma, rho, hmax) -> float:
    """alpha_A = h_max sum_r |gamma_r|^2 ||b_r||^2 + rho: the A-block Hessian bound of §III-A
    under the coil operator."""
    return float(hmax * np.sum(np.abs(gamma) ** 2 * np.sum(np.abs(B) ** 2, axis=0)) + rho)


def mc_lipschitz_B(A, gamma, rho, hmax) -> float:
    """alpha_B = h_max sum_r |gamma_r|^2 ||a_r||^2 + rho (B block, as mc_lipschitz_A)."""
    return float(hmax * np.sum(np.abs(gamma) ** 2 * np.sum(np.abs(A) ** 2, axis=0)) + rho)


class MultiCoilTracker:
    """Online multi-coil tracker (Alg. 3 with C coils, Gauss-Seidel MM iterations,
    forgotten surrogates); the state is that of tracker.Tracker."""

    def __init__(self, Nx, Ny, R, H, lambda_forget, mu, mm_iters=1, A=None, B=None):
        self.Nx, self.Ny, self.R = Nx, Ny, R
        self.H = np.array(H, np.complex128)
        self.C = self.H.shape[0]
        self.hmax = h_max(self.H)
        self.lf = float(lambda_forget)
        self.mu = float(mu)
        self.K = int(mm_iters)
        self.A = np.zeros((Nx, R), np.complex128) if A is None else np.array(A, np.complex128)
        self.B = np.zeros((Ny, R), np.complex128) if B is None else np.array(B, np.complex128)
        self.abar_A = self.abar_B = self.w = 0.0
        self.t = 0
        self.gamma = np.zeros(R, np.complex128)
        self.trace = []

    def push_frame(self, y_rows: np.ndarray, mask: np.ndarray, record=False) -> np.ndarray:
        """Frame t: y_rows (C x |S| x Ny) are each coil's acquired rows in increasing row
        order. Returns X_t = A[t] diag(gamma_t) B[t]^T (Alg. 3 with C coils, §IV-B)."""
        rows = np.flatnonzero(np.asarray(mask))
        Y = np.zeros((self.C, self.Nx, self.Ny), np.complex128)
        Y[:, rows, :] = np.asarray(y_rows, np.complex128)
        y = mc_data(Y, rows)
        lf, mu, H = self.lf, self.mu, self.H
        self.w = lf * self.w + 1.0
        rho = mu / self.w
        A0, B0 = self.A.copy(), self.B.copy()
        A, B, gamma = self.A, self.B, self.gamma
        alpha_A = alpha_B = rho
        self.trace = []

        def Hobj(A_, B_, g_):
            return mc_objective_J(A_, B_, g_, H, Y, rows, mu, rho) \
                + 0.5 * lf * self.abar_A * float(np.vdot(A_ - A0, A_ - A0).real) \
                + 0.5 * lf * self.abar_B * float(np.vdot(B_ - B0, B_ - B0).real)

        if record:
            self.trace.append(("start", Hobj(A, B, gamma)))
        for _ in range(self.K):
            Phi = mc_phi(A, B, H, rows)                    # (S1)
            gamma = T.ridge_gamma(Phi, y, mu)
            if record:
                self.trace.append(("gamma", Hobj(A, B, gamma)))
            alpha_A = mc_lipschitz_A(B, gamma, rho, self.hmax)   # (S2), A block
            A = T.mm_step(A, A0, mc_gradient_A(A, B, gamma, H, Y, rows, rho), alpha_A, self.abar_A, lf)
            if record:
                self.trace.append(("A", Hobj(A, B, gamma)))
            alpha_B = mc_lipschitz_B(A, gamma, rho, self.hmax)   # B block, residual refreshed
            B = T.mm_step(B, B0, mc_gradient_B(A, B, gamma, H, Y, rows, rho), alpha_B, self.abar_B, lf)
            if record:
                self.trace.append(("B", Hobj(A, B, gamma)))
        self.abar_A = lf * self.abar_A + alpha_A
        self.abar_B = lf * self.abar_B + alpha_B
        self.A, self.B, self.gamma = A, B, gamma
        self.t += 1
        return self.image()

    def image(self) -> np.ndarray:
        """X_t = A[t] diag(gamma_t) B[t]^T, the image the coils share (§IV-B)."""
        return self.A @ np.diag(self.gamma) @ self.B.T
