"""FP64 CPU oracle of the online PARAFAC tensor-subspace tracker for undersampled
dynamic MRI (Mardani, Giannakis, Ugurbil: "Tracking tensor subspaces with informative
random sampling for real-time MR imaging").

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
and reference legs may import this module. The product library never does, and this
module imports nothing from it.

It is plain and slow on purpose: every transform is the DFT matrix applied as a dense
product, the regression matrix Phi is formed column by column from the masked 2D DFT of
each rank-one image, and each step follows the paper's algorithm in its order.

Readings of the paper that this oracle takes (the paper is silent or the text is
garbled there):
  * Single coil, H_1 = all-ones (Alg. 3 with C = 1): the image-domain tracker.
  * The factor penalty of f_t is (mu / (2 w)) ||.||_F^2 with w the forgotten frame
    count (w = t when lambda_forget = 1, which is the paper's lambda/(2t), eq. f_t).
  * The past surrogates are forgotten geometrically: the surrogate minimiser of §III-A
    becomes A <- (lf*abar*A0 + alpha*A - grad) / (lf*abar + alpha), which for
    lambda_forget = 1 and one iteration is exactly A[t] = A[t-1] - grad / abar_t
    (the recursion for A_m[t] in §III-A).
  * Several MM iterations per frame, Gauss-Seidel order gamma -> A -> B (Jacobi, the
    paper's parallel form of Alg. 3 (S2), is an option).
  * alpha for the A block is sum_r |gamma_r|^2 ||b_r||^2 + rho, an upper bound of the
    block Hessian of f_t (eq. for the Hessian in §III-A) because the Frobenius norm
    bounds the spectral norm; likewise with ||a_r|| for the B block.
  * The ridge step solves (Phi^H Phi + mu I) gamma = Phi^H y (§III-A, (S1) closed form;
    the transposes there are Hermitian transposes for complex data).
  * Scores are computed on the k-space factor F_Nx A (rows = phase-encode lines),
    marginalised over readout as in §VI-C.
  * Line draws: central lines forced; the remaining lines drawn from an integer CDF
    q_i = floor(p_i 2^52) with Philox4x32-10 uniforms, duplicates rejected.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg

from . import philox

# ---------------------------------------------------------------------------------
# §IV: the 2D DFT in matrix form F(X) = F_l X F_r with orthonormal symmetric DFT
# matrices. (F_N)_{k,n} = N^{-1/2} exp(-2 pi i k n / N), DC at index 0.
# ---------------------------------------------------------------------------------


def dft_matrix(N: int) -> np.ndarray:
    """Unitary, symmetric DFT matrix of size N (complex128): the F_l, F_r of the 2D DFT in
    matrix form F(X) = F_l X F_r (§IV)."""
    k = np.arange(N)
    kn = np.outer(k, k) % N            # exact integer phase index before the angle
    return np.exp(-2j * np.pi * kn / N) / math.sqrt(N)


def fft2(X: np.ndarray) -> np.ndarray:
    """F(X) = F_Nx X F_Ny (§IV)."""
    Nx, Ny = X.shape
    return dft_matrix(Nx) @ X @ dft_matrix(Ny)


def ifft2(Y: np.ndarray) -> np.ndarray:
    """F^{-1}(Y) = conj(F_Nx) Y conj(F_Ny) (F unitary and symmetric, §IV)."""
    Nx, Ny = Y.shape
    return np.conj(dft_matrix(Nx)) @ Y @ np.conj(dft_matrix(Ny))


# ---------------------------------------------------------------------------------
# §III-A (S1): ridge regression for the temporal factor gamma_t.
# ---------------------------------------------------------------------------------


def phi_matrix(A: np.ndarray, B: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """Phi_t: column r is vec over Omega of F(a_r b_r^T) (Alg. 3 (S1) with H_1 = 1),
    Omega = rows x [Ny], vectorised row by row. Shape (|S| Ny) x R."""
    R = A.shape[1]
    cols = []
    for r in range(R):
        img = np.outer(A[:, r], B[:, r])
        cols.append(fft2(img)[rows, :].reshape(-1))
    return np.stack(cols, axis=1)


def ridge_gram(Phi: np.ndarray, y: np.ndarray, mu: float) -> tuple[np.ndarray, np.ndarray]:
    """G = Phi^H Phi + mu I and h = Phi^H y: the normal equations of the ridge step (S1) of
    Alg. 3 (closed form of §III-A)."""
    R = Phi.shape[1]
    G = Phi.conj().T @ Phi + mu * np.eye(R)
    h = Phi.conj().T @ y
    return G, h


def cholesky_solve(G: np.ndarray, h: np.ndarray) -> np.ndarray:
    """gamma = G^{-1} h via the Cholesky factor G = L L^H (LAPACK); solves the (S1) system of
    §III-A, G Hermitian positive definite for mu > 0."""
    c = scipy.linalg.cho_factor(G, lower=True)
    return scipy.linalg.cho_solve(c, h)


def ridge_gamma(Phi: np.ndarray, y: np.ndarray, mu: float) -> np.ndarray:
    """(S1) of Alg. 3: gamma = (Phi^H Phi + mu I)^{-1} Phi^H y (the ridge closed form of
    §III-A)."""
    G, h = ridge_gram(Phi, y, mu)
    return cholesky_solve(G, h)


def ridge_gamma_svd(Phi: np.ndarray, y: np.ndarray, mu: float) -> np.ndarray:
    """The SVD form of (S1) as in Alg. 3: Phi = U Sigma V^H, gamma = V D U^H y with
    D = diag(sigma_i / (sigma_i^2 + mu)). Used only to pin the Cholesky form."""
    U, s, Vh = np.linalg.svd(Phi, full_matrices=False)
    return Vh.conj().T @ ((s / (s * s + mu)) * (U.conj().T @ y))


# ---------------------------------------------------------------------------------
# The per-frame objective (instantaneous cost f_t of §III-A with the readings above)
# ---------------------------------------------------------------------------------


def zero_filled(y_rows: np.ndarray, rows: np.ndarray, Nx: int) -> np.ndarray:
    """P_Omega^T y: the observed rows placed in an Nx x Ny array of zeros (the sampling
    operator of the subsampled data model, §II-B, with Omega = S x [Ny])."""
    Y = np.zeros((Nx, y_rows.shape[1]), np.complex128)
    Y[rows, :] = y_rows
    return Y


def residual(A, B, gamma, Y, rows) -> np.ndarray:
    """Xi = P_Omega(Y - F(A diag(gamma) B^T)), zero off Omega (Alg. 3, e_c^{(i,j)})."""
    X = A @ np.diag(gamma) @ B.T
    E = np.zeros_like(Y)
    E[rows, :] = Y[rows, :] - fft2(X)[rows, :]
    return E


def objective_J(A, B, gamma, Y, rows, mu, rho) -> float:
    """J = 1/2 ||P_Omega(y - F(A diag gamma B^T))||^2 + mu/2 ||gamma||^2
    + rho/2 (||A||^2 + ||B||^2): the instantaneous cost f_t of §III-A with the factor
    penalty weight rho = mu / w of the forgetting reading."""
    E = residual(A, B, gamma, Y, rows)
    return 0.5 * float(np.vdot(E, E).real) + 0.5 * mu * float(np.vdot(gamma, gamma).real) \
        + 0.5 * rho * float(np.vdot(A, A).real + np.vdot(B, B).real)


def gradient_A(A, B, gamma, Y, rows, rho) -> np.ndarray:
    """Gradient of J in A (real-coordinate gradient packed as complex), eq. for the
    column gradient in §III-A specialised by Alg. 3: rho A - Theta conj(B) diag(conj gamma)
    with Theta = F^{-1}(Xi)."""
    Theta = ifft2(residual(A, B, gamma, Y, rows))
    return rho * A - Theta @ np.conj(B) @ np.diag(np.conj(gamma))


def gradient_B(A, B, gamma, Y, rows, rho) -> np.ndarray:
    """rho B - Theta^T conj(A) diag(conj gamma) (Alg. 3 (S2), second factor)."""
    Theta = ifft2(residual(A, B, gamma, Y, rows))
    return rho * B - Theta.T @ np.conj(A) @ np.diag(np.conj(gamma))


def lipschitz_A(B, gamma, rho) -> float:
    """alpha_A = sum_r |gamma_r|^2 ||b_r||^2 + rho: an upper bound of the A-block Hessian of
    f_t (§III-A), Frobenius over spectral norm."""
    return float(np.sum(np.abs(gamma) ** 2 * np.sum(np.abs(B) ** 2, axis=0)) + rho)


def lipschitz_B(A, gamma, rho) -> float:
    """alpha_B = sum_r |gamma_r|^2 ||a_r||^2 + rho: the B-block counterpart of lipschitz_A
    (§III-A)."""
    return float(np.sum(np.abs(gamma) ** 2 * np.sum(np.abs(A) ** 2, axis=0)) + rho)


def mm_step(X, X0, grad, alpha, abar, lf) -> np.ndarray:
    """Minimiser of the forgotten past surrogates (lf*abar/2 ||X - X0||^2 up to a
    constant) plus the quadratic majoriser of f_t at X (§III-A):
    X <- (lf*abar*X0 + alpha*X - grad) / (lf*abar + alpha)."""
    return (lf * abar * X0 + alpha * X - grad) / (lf * abar + alpha)


class Tracker:
    """Online tracker state and the per-frame update (Alg. 3 with C = 1, Alg. 5 order).

    State after frame t-1: factors A (Nx x R), B (Ny x R), the surrogate weights
    abar_A, abar_B, the forgotten frame count w and the frame counter t."""

    def __init__(self, Nx, Ny, R, lambda_forget, mu, mm_iters=1, update="gauss_seidel",
                 A=None, B=None):
        self.Nx, self.Ny, self.R = Nx, Ny, R
        self.lf = float(lambda_forget)
        self.mu = float(mu)
        self.K = int(mm_iters)
        if update not in ("gauss_seidel", "jacobi"):
            raise ValueError(update)
        self.update = update
        self.A = np.zeros((Nx, R), np.complex128) if A is None else np.array(A, np.complex128)
        self.B = np.zeros((Ny, R), np.complex128) if B is None else np.array(B, np.complex128)
        self.abar_A = 0.0
        self.abar_B = 0.0
        self.w = 0.0
        self.t = 0
        self.gamma = np.zeros(R, np.complex128)
        self.trace = []          # per-substep objective values of the last frame (H)

    # -- state access ---------------------------------------------------------------
    def state(self) -> dict:
        return dict(A=self.A.copy(), B=self.B.copy(), abar_A=self.abar_A, abar_B=self.abar_B,
                    w=self.w, t=self.t, gamma=self.gamma.copy())

    def load(self, st: dict) -> None:
        self.A = np.array(st["A"], np.complex128)
        self.B = np.array(st["B"], np.complex128)
        self.abar_A, self.abar_B = float(st["abar_A"]), float(st["abar_B"])
        self.w, self.t = float(st["w"]), int(st["t"])
        self.gamma = np.array(st.get("gamma", np.zeros(self.R)), np.complex128)

    # -- one frame ------------------------------------------------------------------
    def push_frame(self, y_rows: np.ndarray, mask: np.ndarray, record=False) -> np.ndarray:
        """Process frame t: y_rows are the acquired rows (|S| x Ny, increasing row
        order) and mask the Nx-byte line mask with S = flatnonzero(mask).
        Returns the reconstructed image X_t = A[t] diag(gamma_t) B[t]^T. The steps are those of
        Alg. 3 with one coil ((S1) ridge, (S2) majorised factor steps, §III-A surrogates),
        repeated mm_iters times."""
        rows = np.flatnonzero(np.asarray(mask))
        Y = zero_filled(np.asarray(y_rows, np.complex128), rows, self.Nx)
        y = Y[rows, :].reshape(-1)
        lf, mu = self.lf, self.mu
        # step 1: forgotten frame count and the factor penalty weight rho = mu / w
        self.w = lf * self.w + 1.0
        rho = mu / self.w
        # step 2: anchors A[t-1], B[t-1] of the past surrogates
        A0, B0 = self.A.copy(), self.B.copy()
        A, B = self.A, self.B
        gamma = self.gamma
        alpha_A = alpha_B = rho
        self.trace = []

        def H(A_, B_, g_):
            return objective_J(A_, B_, g_, Y, rows, mu, rho) \
                + 0.5 * lf * self.abar_A * float(np.vdot(A_ - A0, A_ - A0).real) \
                + 0.5 * lf * self.abar_B * float(np.vdot(B_ - B0, B_ - B0).real)

        if record:
            self.trace.append(("start", H(A, B, gamma)))
        for _ in range(self.K):
            # (S1) regression matrix from the masked DFTs of the rank-one images,
            # ridge solve for gamma
            Phi = phi_matrix(A, B, rows)
            gamma = ridge_gamma(Phi, y, mu)
            if record:
                self.trace.append(("gamma", H(A, B, gamma)))
            if self.update == "gauss_seidel":
                # (S2) A block: gradient at the current iterate, majorised step
                alpha_A = lipschitz_A(B, gamma, rho)
                gA = gradient_A(A, B, gamma, Y, rows, rho)
                A = mm_step(A, A0, gA, alpha_A, self.abar_A, lf)
                if record:
                    self.trace.append(("A", H(A, B, gamma)))
                # B block with the refreshed residual (uses the new A)
                alpha_B = lipschitz_B(A, gamma, rho)
                gB = gradient_B(A, B, gamma, Y, rows, rho)
                B = mm_step(B, B0, gB, alpha_B, self.abar_B, lf)
                if record:
                    self.trace.append(("B", H(A, B, gamma)))
            else:
                # Jacobi: both blocks from the same iterate (Alg. 3 (S2) in parallel)
                alpha_A = lipschitz_A(B, gamma, rho)
                alpha_B = lipschitz_B(A, gamma, rho)
                gA = gradient_A(A, B, gamma, Y, rows, rho)
                gB = gradient_B(A, B, gamma, Y, rows, rho)
                A, B = (mm_step(A, A0, gA, alpha_A, self.abar_A, lf),
                        mm_step(B, B0, gB, alpha_B, self.abar_B, lf))
                if record:
                    self.trace.append(("AB", H(A, B, gamma)))
        # surrogate weights: forgotten sums of the last iteration's alphas
        self.abar_A = lf * self.abar_A + alpha_A
        self.abar_B = lf * self.abar_B + alpha_B
        self.A, self.B, self.gamma = A, B, gamma
        self.t += 1
        return self.image()

    def image(self) -> np.ndarray:
        """X_t = A[t] diag(gamma_t) B[t]^T (the image-domain analogue of the
        interpolated frame of §IV-A)."""
        return self.A @ np.diag(self.gamma) @ self.B.T

    # -- S0: the next frame's lines ------------------------------------------------
    def line_probs(self) -> np.ndarray:
        """The line scores of §V-B (eq. score) for the next frame, marginalised (§VI-C)."""
        return informative_line_probs(self.A, self.Ny)

    def next_mask(self, k_lines: int, central: int, seed: int, stream_id: int = 0,
                  with_replacement: bool = False) -> np.ndarray:
        """Draw the lines of frame t (the next frame to be pushed) from the scores
        of the current subspace (Alg. 4 marginalised over readout, §VI-C)."""
        ctr = line_draw_counter(self.t, stream_id)
        return sample_lines_from_probs(self.line_probs(), k_lines, central, seed, ctr,
                                       with_replacement)


# ---------------------------------------------------------------------------------
# §V: importance scores and randomized line selection (Alg. 4, eq. score, §VI-C)
# ---------------------------------------------------------------------------------


def informative_line_probs(A: np.ndarray, Ny: int) -> np.ndarray:
    """s(n1) = (Ny ||abar_{n1}||^2 + R) / (R (Nx + Ny)) with abar the rows of the
    column-normalised k-space factor F_Nx A (§V-B score, marginalised as in §VI-C).
    A zero column contributes uniformly (|abar_{i,r}|^2 = 1/Nx)."""
    Nx, R = A.shape
    Ahat = dft_matrix(Nx) @ A
    norms2 = np.sum(np.abs(Ahat) ** 2, axis=0)
    Abar2 = np.empty((Nx, R))
    for r in range(R):
        if norms2[r] > 0.0:
            Abar2[:, r] = np.abs(Ahat[:, r]) ** 2 / norms2[r]
        else:
            Abar2[:, r] = 1.0 / Nx
    row = np.sum(Abar2, axis=1)
    return (Ny * row + R) / (R * (Nx + Ny))


def uniform_line_probs(Nx: int) -> np.ndarray:
    """Uniform random phase-encode lines: the masks of the small-cine workload (the paper
    itself compares its scores with the variable-density policy, §VI-C)."""
    return np.full(Nx, 1.0 / Nx)


def vardens_line_probs(Nx: int, alpha: float) -> np.ndarray:
    """Variable-density weights p_i proportional to d_i^alpha, d_i >= 1 the distance of
    line i from the centre line (§VI, polynomial distribution; DC at index 0)."""
    i = np.arange(Nx)
    d = np.minimum(i, Nx - i).astype(np.float64)
    d = np.maximum(d, 1.0)
    if alpha == -1.0:
        wgt = 1.0 / d
    elif alpha == -0.5:
        wgt = 1.0 / np.sqrt(d)
    else:
        wgt = d ** alpha
    return wgt / np.sum(wgt)


PURPOSE_LINES = 1


def line_draw_counter(t: int, stream_id: int = 0) -> int:
    """64-bit draw context of frame t of a stream: (stream_id << 40) | t. The paper leaves
    the random source of the draws of Alg. 4 open; this counter layout is this oracle's."""
    return ((int(stream_id) & 0xFFFFFF) << 40) | (int(t) & ((1 << 40) - 1))


def central_lines(Nx: int, central: int) -> list[int]:
    """{-c/2, ..., c/2 - 1} mod Nx: the always-acquired low-frequency lines (DC at index 0) of
    the Cartesian masks of §VI."""
    c = min(central, Nx)
    return sorted(((k - c // 2) % Nx) for k in range(c))


def sample_lines_from_probs(p, k_lines: int, central: int, seed: int, ctr: int,
                            with_replacement: bool = False) -> np.ndarray:
    """Random line selection of Alg. 4 for Cartesian lines.

    The central lines are always kept. The other lines carry integer weights
    q_i = floor(p_i 2^52) with inclusive prefix sums Q. Draw d uses the Philox4x32-10
    block at counter (d, PURPOSE_LINES, ctr_lo, ctr_hi) under key (seed_lo, seed_hi);
    u = word0 | word1 << 32, x = floor(u * Q_total / 2^64), and the drawn line is the
    first with Q > x. Without replacement a line drawn twice is rejected and drawing
    goes on until k_lines lines are held or 64 * (k_lines - central) draws are spent,
    after which the remaining lines are taken in decreasing q (lower index first on
    ties). With replacement exactly k_lines - central draws are made."""
    p = np.asarray(p, np.float64)
    Nx = p.shape[0]
    mask = np.zeros(Nx, np.uint8)
    for i in central_lines(Nx, central):
        mask[i] = 1
    k_lines = min(int(k_lines), Nx)
    need = k_lines - int(mask.sum())
    if need <= 0:
        return mask
    cand = [i for i in range(Nx) if not mask[i]]
    two52 = float(1 << 52)
    q = [int(math.floor(float(p[i]) * two52)) if p[i] > 0.0 else 0 for i in cand]
    Q = []
    acc = 0
    for v in q:
        acc += v
        Q.append(acc)
    Qtot = acc
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    c_lo, c_hi = ctr & 0xFFFFFFFF, (ctr >> 32) & 0xFFFFFFFF
    got = 0
    if Qtot > 0:
        n_draws = need if with_replacement else 64 * need
        for d in range(n_draws):
            w0, w1, _, _ = philox.philox4x32_10((d & 0xFFFFFFFF, PURPOSE_LINES, c_lo, c_hi), key)
            u = w0 | (w1 << 32)
            x = (u * Qtot) >> 64
            k = _upper_bound(Q, x)
            line = cand[k]
            if with_replacement:
                mask[line] = 1
                continue
            if not mask[line]:
                mask[line] = 1
                got += 1
                if got == need:
                    break
    if not with_replacement and got < need:
        rest = [(-q[k], cand[k]) for k in range(len(cand)) if not mask[cand[k]]]
        rest.sort()
        for _, line in rest[: need - got]:
            mask[line] = 1
    return mask


def _upper_bound(Q: list[int], x: int) -> int:
    """First index k with Q[k] > x (binary search): inverts the integer CDF for one draw of
    Alg. 4."""
    lo, hi = 0, len(Q)
    while lo < hi:
        mid = (lo + hi) // 2
        if Q[mid] > x:
            hi = mid
        else:
            lo = mid + 1
    return lo


def expected_distinct_lines(p_cand: np.ndarray, n_draws: int) -> float:
    """E|Omega| = sum_i (1 - (1 - s_i)^K) for K draws with replacement (§V-B)."""
    return float(np.sum(1.0 - (1.0 - np.asarray(p_cand)) ** n_draws))


def nrmse(x: np.ndarray, ref: np.ndarray) -> float:
    """||x - ref||_F / ||ref||_F: the square root of the per-frame NMSE of §VI-A."""
    return float(np.linalg.norm(np.asarray(x) - ref) / np.linalg.norm(ref))
