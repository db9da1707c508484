"""Pins of the FP64 oracle against what the paper and the mathematics fix
(closed forms, identities, brute force on tiny inputs, invariants). CPU only."""
import math

import numpy as np
import pytest

from oracle import philox
from oracle import tracker as O


def cn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# ----------------------------------------------------------------------------------
# DFT (§IV: F(X) = F_l X F_r, orthonormal symmetric DFT matrices)
# ----------------------------------------------------------------------------------

@pytest.mark.parametrize("Nx,Ny", [(1, 1), (2, 3), (4, 4), (5, 7), (6, 10), (12, 9)])
def test_dft_matches_bruteforce_2d_sum(Nx, Ny):
    rng = np.random.default_rng(Nx * 100 + Ny)
    X = cn(rng, Nx, Ny)
    ref = np.zeros((Nx, Ny), np.complex128)
    for k in range(Nx):
        for l in range(Ny):
            s = 0j
            for n in range(Nx):
                for m in range(Ny):
                    s += X[n, m] * np.exp(-2j * np.pi * (k * n / Nx + l * m / Ny))
            ref[k, l] = s / math.sqrt(Nx * Ny)
    np.testing.assert_allclose(O.fft2(X), ref, atol=1e-12)


@pytest.mark.parametrize("N", [1, 3, 8, 12, 64, 160, 192, 256])
def test_dft_matrix_unitary_symmetric(N):
    F = O.dft_matrix(N)
    np.testing.assert_allclose(F, F.T, atol=0)
    np.testing.assert_allclose(F @ F.conj().T, np.eye(N), atol=1e-12)


def test_dft_against_library_fft_and_closed_forms():
    rng = np.random.default_rng(1)
    X = cn(rng, 24, 20)
    np.testing.assert_allclose(O.fft2(X), np.fft.fft2(X, norm="ortho"), atol=1e-12)
    # Parseval and inverse
    assert abs(np.linalg.norm(O.fft2(X)) - np.linalg.norm(X)) < 1e-12 * np.linalg.norm(X)
    np.testing.assert_allclose(O.ifft2(O.fft2(X)), X, atol=1e-12)
    # impulse at the origin -> constant 1/sqrt(Nx Ny); constant -> impulse at DC
    d = np.zeros((6, 10)); d[0, 0] = 1.0
    np.testing.assert_allclose(O.fft2(d), np.full((6, 10), 1 / math.sqrt(60)), atol=1e-14)
    c = np.ones((6, 10))
    e = np.zeros((6, 10)); e[0, 0] = math.sqrt(60)
    np.testing.assert_allclose(O.fft2(c), e, atol=1e-12)
    # a shifted impulse gives a linear phase with the minus sign of the forward DFT
    s = np.zeros((8, 8)); s[1, 0] = 1.0
    k = np.arange(8)
    np.testing.assert_allclose(O.fft2(s)[:, 0], np.exp(-2j * np.pi * k / 8) / 8, atol=1e-14)


# ----------------------------------------------------------------------------------
# Phi and the normal equations (Alg. 3 (S1)); separable closed form
# ----------------------------------------------------------------------------------

def test_phi_gram_separable_closed_form():
    """With Omega = S x [Ny], Phi^H Phi = (Ahat_S^H Ahat_S) .* (B^H B) with
    Ahat = F_Nx A (F(a b^T) = (F a)(F b)^T and F_Ny unitary)."""
    rng = np.random.default_rng(2)
    Nx, Ny, R = 10, 7, 3
    A, B = cn(rng, Nx, R), cn(rng, Ny, R)
    rows = np.array([0, 3, 4, 9])
    Phi = O.phi_matrix(A, B, rows)
    Ah = O.dft_matrix(Nx) @ A
    G_sep = (Ah[rows].conj().T @ Ah[rows]) * (B.conj().T @ B)
    np.testing.assert_allclose(Phi.conj().T @ Phi, G_sep, rtol=1e-12, atol=1e-12)
    # full sampling: (A^H A) .* (B^H B)
    Phi_f = O.phi_matrix(A, B, np.arange(Nx))
    np.testing.assert_allclose(Phi_f.conj().T @ Phi_f, (A.conj().T @ A) * (B.conj().T @ B),
                               rtol=1e-12, atol=1e-12)
    # one column against a hand-built masked DFT of the rank-one image
    col = (np.fft.fft2(np.outer(A[:, 1], B[:, 1]), norm="ortho")[rows]).reshape(-1)
    np.testing.assert_allclose(Phi[:, 1], col, atol=1e-12)


def test_ridge_cholesky_matches_svd_form_and_normal_equations():
    rng = np.random.default_rng(3)
    Phi = cn(rng, 40, 6)
    Phi[:, 5] = Phi[:, 4] + 1e-3 * Phi[:, 5]       # ill-conditioned on purpose
    y = cn(rng, 40)
    for mu in (1e-2, 1.0, 37.0):
        g = O.ridge_gamma(Phi, y, mu)
        np.testing.assert_allclose(g, O.ridge_gamma_svd(Phi, y, mu), rtol=1e-9, atol=1e-11)
        G, h = O.ridge_gram(Phi, y, mu)
        assert np.linalg.norm(G @ g - h) <= 1e-12 * np.linalg.norm(h) * np.linalg.cond(G)
    # Phi = I: gamma = y / (1 + mu)
    y6 = cn(rng, 6)
    np.testing.assert_allclose(O.ridge_gamma(np.eye(6), y6, 0.5), y6 / 1.5, atol=1e-14)


# ----------------------------------------------------------------------------------
# Gradient (§III-A column gradient, Alg. 3 (S2)): complex finite differences
# ----------------------------------------------------------------------------------

def test_gradients_match_finite_differences():
    rng = np.random.default_rng(4)
    Nx, Ny, R = 5, 4, 2
    A, B, g = cn(rng, Nx, R), cn(rng, Ny, R), cn(rng, R)
    rows = np.array([0, 2, 3])
    Y = O.zero_filled(cn(rng, 3, Ny), rows, Nx)
    mu, rho = 0.3, 0.07
    J = lambda A_, B_: O.objective_J(A_, B_, g, Y, rows, mu, rho)
    gA = O.gradient_A(A, B, g, Y, rows, rho)
    gB = O.gradient_B(A, B, g, Y, rows, rho)
    eps = 1e-6
    for X, grad, which in ((A, gA, "A"), (B, gB, "B")):
        for idx in np.ndindex(X.shape):
            num = 0j
            for unit in (1.0, 1j):
                Xp, Xm = X.copy(), X.copy()
                Xp[idx] += eps * unit
                Xm[idx] -= eps * unit
                fp = J(Xp, B) if which == "A" else J(A, Xp)
                fm = J(Xm, B) if which == "A" else J(A, Xm)
                num += unit * (fp - fm) / (2 * eps)
            assert abs(num - grad[idx]) < 1e-6 * max(1.0, abs(grad[idx])), (which, idx)


def test_lipschitz_bound_majorises_block():
    """f(A + D) <= f(A) + Re<grad, D> + alpha/2 ||D||^2 for the A block (alpha_A bound)."""
    rng = np.random.default_rng(5)
    Nx, Ny, R = 6, 5, 3
    A, B, g = cn(rng, Nx, R), cn(rng, Ny, R), cn(rng, R)
    rows = np.array([1, 2, 5])
    Y = O.zero_filled(cn(rng, 3, Ny), rows, Nx)
    mu, rho = 0.1, 0.05
    f0 = O.objective_J(A, B, g, Y, rows, mu, rho)
    gA = O.gradient_A(A, B, g, Y, rows, rho)
    aA = O.lipschitz_A(B, g, rho)
    for _ in range(50):
        D = cn(rng, Nx, R) * rng.uniform(0.01, 3)
        lhs = O.objective_J(A + D, B, g, Y, rows, mu, rho)
        rhs = f0 + np.vdot(gA, D).real + 0.5 * aA * np.vdot(D, D).real
        assert lhs <= rhs + 1e-9 * abs(rhs)


# ----------------------------------------------------------------------------------
# The tracker: monotone MM, recursion, exact recovery, stationarity (Lemma 2)
# ----------------------------------------------------------------------------------

def test_mm_objective_monotone_per_substep():
    rng = np.random.default_rng(6)
    Nx, Ny, R = 12, 10, 3
    tr = O.Tracker(Nx, Ny, R, 0.9, 1e-2, 4, A=0.3 * cn(rng, Nx, R), B=0.3 * cn(rng, Ny, R))
    for t in range(8):
        mask = np.zeros(Nx, np.uint8)
        mask[rng.choice(Nx, 5, replace=False)] = 1
        Y = O.fft2(cn(rng, Nx, 2) @ cn(rng, 2, Ny))
        tr.push_frame(Y[np.flatnonzero(mask)], mask, record=True)
        vals = [v for _, v in tr.trace]
        assert len(vals) == 1 + 3 * 4
        for a, b in zip(vals, vals[1:]):
            assert b <= a + 1e-12 * abs(a), (t, vals)


@pytest.mark.parametrize("lf", [1.0, 0.9])
def test_recursion_equals_explicit_surrogate_minimiser(lf):
    """With one iteration per frame, A[t] = argmin of the forgotten sum of the
    quadratic surrogates built at A[tau-1] (§III-A), computed here from the stored
    history, equals the recursion."""
    rng = np.random.default_rng(7)
    Nx, Ny, R = 6, 5, 2
    A_init, B_init = 0.5 * cn(rng, Nx, R), 0.5 * cn(rng, Ny, R)
    tr = O.Tracker(Nx, Ny, R, lf, 0.05, 1, A=A_init, B=B_init)
    histA, histB = [], []
    for t in range(15):
        mask = np.zeros(Nx, np.uint8)
        mask[rng.choice(Nx, 3, replace=False)] = 1
        rows = np.flatnonzero(mask)
        Yf = O.fft2(cn(rng, Nx, Ny))
        Y = O.zero_filled(Yf[rows], rows, Nx)
        Aprev, Bprev = tr.A.copy(), tr.B.copy()
        w = lf * tr.w + 1.0
        rho = tr.mu / w
        g = O.ridge_gamma(O.phi_matrix(Aprev, Bprev, rows), Y[rows].reshape(-1), tr.mu)
        aA = O.lipschitz_A(Bprev, g, rho)
        gA = O.gradient_A(Aprev, Bprev, g, Y, rows, rho)
        histA.append((aA, gA, Aprev))
        tr.push_frame(Yf[rows], mask)
        aB = O.lipschitz_B(tr.A, g, rho)
        gB = O.gradient_B(tr.A, Bprev, g, Y, rows, rho)
        histB.append((aB, gB, Bprev))
        for hist, X in ((histA, tr.A), (histB, tr.B)):
            num = sum(lf ** (t - k) * (a * Xp - gr) for k, (a, gr, Xp) in enumerate(hist))
            den = sum(lf ** (t - k) * a for k, (a, _, _) in enumerate(hist))
            np.testing.assert_allclose(X, num / den, rtol=1e-10, atol=1e-12)
        assert abs(tr.abar_A - den_of(histA, lf, t)) <= 1e-10 * tr.abar_A


def den_of(hist, lf, t):
    return sum(lf ** (t - k) * a for k, (a, _, _) in enumerate(hist))


def test_exact_recovery_noiseless_fully_sampled_rank_R():
    rng = np.random.default_rng(5)
    Nx, Ny, R = 8, 6, 2
    As, Bs = cn(rng, Nx, R), cn(rng, Ny, R)
    tr = O.Tracker(Nx, Ny, R, 0.5, 1e-12, 20, A=0.3 * cn(rng, Nx, R), B=0.3 * cn(rng, Ny, R))
    full = np.ones(Nx, np.uint8)
    for t in range(200):
        X = As @ np.diag(cn(rng, R)) @ Bs.T
        x = tr.push_frame(O.fft2(X), full)
    assert O.nrmse(x, X) < 1e-8


def test_stationary_point_has_equal_norm_bases():
    """Lemma 2 analogue: on a repeated frame the iterates approach a stationary point,
    the gradient decays and ||a_r|| = ||b_r||, rho ||a_r||^2 = mu |gamma_r|^2."""
    rng = np.random.default_rng(5)
    Nx, Ny, R = 8, 6, 2
    As, Bs = cn(rng, Nx, R), cn(rng, Ny, R)
    A0, B0 = 0.3 * cn(rng, Nx, R), 0.3 * cn(rng, Ny, R)
    mask = np.zeros(Nx, np.uint8); mask[[0, 1, 3, 6]] = 1
    rows = np.flatnonzero(mask)
    Y = O.fft2(As @ np.diag(cn(rng, R)) @ Bs.T) + 0.01 * cn(rng, Nx, Ny)
    tr = O.Tracker(Nx, Ny, R, 0.3, 1.0, 20, A=A0, B=B0)
    Yz = O.zero_filled(Y[rows], rows, Nx)
    gnorm = []
    for t in range(400):
        tr.push_frame(Y[rows], mask)
        if t in (49, 399):
            rho = tr.mu / tr.w
            gnorm.append(np.linalg.norm(O.gradient_A(tr.A, tr.B, tr.gamma, Yz, rows, rho)))
    assert gnorm[1] < 0.5 * gnorm[0]
    na, nb = np.linalg.norm(tr.A, axis=0), np.linalg.norm(tr.B, axis=0)
    np.testing.assert_allclose(na, nb, rtol=1e-4)
    rho = tr.mu / tr.w
    np.testing.assert_allclose(na, math.sqrt(tr.mu / rho) * np.abs(tr.gamma), rtol=5e-3)


def test_jacobi_form_one_iteration_is_papers_parallel_update():
    """Jacobi, K = 1, lambda_forget = 1: each factor takes the step of Alg. 3 (S2),
    a_r <- (1 - mu_t lambda / t) a_r + mu_t gamma_r^* Theta conj(b_r) with
    mu_t = 1 / abar_t."""
    rng = np.random.default_rng(8)
    Nx, Ny, R = 6, 5, 2
    A, B = cn(rng, Nx, R), cn(rng, Ny, R)
    tr = O.Tracker(Nx, Ny, R, 1.0, 0.2, 1, update="jacobi", A=A, B=B)
    mask = np.array([1, 0, 1, 1, 0, 0], np.uint8)
    rows = np.flatnonzero(mask)
    Yf = O.fft2(cn(rng, Nx, Ny))
    tr.push_frame(Yf[rows], mask)
    g = O.ridge_gamma(O.phi_matrix(A, B, rows), Yf[rows].reshape(-1), 0.2)
    Theta = O.ifft2(O.residual(A, B, g, O.zero_filled(Yf[rows], rows, Nx), rows))
    t, lam = 1, 0.2
    abarA = O.lipschitz_A(B, g, lam / t)
    abarB = O.lipschitz_B(A, g, lam / t)
    for r in range(R):
        a = (1 - lam / t / abarA) * A[:, r] + (1 / abarA) * np.conj(g[r]) * Theta @ np.conj(B[:, r])
        b = (1 - lam / t / abarB) * B[:, r] + (1 / abarB) * np.conj(g[r]) * Theta.T @ np.conj(A[:, r])
        np.testing.assert_allclose(tr.A[:, r], a, atol=1e-12)
        np.testing.assert_allclose(tr.B[:, r], b, atol=1e-12)


# ----------------------------------------------------------------------------------
# Scores and line draws (§V, Alg. 4, §VI-C)
# ----------------------------------------------------------------------------------

def test_scores_sum_to_one_and_uniform_for_impulse_factors():
    rng = np.random.default_rng(9)
    A = cn(rng, 16, 4)
    p = O.informative_line_probs(A, 12)
    assert abs(p.sum() - 1.0) < 1e-14
    assert np.all(p > 0)
    # image-domain impulses have flat k-space rows -> uniform scores
    Ai = np.zeros((16, 4), np.complex128)
    for r in range(4):
        Ai[3 * r, r] = 2.0 + r
    np.testing.assert_allclose(O.informative_line_probs(Ai, 12), np.full(16, 1 / 16), atol=1e-15)
    # a zero column counts as uniform
    Az = A.copy(); Az[:, 2] = 0
    assert abs(O.informative_line_probs(Az, 12).sum() - 1) < 1e-14
    # a column that is one k-space line puts (Ny + R)/(R (Nx + Ny)) + ... on it
    Ak = np.conj(O.dft_matrix(16))[:, [5]]      # F a = e_5
    p1 = O.informative_line_probs(Ak, 12)
    np.testing.assert_allclose(p1[5], (12 * 1 + 1) / (1 * (16 + 12)), rtol=1e-12)
    np.testing.assert_allclose(np.delete(p1, 5), 1 / 28, rtol=1e-10)


def test_vardens_probs_closed_form():
    p = O.vardens_line_probs(8, -1.0)
    d = np.array([1, 1, 2, 3, 4, 3, 2, 1], float)
    np.testing.assert_allclose(p, (1 / d) / np.sum(1 / d), rtol=1e-15)


def test_line_draw_without_replacement_exact_count_and_central():
    rng = np.random.default_rng(10)
    for Nx, k in ((64, 16), (256, 32), (13, 9), (10, 10), (8, 8), (40, 8)):
        p = rng.uniform(0.1, 1, Nx); p /= p.sum()
        m = O.sample_lines_from_probs(p, k, 8, seed=123, ctr=7)
        assert m.sum() == min(k, Nx)
        assert all(m[i] for i in O.central_lines(Nx, 8))


def test_line_draw_fallback_fill_by_weight():
    """When the weights leave too few drawable lines the fill takes the largest q."""
    Nx = 32
    p = np.zeros(Nx); p[10] = 0.5; p[20] = 0.5
    p[15] = 1e-300                                  # q = 0 after quantisation
    m = O.sample_lines_from_probs(p, 13, 8, seed=1, ctr=0)
    assert m.sum() == 13
    assert m[10] and m[20]
    taken = sorted(set(np.flatnonzero(m)) - set(O.central_lines(Nx, 8)) - {10, 20})
    # remaining three lines: all q = 0, lower index first
    assert taken == [4, 5, 6]


def test_line_draw_frequencies_match_expected_count_with_replacement():
    """Monte-Carlo check of E|Omega| = sum_i (1 - (1 - s_i)^K) (§V-B) and of per-line
    inclusion frequencies, sampling with replacement."""
    Nx, K, central = 24, 10, 0
    rng = np.random.default_rng(11)
    p = rng.uniform(0, 1, Nx) ** 3
    p /= p.sum()
    n = 3000
    counts = np.zeros(Nx)
    sizes = []
    for c in range(n):
        m = O.sample_lines_from_probs(p, K, central, seed=99, ctr=c, with_replacement=True)
        counts += m
        sizes.append(m.sum())
    q = np.floor(p * 2.0 ** 52)
    s = q / q.sum()
    expect = O.expected_distinct_lines(s, K)
    sizes = np.array(sizes, float)
    assert abs(sizes.mean() - expect) < 4 * sizes.std() / math.sqrt(n)
    incl = 1 - (1 - s) ** K
    se = np.sqrt(incl * (1 - incl) / n)
    assert np.all(np.abs(counts / n - incl) < 5 * se + 1e-12)


def test_philox_words_uniform():
    """Chi-square of the top byte of Philox words over 20k blocks (not a KAT)."""
    hist = np.zeros(256)
    for i in range(20000):
        w = philox.philox4x32_10((i, 1, 0, 0), (12345, 0))
        for v in w:
            hist[v >> 24] += 1
    e = hist.sum() / 256
    chi2 = np.sum((hist - e) ** 2 / e)
    assert 180 < chi2 < 340          # 255 degrees of freedom
    # counter and key both matter
    assert philox.philox4x32_10((0, 0, 0, 0), (0, 0)) != philox.philox4x32_10((1, 0, 0, 0), (0, 0))
    assert philox.philox4x32_10((0, 0, 0, 0), (0, 0)) != philox.philox4x32_10((0, 0, 0, 0), (1, 0))


def test_mm_step_minimises_its_surrogate():
    """The MM step returns the minimiser of the quadratic surrogate
    s(Z) = <grad, Z - X> + alpha/2 ||Z - X||^2 + lf abar/2 ||Z - X0||^2 (§III-A): its
    gradient vanishes there (checked by central differences of s, not by the closed form),
    and every random perturbation raises s."""
    rng = np.random.default_rng(12)
    X, X0, G = (rng.standard_normal((5, 3)) + 1j * rng.standard_normal((5, 3)) for _ in range(3))
    alpha, abar, lf = 2.5, 7.0, 0.9

    def surrogate(Z):
        return float(np.vdot(G, Z - X).real) + 0.5 * alpha * float(np.vdot(Z - X, Z - X).real) \
            + 0.5 * lf * abar * float(np.vdot(Z - X0, Z - X0).real)

    Z = O.mm_step(X, X0, G, alpha, abar, lf)
    h = 1e-6
    for idx in np.ndindex(Z.shape):
        for unit in (1.0, 1j):
            E = np.zeros_like(Z)
            E[idx] = unit * h
            d = (surrogate(Z + E) - surrogate(Z - E)) / (2 * h)
            assert abs(d) < 1e-6
    for _ in range(20):
        P = 1e-2 * (rng.standard_normal(Z.shape) + 1j * rng.standard_normal(Z.shape))
        assert surrogate(Z + P) > surrogate(Z)


def test_philox_key_schedule_constants_from_their_definition():
    """The Weyl increments of the Philox key schedule are the fractional parts of the
    golden ratio and of sqrt(3) in 32-bit fixed point (SC'11 definition); derived here in
    exact integer arithmetic rather than copied."""
    golden = (math.isqrt(5 << 64) - (1 << 32)) // 2        # floor(2^32 (sqrt 5 - 1) / 2)
    sqrt3 = math.isqrt(3 << 64) - (1 << 32)                # floor(2^32 (sqrt 3 - 1))
    assert philox.W0 == golden and philox.W1 == sqrt3
    # the multipliers are odd, so each round is a bijection of the 128-bit block
    assert philox.M0 % 2 == 1 and philox.M1 % 2 == 1


def test_philox_round_is_invertible():
    """One round inverted from its definition (odd multipliers have inverses mod 2^32):
    c0 and c2 come back from the low product words, then c1 and c3 from the high words
    and the key; a swapped output word or a hi/lo mix-up would break the round trip."""
    inv0, inv1 = pow(philox.M0, -1, 1 << 32), pow(philox.M1, -1, 1 << 32)
    rng = np.random.default_rng(2)
    for _ in range(200):
        c = tuple(int(v) for v in rng.integers(0, 1 << 32, 4, dtype=np.uint64))
        k = tuple(int(v) for v in rng.integers(0, 1 << 32, 2, dtype=np.uint64))
        o = philox.philox4x32_round(c, k)
        c0 = (o[3] * inv0) & philox.MASK32
        c2 = (o[1] * inv1) & philox.MASK32
        c1 = o[0] ^ ((philox.M1 * c2) >> 32) ^ k[0]
        c3 = o[2] ^ ((philox.M0 * c0) >> 32) ^ k[1]
        assert (c0, c1, c2, c3) == c


def test_line_draw_integer_cdf_boundaries():
    """With p_i = k_i 2^-52 the weights are the small integers k_i, so the draws hit
    the CDF boundaries constantly: zero-weight lines are never drawn and line i is
    drawn with probability k_i / sum k."""
    k = np.array([0, 3, 0, 1, 0, 0, 4, 2, 0, 0], float)
    p = k * 2.0 ** -52
    counts = np.zeros(len(k))
    n = 4000
    for c in range(n):
        counts += O.sample_lines_from_probs(p, 1, 0, seed=5, ctr=c, with_replacement=True)
    assert np.all(counts[k == 0] == 0)
    freq = counts / n
    expect = k / k.sum()
    assert np.all(np.abs(freq - expect) < 5 * np.sqrt(expect * (1 - expect) / n) + 1e-12)


@pytest.mark.parametrize("update,K", [("gauss_seidel", 1), ("gauss_seidel", 3), ("jacobi", 2)])
def test_frame_without_lines_is_the_data_free_step(update, K):
    """A frame with no acquired line (S empty) has no data term: Phi has no rows, so the
    ridge gives gamma = 0 and the image is zero. What is left of each block's objective is
    the forgotten past surrogates plus the factor penalty, lf abar / 2 ||X - X[t-1]||^2 +
    rho / 2 ||X||^2, whose minimiser is X[t-1] lf abar / (lf abar + rho): the frame shrinks
    both factors by that ratio at any K, and the surrogate weights grow by rho = mu / w."""
    rng = np.random.default_rng(41)
    Nx, Ny, R, lf, mu = 12, 10, 3, 0.9, 0.05
    A = rng.standard_normal((Nx, R)) + 1j * rng.standard_normal((Nx, R))
    B = rng.standard_normal((Ny, R)) + 1j * rng.standard_normal((Ny, R))
    tr = O.Tracker(Nx, Ny, R, lf, mu, mm_iters=K, update=update, A=A, B=B)
    for t in range(3):
        m = (rng.random(Nx) < 0.5).astype(np.uint8)
        m[0] = 1
        Y = rng.standard_normal((Nx, Ny)) + 1j * rng.standard_normal((Nx, Ny))
        tr.push_frame(Y[np.flatnonzero(m)], m)
    A1, B1, aA, aB, w = tr.A.copy(), tr.B.copy(), tr.abar_A, tr.abar_B, tr.w
    x = tr.push_frame(np.zeros((0, Ny), np.complex128), np.zeros(Nx, np.uint8))
    rho = mu / (lf * w + 1.0)
    assert np.all(x == 0) and np.all(tr.gamma == 0)
    np.testing.assert_allclose(tr.A, A1 * (lf * aA / (lf * aA + rho)), rtol=1e-13, atol=0)
    np.testing.assert_allclose(tr.B, B1 * (lf * aB / (lf * aB + rho)), rtol=1e-13, atol=0)
    assert tr.abar_A == pytest.approx(lf * aA + rho, rel=1e-15)
    assert tr.abar_B == pytest.approx(lf * aB + rho, rel=1e-15)
    assert tr.w == pytest.approx(lf * w + 1.0, rel=1e-15)
