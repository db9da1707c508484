"""FP64-grade ridge step (S1 of Alg. 3, the closed form of §III-A) on the frame path.

The frame kernel forms the normal equations (Phi^H Phi + mu I) gamma = Phi^H y from its FP32
operands (the acquired rows of the transformed factor, Ahat_S, the factor B and the
transformed rows Yt) with every sum accumulated in float-float, and refines an FP32
Gauss-Jordan solution against that system. gamma_t therefore equals the FP64 solution of the
normal equations of those operands to about kappa(G) u_float-float. The tests bound it at
1e-10 relative for kappa(G) <= 1e4, with no allowance for kappa:

- k-space factors (Alg. 2): the operands are the inputs themselves (a row selection and the
  untransformed rows), so gamma is compared with the oracle's ridge solve from (A1, A2, y);
- a 4 x 4 image grid with small-integer factors and data, whose DFT entries are +-1/2, +-i/2
  (exact in FP32 up to the 1e-17 residue of cos(pi/2) in the twiddle table) so that every
  FP32 sum of the transforms is exact: compared with the oracle's ridge solve from (A, B, y)
  through its literal 2D DFTs;
- cine-size image grids: compared with the FP64 solve of the normal equations built from the
  frame's own FP32 operands (read back by the test hook tts_get_ridge_operands), and with the
  oracle's solve from (A, B, y) at the bound the FP32 transforms leave (kappa x 1e-6)."""
import numpy as np
import pytest

from oracle import kspace as KS
from oracle import tracker as O

pytestmark = pytest.mark.gpu

TOL = 1e-10
KAPPA_MAX = 1e4


def cn(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)


def factors_with_condition(rng, Nx, Ny, R, rows, mu, phi_fn, target):
    """CN factors in FP32 with two nearly parallel columns: along a geometric sweep of their
    closeness, the last one whose kappa(Phi^H Phi + mu I) (host FP64) is not above `target`."""
    A0 = cn(rng, Nx, R).astype(np.complex64)
    B0 = cn(rng, Ny, R).astype(np.complex64)
    dA, dB = cn(rng, Nx), cn(rng, Ny)
    best = None
    for eps in np.geomspace(1.0, 1e-4, 41):
        A, B = A0.copy(), B0.copy()
        if R > 1:
            A[:, 1] = (A0[:, 0] + eps * dA).astype(np.complex64)
            B[:, 1] = (B0[:, 0] + eps * dB).astype(np.complex64)
        Phi = phi_fn(A.astype(np.complex128), B.astype(np.complex128), rows)
        G = Phi.conj().T @ Phi + mu * np.eye(R)
        k = np.linalg.cond(G)
        if best is None or k <= target:
            best = (A, B, k)
        if k > target:
            break
    return best


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("Nx,Ny,R,nlines,target", [(64, 64, 8, 16, 1e2), (64, 48, 16, 12, 1e4),
                                                   (128, 96, 32, 24, 1e3), (96, 128, 32, 40, 1e4),
                                                   (40, 30, 5, 40, 1e4)])
@pytest.mark.parametrize("prec", [0, 1])
def test_kspace_gamma_matches_oracle_ridge(tts, Nx, Ny, R, nlines, target, prec):
    """Alg. 2 frame (one MM iteration): gamma_t from the frame kernel against the oracle's
    Cholesky solve of (Phi^H Phi + mu I) gamma = Phi^H y, Phi of Alg. 2 (S1) from the same
    A1, A2, y; <= 1e-10 relative at kappa <= 1e4."""
    rng = np.random.default_rng(Nx * 1000 + Ny + R)
    mu = 1e-2
    rows = np.sort(rng.choice(Nx, size=nlines, replace=False))
    mask = np.zeros(Nx, np.uint8)
    mask[rows] = 1
    A1, A2, kappa = factors_with_condition(rng, Nx, Ny, R, rows, mu, KS.ks_phi, target)
    assert kappa <= KAPPA_MAX
    y = (A1[rows] @ np.diag(cn(rng, R)) @ A2.T + 0.05 * cn(rng, nlines, Ny)).astype(np.complex64)
    trk = tts.Tracker(Nx, Ny, R, 0.95, mu, mm_iters=1, kspace=1, ridge_precision=prec)
    trk.set_factors(A1, A2)
    trk.push_frame(y, mask)
    g = trk.gamma_fp64()
    ref = O.ridge_gamma(KS.ks_phi(A1.astype(np.complex128), A2.astype(np.complex128), rows),
                        y.astype(np.complex128).reshape(-1), mu)
    assert rel(g, ref) <= TOL, (rel(g, ref), kappa)
    trk.close()


@pytest.mark.parametrize("R,lines", [(1, [0]), (2, [0, 2]), (3, [0, 1, 3]), (4, [0, 1, 2, 3])])
def test_exact_dft_grid_gamma_matches_oracle_ridge(tts, R, lines):
    """4 x 4 image grid with small-integer factors and data: every DFT entry is +-1/2 or
    +-i/2 (up to the 1e-17 residue of cos(pi/2) in the twiddle table) and every FP32 sum of the
    transforms is exact, so the image-domain frame path's operands carry no rounding. Its
    gamma_t against the oracle's ridge solve through its literal masked 2D DFTs of the rank-one
    images (Alg. 3 (S1)) from the same A, B, y; <= 1e-10 at kappa <= 1e4."""
    rng = np.random.default_rng(40 + R)
    N, mu = 4, 1e-2
    rows = np.array(lines)
    mask = np.zeros(N, np.uint8)
    mask[rows] = 1
    ints = lambda *shape: (rng.integers(-3, 4, shape) + 1j * rng.integers(-3, 4, shape)).astype(np.complex64)
    A, B = ints(N, R), ints(N, R)
    y = ints(len(rows), N)
    Phi = O.phi_matrix(A.astype(np.complex128), B.astype(np.complex128), rows)
    G = Phi.conj().T @ Phi + mu * np.eye(R)
    kappa = np.linalg.cond(G)
    assert kappa <= KAPPA_MAX
    trk = tts.Tracker(N, N, R, 0.95, mu, mm_iters=1, central_lines=0)
    trk.set_factors(A, B)
    trk.push_frame(y, mask)
    g = trk.gamma_fp64()
    ref = O.ridge_gamma(Phi, y.astype(np.complex128).reshape(-1), mu)
    assert rel(g, ref) <= TOL, (rel(g, ref), kappa)
    trk.close()


@pytest.mark.parametrize("Nx,Ny,R,nlines,target", [(256, 256, 32, 32, 1e2), (256, 256, 32, 32, 1e4),
                                                   (64, 64, 8, 16, 1e4), (192, 160, 24, 30, 1e3),
                                                   (128, 128, 48, 64, 1e3), (256, 256, 32, 256, 1e3)])
@pytest.mark.parametrize("prec", [0, 1])
def test_image_gamma_is_the_fp64_solution_of_its_operands(tts, Nx, Ny, R, nlines, target, prec):
    """Image-domain frame (one MM iteration) at cine sizes, including a fully sampled frame:
    gamma_t equals the FP64 Cholesky solution of the normal equations built in FP64 from the
    frame's own FP32 operands (Ahat_S, Yt and B[t-1]) to <= 1e-10 at kappa <= 1e4; against the
    oracle's solve from (A, B, y) it agrees to the FP32 transforms' error, <= kappa x 1e-6."""
    rng = np.random.default_rng(Nx + 7 * Ny + R + nlines)
    mu = 1e-2
    central = O.central_lines(Nx, 8)
    rest = np.setdiff1d(np.arange(Nx), central)
    rows = np.sort(np.concatenate([central, rng.choice(rest, size=nlines - len(central), replace=False)]))
    mask = np.zeros(Nx, np.uint8)
    mask[rows] = 1
    sep = lambda A, B, r: KS.ks_phi(np.fft.fft(A, axis=0, norm="ortho"), np.fft.fft(B, axis=0, norm="ortho"), r)
    A, B, kappa = factors_with_condition(rng, Nx, Ny, R, rows, mu, sep, target)
    assert kappa <= KAPPA_MAX
    y = (O.fft2(A @ np.diag(cn(rng, R)) @ B.T)[rows] + 0.05 * cn(rng, len(rows), Ny)).astype(np.complex64)
    trk = tts.Tracker(Nx, Ny, R, 0.95, mu, mm_iters=1, ridge_precision=prec)
    trk.set_factors(A, B)
    trk.push_frame(y, mask)
    g = trk.gamma_fp64()
    Ah, Yt, got_rows = trk.ridge_operands()
    assert np.array_equal(got_rows, rows)
    Ah, Yt = Ah.astype(np.complex128), Yt.astype(np.complex128)
    Bd = B.astype(np.complex128)
    G = (Ah.conj().T @ Ah) * (Bd.conj().T @ Bd) + mu * np.eye(R)
    h = np.sum(Ah.conj() * (Yt @ Bd.conj()), axis=0)
    k_ops = np.linalg.cond(G)
    assert k_ops <= KAPPA_MAX
    assert rel(g, O.cholesky_solve(G, h)) <= TOL, (rel(g, O.cholesky_solve(G, h)), k_ops)
    ref = O.ridge_gamma(O.phi_matrix(A.astype(np.complex128), Bd, rows), y.astype(np.complex128).reshape(-1), mu)
    assert rel(g, ref) <= kappa * 1e-6, (rel(g, ref), kappa)
    trk.close()
