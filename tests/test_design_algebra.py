"""The algebra the CUDA kernels are built on, restated in numpy from the
derivations in their file headers and checked against the oracle's literal
pencil (CPU only).  A wrong step in a derivation (a block of C(k), a factor
V, a stress direction's weight) fails here before any kernel runs."""
import numpy as np
import pytest

from oracle import mixed_variational as mv
from oracle import mixed_variational_3d as mv3
from oracle import mode_shapes as ms
from paper_1310_6380_gb300 import cells

Q2 = [np.array([0.21, -0.13]), np.array([0.5, 0.5])]


def reduced(oc, Q):
    A, Om = oc.pencil(Q)
    Li = np.linalg.inv(np.linalg.cholesky(Om))
    return Li @ A @ Li.conj().T


def gram(cell, M, fields):
    x, w, ph = mv.subdomains(cell)
    return mv.toeplitz(mv.form_factors(np.asarray(fields)[:, ph], x, w, cell.h1, cell.h2, M), M)


def gvec(cell, M):
    a, b = mv.plane_wave_indices(M)
    q1, q2 = mv.reciprocal_basis(cell.h1, cell.h2)
    return np.outer(a, q1) + np.outer(b, q2)          # (N, 2) Cartesian G


@pytest.mark.parametrize("mesh", [False, True])
def test_isotropic_2d_blocks(mesh):
    """Phi = diag(T_k/2, T_m/2, T_m) in the rotated stress basis; W_{X,i}(k) =
    A_R diag(K_i) Z_X, A_R = V L_R^-1 (pixels) or L_R^-1 I1 (mesh); the three
    blocks of C(k) as listed in the header of the dense kernels."""
    cell = cells.mesh_voronoi_cell(12, 5, seed=2) if mesh else cells.voronoi_cell(16, 5, seed=2)
    M = 2
    oc = mv.OracleCell(cell, M)
    Tk, Tm, R, I1 = gram(cell, M, [1 / (cell.lam + cell.mu), 1 / cell.mu, cell.rho,
                                   np.ones_like(cell.mu)])
    V = abs(np.linalg.det(np.array([cell.h1, cell.h2])))
    LRi = np.linalg.inv(np.linalg.cholesky(R))
    AR = LRi @ I1 if mesh else V * LRi
    Z = {X: np.linalg.inv(np.linalg.cholesky(T)).conj().T for X, T in (("k", Tk), ("m", Tm))}
    G = gvec(cell, M)
    for Q in Q2:
        q1, q2 = mv.reciprocal_basis(cell.h1, cell.h2)
        K = G + Q[0] * q1 + Q[1] * q2
        Wf = {(X, i): AR @ np.diag(K[:, i]) @ Z[X] for X in Z for i in (0, 1)}
        W = lambda X, i: Wf[(X, i)]
        C11 = W("k", 0) @ W("k", 0).conj().T + W("m", 0) @ W("m", 0).conj().T \
            + W("m", 1) @ W("m", 1).conj().T
        C22 = W("k", 1) @ W("k", 1).conj().T + W("m", 1) @ W("m", 1).conj().T \
            + W("m", 0) @ W("m", 0).conj().T
        C12 = W("k", 0) @ W("k", 1).conj().T - W("m", 0) @ W("m", 1).conj().T \
            + W("m", 1) @ W("m", 0).conj().T
        C = np.block([[C11, C12], [C12.conj().T, C22]])
        ref = reduced(oc, Q)
        assert np.abs(C - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("mesh", [False, True])
def test_anisotropic_2d_w_form(mesh):
    """Phi = [T[S_rc]] factored whole, W_i = L_Omega^-1 H_i L_Phi^-dagger and
    C(k) = W W^dagger with W = k1 W1 + k2 W2 + W0 (the header of the
    anisotropic kernels); A_R = L_R^-1 I1 on a mesh."""
    base = (cells.mesh_voronoi_cell(12, 4, seed=6, lattice="hex") if mesh
            else cells.voronoi_cell(16, 4, seed=6, lattice="hex"))
    cell = cells.anisotropic_cell(base, seed=2)
    M = 2
    oc = mv.OracleCell(cell, M)
    S = np.linalg.inv(cell.stiffness)
    T = gram(cell, M, [S[:, 0, 0], S[:, 1, 1], cell.rho, S[:, 0, 1], S[:, 0, 2], S[:, 1, 2],
                       S[:, 2, 2], np.ones_like(cell.rho)])
    f = {(0, 0): 0, (1, 1): 1, (2, 2): 6, (0, 1): 3, (0, 2): 4, (1, 2): 5}
    Phi = np.block([[T[f[(min(r, c), max(r, c))]] for c in range(3)] for r in range(3)])
    Z = np.linalg.inv(np.linalg.cholesky(Phi)).conj().T
    N = oc.N
    V = abs(np.linalg.det(np.array([cell.h1, cell.h2])))
    LRi = np.linalg.inv(np.linalg.cholesky(T[2]))
    AR = LRi @ T[7] if mesh else V * LRi
    Zr = [Z[r * N:(r + 1) * N] for r in range(3)]
    G = gvec(cell, M)
    W1 = np.vstack([AR @ Zr[0], AR @ Zr[2]])
    W2 = np.vstack([AR @ Zr[2], AR @ Zr[1]])
    W0 = np.vstack([AR @ (G[:, :1] * Zr[0] + G[:, 1:] * Zr[2]),
                    AR @ (G[:, 1:] * Zr[1] + G[:, :1] * Zr[2])])
    q1, q2 = mv.reciprocal_basis(cell.h1, cell.h2)
    for Q in Q2:
        k = Q[0] * q1 + Q[1] * q2
        W = k[0] * W1 + k[1] * W2 + W0
        ref = reduced(oc, Q)
        assert np.abs(W @ W.conj().T - ref).max() <= 1e-12 * np.abs(ref).max()


def test_isotropic_2d_stress_formula():
    """S11 = iV [T_k^-1 (K1 u1 + K2 u2) + T_m^-1 (K1 u1 - K2 u2)], S22 with the
    sign flipped, S12 = iV T_m^-1 (K2 u1 + K1 u2) (header of the mode kernels)."""
    cell = cells.config0()["cell"]
    M = 2
    oc = mv.OracleCell(cell, M)
    Tk, Tm = gram(cell, M, [1 / (cell.lam + cell.mu), 1 / cell.mu])
    V = abs(np.linalg.det(np.array([cell.h1, cell.h2])))
    rng = np.random.default_rng(0)
    U = rng.standard_normal((3, 2 * oc.N)) + 1j * rng.standard_normal((3, 2 * oc.N))
    Q = Q2[0]
    K = mv.wavevectors(Q, cell.h1, cell.h2, M)
    u1, u2 = U[:, :oc.N].T, U[:, oc.N:].T
    a = np.linalg.solve(Tk, K[:, :1] * u1 + K[:, 1:] * u2)
    b = np.linalg.solve(Tm, K[:, :1] * u1 - K[:, 1:] * u2)
    c = np.linalg.solve(Tm, K[:, 1:] * u1 + K[:, :1] * u2)
    S = 1j * V * np.vstack([a + b, a - b, c]).T
    ref = ms.stress_coefficients(oc, Q, U)
    assert np.abs(S - ref).max() <= 1e-11 * np.abs(ref).max()


def test_3d_stress_directions_and_monomials():
    """3-D: Phi split into the hydrostatic (weight 1, T[1/(3 lam + 2 mu)]), two
    deviatoric (weight 2, T[1/mu]) and three shear (weight 1, T[1/mu])
    directions; C(k) = V^2 sum_c s_c (A h_c Z_X)(A h_c Z_X)^dagger, and the
    ten monomial coefficients built from the products F^a F^b^dagger."""
    cell = cells.voronoi_cell3(6, 4, seed=2)
    M = 1
    oc = mv3.OracleCell3(cell, M)
    N = oc.N
    x, w = mv3.quadrature3(cell)
    ph = cell.phase.reshape(-1).astype(int)
    q = mv3.reciprocal_basis3(cell.h1, cell.h2, cell.h3)
    T = mv3.toeplitz3(mv3.form_factors3(np.array([1 / (3 * cell.lam + 2 * cell.mu), 1 / cell.mu,
                                                  cell.rho])[:, ph], x, w, q, M), M)
    LRi = np.linalg.inv(np.linalg.cholesky(T[2]))
    Z = [np.linalg.inv(np.linalg.cholesky(T[X])).conj().T for X in (0, 1)]
    a_, b_, c_ = mv3.plane_wave_indices3(M)
    G = np.array([a_ * q[0][j] + b_ * q[1][j] + c_ * q[2][j] for j in range(3)])
    F = [[LRi @ np.diag(s) @ Z[X] for s in (np.ones(N), G[0], G[1], G[2])] for X in (0, 1)]
    comp = mv3.STRESS3
    r3, r2, r6 = 1 / np.sqrt(3), 1 / np.sqrt(2), 1 / np.sqrt(6)
    v = np.array([[r3, r3, r3, 0, 0, 0], [r2, -r2, 0, 0, 0, 0], [r6, r6, -2 * r6, 0, 0, 0],
                  [0, 0, 0, 1, 0, 0], [0, 0, 0, 0, 1, 0], [0, 0, 0, 0, 0, 1]])
    sc, Xof = [1, 2, 2, 1, 1, 1], [0, 1, 1, 1, 1, 1]
    alpha = np.zeros((6, 3, 3))
    for c in range(6):
        for qq, (m, n) in enumerate(comp):
            for l in range(3):
                if l == m:
                    alpha[c, l, n] += v[c, qq]
                if l == n and m != n:
                    alpha[c, l, m] += v[c, qq]
    coef = np.zeros((10, 3, 3, 2, 4, 4))
    quad = [[4, 7, 8], [7, 5, 9], [8, 9, 6]]
    for c in range(6):
        for l in range(3):
            for lp in range(3):
                for j in range(3):
                    for jp in range(3):
                        wgt = sc[c] * alpha[c, l, j] * alpha[c, lp, jp]
                        X = Xof[c]
                        coef[0, l, lp, X, j + 1, jp + 1] += wgt
                        coef[1 + j, l, lp, X, 0, jp + 1] += wgt
                        coef[1 + jp, l, lp, X, j + 1, 0] += wgt
                        coef[quad[j][jp], l, lp, X, 0, 0] += wgt
    P = [[[F[X][a] @ F[X][b].conj().T for b in range(4)] for a in range(4)] for X in (0, 1)]
    V = abs(np.linalg.det(np.array([cell.h1, cell.h2, cell.h3])))
    Cm = np.zeros((10, 3 * N, 3 * N), complex)
    for t in range(10):
        for l in range(3):
            for lp in range(3):
                Cm[t, l * N:(l + 1) * N, lp * N:(lp + 1) * N] = V * V * sum(
                    coef[t, l, lp, X, a, b] * P[X][a][b]
                    for X in (0, 1) for a in range(4) for b in range(4))
    for Q in (np.array([0.21, 0.07, -0.13]), np.array([0.5, 0.5, 0.5])):
        k = Q[0] * q[0] + Q[1] * q[1] + Q[2] * q[2]
        cf = [1, k[0], k[1], k[2], k[0] ** 2, k[1] ** 2, k[2] ** 2, k[0] * k[1], k[0] * k[2],
              k[1] * k[2]]
        C = sum(cf[t] * Cm[t] for t in range(10))
        ref = reduced(oc, Q)
        assert np.abs(C - ref).max() <= 1e-12 * np.abs(ref).max()
