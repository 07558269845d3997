"""Pins of the mode-shape oracle (stress coefficients, fields on a grid)
against what the paper and elasticity fix independently of its formulas."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import mixed_variational as mv
from oracle import mode_shapes as ms
from paper_1310_6380_gb300 import cells

LAM, MU, RHO = 4.0, 1.5, 1.2


def test_homogeneous_stress_is_hookes_law():
    """On a homogeneous cell, S of any U is sigma = lam tr(eps) I + 2 mu eps
    with eps = sym(i K (x) u), plane wave by plane wave (Sec. IV constitutive law)."""
    cell = cells.homogeneous_cell(16, LAM, MU, RHO)
    M = 2
    oc = mv.OracleCell(cell, M)
    N = oc.N
    Q = np.array([0.23, 0.11])
    rng = np.random.default_rng(1)
    U = rng.standard_normal((3, 2 * N)) + 1j * rng.standard_normal((3, 2 * N))
    S = ms.stress_coefficients(oc, Q, U)
    alpha, beta = mv.plane_wave_indices(M)
    q1, q2 = mv.reciprocal_basis(cell.h1, cell.h2)
    K1 = (Q[0] + alpha) * q1[0] + (Q[1] + beta) * q2[0]
    K2 = (Q[0] + alpha) * q1[1] + (Q[1] + beta) * q2[1]
    u1, u2 = U[:, :N], U[:, N:]
    e11, e22, e12 = 1j * K1 * u1, 1j * K2 * u2, 0.5j * (K2 * u1 + K1 * u2)
    s11 = LAM * (e11 + e22) + 2 * MU * e11
    s22 = LAM * (e11 + e22) + 2 * MU * e22
    s12 = 2 * MU * e12
    ref = np.concatenate([s11, s22, s12], axis=1)
    assert np.abs(S - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("mk, M, Q", [
    (lambda: cells.config0()["cell"], 3, (0.21, 0.07)),
    (lambda: cells.voronoi_cell(24, 6, seed=5, lattice="hex"), 3, (0.4, 0.13)),
])
def test_first_block_row_holds_for_eigenpairs(mk, M, Q):
    """S from the second block row of the matrix system also satisfies the
    first one, H S + lambda Omega U = 0, for eigenpairs of the pencil; and the
    energy identity lambda U^H Omega U = S^H Phi S."""
    cell = mk()
    oc = mv.OracleCell(cell, M)
    Q = np.array(Q)
    A, Om = oc.pencil(Q)
    lam, V = sla.eigh(A, Om, subset_by_index=[0, 7])
    U = V.T
    S = ms.stress_coefficients(oc, Q, U)
    H = oc.H(Q)
    for i in range(len(lam)):
        r = H @ S[i] + lam[i] * (Om @ U[i])
        assert np.linalg.norm(r) <= 1e-9 * lam[i] * np.linalg.norm(Om @ U[i]), i
        kin = lam[i] * np.real(U[i].conj() @ Om @ U[i])
        pot = np.real(S[i].conj() @ oc.Phi @ S[i])
        assert abs(kin - pot) <= 1e-9 * kin, i


def test_single_plane_wave_on_grid():
    """A unit coefficient at (alpha, beta) is exp(2 pi i ((Q1 + alpha) s + (Q2 + beta) t))
    at the fractional grid coordinates s = (p + 1/2)/G, t = (q + 1/2)/G."""
    cell = cells.voronoi_cell(16, 4, seed=2, lattice="hex")
    M, G = 2, 9
    Q = np.array([0.31, -0.17])
    alpha, beta = mv.plane_wave_indices(M)
    coef = np.eye(len(alpha))
    F = ms.field_on_grid(cell, M, Q, coef, G)
    s = (np.arange(G) + 0.5) / G
    for a in (0, 7, 12, 24):
        ref = np.exp(2j * np.pi * ((Q[0] + alpha[a]) * s[:, None] + (Q[1] + beta[a]) * s[None, :]))
        assert np.abs(F[a] - ref).max() <= 1e-12, a


@pytest.mark.parametrize("G", [5, 7, 12])
def test_parseval_on_the_grid(G):
    """The plane waves |alpha|, |beta| <= M are orthogonal on a G x G grid with
    G >= 2M + 1, so the grid mean of |field|^2 equals sum |coef|^2."""
    cell = cells.config0()["cell"]
    M = 2
    rng = np.random.default_rng(G)
    c = rng.standard_normal((2, 25)) + 1j * rng.standard_normal((2, 25))
    F = ms.field_on_grid(cell, M, np.array([0.4, 0.1]), c, G)
    assert np.allclose(np.mean(np.abs(F) ** 2, axis=(1, 2)), np.sum(np.abs(c) ** 2, axis=1),
                       rtol=1e-12)


def test_bloch_quasi_periodicity():
    """u(x + h1) = exp(2 pi i Q1) u(x), u(x + h2) = exp(2 pi i Q2) u(x)."""
    cell = cells.voronoi_cell(16, 4, seed=9, lattice="hex")
    M = 3
    Q = np.array([0.27, 0.42])
    rng = np.random.default_rng(3)
    c = rng.standard_normal(49) + 1j * rng.standard_normal(49)
    x = ms.grid_points(cell, 6)
    f0 = ms.plane_wave_sum(cell, M, Q, c, x)
    f1 = ms.plane_wave_sum(cell, M, Q, c, x + np.asarray(cell.h1))
    f2 = ms.plane_wave_sum(cell, M, Q, c, x + np.asarray(cell.h2))
    assert np.allclose(f1, np.exp(2j * np.pi * Q[0]) * f0, atol=1e-11)
    assert np.allclose(f2, np.exp(2j * np.pi * Q[1]) * f0, atol=1e-11)


def test_planted_mistakes_fail_the_pins():
    """A flipped sign or swapped stress column in the oracle breaks the pins."""
    cell = cells.config0()["cell"]
    M = 2
    oc = mv.OracleCell(cell, M)
    Q = np.array([0.21, 0.07])
    A, Om = oc.pencil(Q)
    lam, V = sla.eigh(A, Om, subset_by_index=[3, 3])
    U = V.T
    S = ms.stress_coefficients(oc, Q, U)
    H = oc.H(Q)
    good = np.linalg.norm(H @ S[0] + lam[0] * (Om @ U[0]))
    flipped = np.linalg.norm(H @ (-S[0]) + lam[0] * (Om @ U[0]))
    N = oc.N
    sw = S[0].copy()
    sw[:N], sw[N:2 * N] = S[0][N:2 * N], S[0][:N]
    swapped = np.linalg.norm(H @ sw + lam[0] * (Om @ U[0]))
    scale = lam[0] * np.linalg.norm(Om @ U[0])
    assert good <= 1e-9 * scale
    assert flipped > 0.5 * scale and swapped > 1e-3 * scale
