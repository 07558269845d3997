"""Plain FP64 CPU oracle of the mode shapes of the mixed-variational method:
stress coefficients of a Bloch mode and both fields evaluated on a grid.

TEST INFRASTRUCTURE ONLY.  Like `oracle.mixed_variational`, this module is
the slow, obviously correct reference the CUDA path is checked against; only
the test suite, the smoke check and the benchmark's CPU-baseline leg may
import it.

It follows the paper step by step, in float64 / complex128:

  * stress coefficients S = -Phi^-1 H^* U ......... Eq. (equationshomogeneousMatrix),
    second block row (Phi S + H^* U = 0), as stated after Eq. (eigenvalueproblem)
  * u(x) = sum_a U_a f^a(x), sigma(x) = sum_a S_a f^a(x), f^a = exp(i K_a . x)
    ............................................... Eq. (approximation2d), Sec. IV

Readings (also listed with the others in the design notes):
  * H^* is H^dagger and H, Phi are the literal matrices of `OracleCell`
    (the full 3N x 3N Phi, solved by LU; no block-diagonal shortcut);
  * the expansion uses the same f^a as the integrals of `OracleCell` with its
    default conjugation (Omega_ab = int rho conj(f^a) f^b), so u(x) is
    sum_b U_b exp(i K_b . x);
  * grid points are x_pq = ((p + 1/2)/G) h1 + ((q + 1/2)/G) h2, p, q < G,
    the pixel centres when G = P; p indexes h1 (rows), q indexes h2.

Parity status: pinned (tests/test_oracle_modes.py) by Hooke's law on a
homogeneous cell, the first block row of the matrix system (H S + lambda
Omega U = 0) for eigenpairs of the pencil, the energy identity
lambda U^H Omega U = S^H Phi S, the closed form of a single plane wave on the
grid, discrete Parseval and Bloch quasi-periodicity.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .mixed_variational import wavevectors

__all__ = ["stress_coefficients", "grid_points", "plane_wave_sum", "field_on_grid"]


def stress_coefficients(oc, Q, U):
    """S (nvec, 3N) with columns (S11, S22, S12) in the index maps I1, I2, I3
    for displacement coefficients U (nvec, 2N), columns (u1, u2):
    Phi S = -H^dagger U solved with the LU factors of the literal Phi."""
    if oc.paper_conj:
        raise ValueError("mode shapes use the default conjugation of the integrals")
    U = np.atleast_2d(np.asarray(U, complex))
    H = oc.H(np.asarray(Q, float))
    rhs = -(H.conj().T @ U.T)                        # (3N, nvec)
    return sla.lu_solve(oc._lu, rhs).T


def grid_points(cell, G):
    """Cartesian x_pq (G*G, 2), p-major: ((p + 1/2)/G) h1 + ((q + 1/2)/G) h2."""
    f = (np.arange(G) + 0.5) / G
    S, T = np.meshgrid(f, f, indexing="ij")
    h1, h2 = np.asarray(cell.h1, float), np.asarray(cell.h2, float)
    return S.reshape(-1, 1) * h1 + T.reshape(-1, 1) * h2


def plane_wave_sum(cell, M, Q, coef, points):
    """sum_a coef[..., a] exp(i K_a . x) at every point x of `points` (npts, 2)."""
    K = wavevectors(np.asarray(Q, float), cell.h1, cell.h2, M)     # (N, 2)
    phase = np.exp(1j * (np.asarray(points, float) @ K.T))        # (npts, N)
    return np.asarray(coef, complex) @ phase.T


def field_on_grid(cell, M, Q, coef, G):
    """coef (..., N) -> fields (..., G, G) on the grid of `grid_points`."""
    coef = np.asarray(coef, complex)
    out = plane_wave_sum(cell, M, Q, coef.reshape(-1, coef.shape[-1]), grid_points(cell, G))
    return out.reshape(coef.shape[:-1] + (G, G))
