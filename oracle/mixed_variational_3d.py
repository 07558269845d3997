"""Plain FP64 CPU oracle of the mixed-variational band structure of 3-D
voxelated unit cells (the paper's outlook: three displacement and six
stress components, 9 (2M+1)^3 unknowns).

TEST INFRASTRUCTURE ONLY.  Like `oracle.mixed_variational`, this module is
the slow, obviously correct reference the CUDA path is checked against; only
the test suite, the smoke check and the benchmark's CPU-baseline leg may
import it.

It is the 2-D oracle with a third index everywhere, step by step:

  * reciprocal basis q^i = 2 pi (h_j x h_k) / (h_i . (h_j x h_k)) ...... Eq. (1)
  * plane waves f^{abc} = exp(i (k + G_abc) . x), a, b, c in [-M, M],
    alpha-major index (a + M)(2M+1)^2 + (b + M)(2M+1) + (c + M) ....... Eq. (approximation)
  * centroid rule over voxels ........................................ Sec. III
  * isotropic compliance D = (1/2mu) [sym - lam/(3 lam + 2 mu) d d] .. Sec. IV, in 3-D
  * H (3N x 6N), Omega (3N x 3N), Phi (6N x 6N) with the Voigt factors
    2 (and 4) of the shear components ................................. Eqs. (eh), (eo), (ep)
  * A U = lambda Omega U, A = H Phi^-1 H^* ........................... Eq. (eigenvalueproblem)

Stress components in the order 11, 22, 33, 23, 13, 12.  Readings as in 2-D
(integrals with conj(f_a) f_b, H with the trial wave's K, H^* = H^dagger).

Parity status: pinned (tests/test_oracle_3d.py) by the homogeneous closed
form, the three zero modes at Gamma, a cell uniform along x3 reproducing
the pinned 2-D oracle's in-plane bands, translation invariance and scaling.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

__all__ = ["reciprocal_basis3", "plane_wave_indices3", "wavevectors3", "quadrature3",
           "compliance3", "form_factors3", "toeplitz3", "OracleCell3", "STRESS3"]

STRESS3 = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


def reciprocal_basis3(h1, h2, h3):
    h = [np.asarray(v, float) for v in (h1, h2, h3)]
    vol = np.dot(h[0], np.cross(h[1], h[2]))
    return (2 * np.pi * np.cross(h[1], h[2]) / vol, 2 * np.pi * np.cross(h[2], h[0]) / vol,
            2 * np.pi * np.cross(h[0], h[1]) / vol)


def plane_wave_indices3(M):
    r = np.arange(-M, M + 1)
    A, B, C = np.meshgrid(r, r, r, indexing="ij")
    return A.ravel(), B.ravel(), C.ravel()


def wavevectors3(Q, h1, h2, h3, M):
    """K = (Q1 + a) q^1 + (Q2 + b) q^2 + (Q3 + c) q^3, shape (N, 3)."""
    q = reciprocal_basis3(h1, h2, h3)
    a, b, c = plane_wave_indices3(M)
    return (np.outer(Q[0] + a, q[0]) + np.outer(Q[1] + b, q[1]) + np.outer(Q[2] + c, q[2]))


def quadrature3(cell):
    """Voxel centres (P^3, 3) and weights V / P^3, p-major (p along h1)."""
    P = cell.P
    f = (np.arange(P) + 0.5) / P
    S, T, U = np.meshgrid(f, f, f, indexing="ij")
    x = (S.reshape(-1, 1) * cell.h1 + T.reshape(-1, 1) * cell.h2 + U.reshape(-1, 1) * cell.h3)
    V = abs(np.linalg.det(np.array([cell.h1, cell.h2, cell.h3])))
    return x, np.full(P ** 3, V / P ** 3)


def compliance3(lam, mu):
    """Isotropic compliance D_ijkl (..., 3,3,3,3):
    eps = D sigma, D = (1/(2 mu)) [ (d_ik d_jl + d_il d_jk)/2 - lam/(3 lam + 2 mu) d_ij d_kl ]."""
    lam = np.asarray(lam, float)[..., None, None, None, None]
    mu = np.asarray(mu, float)[..., None, None, None, None]
    d = np.eye(3)
    sym = 0.5 * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d))
    vol = np.einsum("ij,kl->ijkl", d, d)
    return (sym - lam / (3.0 * lam + 2.0 * mu) * vol) / (2.0 * mu)


def form_factors3(fields, x, w, q, M):
    """ghat[f, da, db, dc] (indices + 2M) = sum_i g_f(x_i) V_i exp(-i G_d . x_i),
    d in [-2M, 2M]^3, G_d = da q^1 + db q^2 + dc q^3, by direct summation."""
    fields = np.atleast_2d(np.asarray(fields, float))
    D = 4 * M + 1
    d = np.arange(-2 * M, 2 * M + 1)
    gw = fields * w
    xa, xb, xc = x @ q[0], x @ q[1], x @ q[2]
    out = np.empty((fields.shape[0], D, D, D), complex)
    for ia, da in enumerate(d):
        for ib, db in enumerate(d):
            ph = np.exp(-1j * (da * xa[None, :] + db * xb[None, :] + d[:, None] * xc[None, :]))
            out[:, ia, ib, :] = gw @ ph.T
    return out


def toeplitz3(ghat, M):
    a, b, c = plane_wave_indices3(M)
    ia = a[:, None] - a[None, :] + 2 * M
    ib = b[:, None] - b[None, :] + 2 * M
    ic = c[:, None] - c[None, :] + 2 * M
    return ghat[..., ia, ib, ic]


class OracleCell3:
    """k-independent integrals of one 3-D cell, and the per-k pencil."""

    def __init__(self, cell, M):
        if 2 * M + 1 > cell.P:
            raise ValueError("truncation needs 2M+1 <= P")
        self.cell, self.M = cell, M
        self.N = N = (2 * M + 1) ** 3
        self.q = reciprocal_basis3(cell.h1, cell.h2, cell.h3)
        x, w = quadrature3(cell)
        ph = cell.phase.reshape(-1).astype(np.int64)
        rho = cell.rho[ph]
        D = compliance3(cell.lam, cell.mu)[ph]
        fields = [np.ones_like(rho), rho]
        for (j, k) in STRESS3:
            for (m, n) in STRESS3:
                fields.append(D[:, j, k, m, n])
        T = toeplitz3(form_factors3(np.array(fields), x, w, self.q, M), M)
        self.I1 = T[0]
        R = T[1]
        self.Omega = np.zeros((3 * N, 3 * N), complex)
        for l in range(3):
            self.Omega[l * N:(l + 1) * N, l * N:(l + 1) * N] = R
        Phi = np.zeros((6 * N, 6 * N), complex)
        t = 2
        for r, (j, k) in enumerate(STRESS3):
            for c, (m, n) in enumerate(STRESS3):
                fac = (2.0 if j != k else 1.0) * (2.0 if m != n else 1.0)
                Phi[r * N:(r + 1) * N, c * N:(c + 1) * N] = fac * T[t]
                t += 1
        self.Phi = Phi
        self._lu = sla.lu_factor(Phi)

    def H(self, Q):
        """Rows u1, u2, u3; columns the six stress components; entry
        i K_{b,n} int conj(f_a) f_b for the derivative d/dx_n of the trial wave b."""
        N = self.N
        c = self.cell
        K = wavevectors3(np.asarray(Q, float), c.h1, c.h2, c.h3, self.M)
        H = np.zeros((3 * N, 6 * N), complex)
        for row in range(3):
            for col, (m, n) in enumerate(STRESS3):
                coef = np.zeros(N)
                if row == m:
                    coef = coef + K[:, n]
                if row == n and m != n:
                    coef = coef + K[:, m]
                if np.any(coef):
                    H[row * N:(row + 1) * N, col * N:(col + 1) * N] = 1j * self.I1 * coef[None, :]
        return H

    def pencil(self, Q):
        H = self.H(Q)
        A = H @ sla.lu_solve(self._lu, H.conj().T)
        return 0.5 * (A + A.conj().T), self.Omega

    def eigenvalues(self, Q, nbands=None):
        A, Om = self.pencil(Q)
        nb = A.shape[0] if nbands is None else nbands
        return sla.eigh(A, Om, eigvals_only=True, subset_by_index=[0, nb - 1])

    def omega(self, Q, nbands=None):
        return np.sqrt(np.maximum(self.eigenvalues(Q, nbands), 0.0))
