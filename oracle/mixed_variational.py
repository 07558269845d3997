"""Plain FP64 CPU oracle of the mixed-variational phononic band structure.

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously correct
reference that the CUDA path is checked against.  Only the test suite,
the smoke check and the benchmark's CPU-baseline leg may import it; the
product path (the C-ABI library and its Python binding) never does.

It follows the paper (Srivastava, "Fast phononic band-structure
calculations through a GPU accelerated mixed-variational formulation")
step by step, in the paper's notation, in float64 / complex128:

  * reciprocal basis q^i ............................ Eq. (1)
  * Bloch wavevector k = Q_i q^i .................... Sec. II
  * plane waves f^{ab} = exp(i (k + G_ab) . x) ...... Eq. (approximation), Eq. (approximation2d)
  * index maps I1, I2, I3 (alpha-major) ............. Sec. IV.A
  * H, Omega, Phi entries ........................... Eqs. (eh), (eo), (ep)
  * isotropic plane-strain compliance D_jkmn ........ Sec. IV, constitutive law
    (or the compliance of a general in-plane stiffness per phase)
  * centroid quadrature over subdomains ............. Sec. III (int F = sum F_i V_i),
    pixels of a phase map or the elements of a mesh (centroid, area, phase)
  * eigenproblem A U = lambda Omega U, A = H Phi^-1 H^*,
    omega = sqrt(lambda) ............................ Eq. (eigenvalueproblem)

Readings of points the paper leaves open:
  * subdomain = pixel, centroid = pixel centre, weight V / P^2;
  * H is 2N x 3N (rows u1, u2; columns S11, S22, S12) and H^* = H^dagger;
  * H uses the wavevector of the trial (column) plane wave;
  * integrals use f_a^* f_b (conjugate of the paper's f; `paper_conj=True`
    switches to the paper's sign, which gives the conjugate pencil and the
    same eigenvalues);
  * the pencil is solved as A U = lambda Omega U (identical to the
    inverted form for lambda != 0 and well posed at Gamma).

Parity status: pinned (tests/test_oracle_*.py) by closed forms
(homogeneous dispersion, Rytov bilayer, Dirichlet-kernel form factors),
invariants and the paper's own stop bands.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

__all__ = [
    "reciprocal_basis", "plane_wave_indices", "wavevectors", "quadrature", "subdomains",
    "compliance", "compliance_from_stiffness", "form_factors", "toeplitz", "integrals_literal", "OracleCell",
    "bands",
]


# ---------------------------------------------------------------- geometry
def reciprocal_basis(h1, h2):
    """q^1, q^2 of Eq. (1) for a 2-D cell, with h^3 = e^3."""
    H1 = np.array([h1[0], h1[1], 0.0])
    H2 = np.array([h2[0], h2[1], 0.0])
    H3 = np.array([0.0, 0.0, 1.0])
    q1 = 2 * np.pi * np.cross(H2, H3) / np.dot(H1, np.cross(H2, H3))
    q2 = 2 * np.pi * np.cross(H3, H1) / np.dot(H2, np.cross(H3, H1))
    return q1[:2], q2[:2]


def plane_wave_indices(M):
    """(alpha, beta) for every plane wave, in the order of the index map
    I1 = (alpha + M)(2M + 1) + (beta + M) (0-based form of Sec. IV.A)."""
    r = np.arange(-M, M + 1)
    alpha = np.repeat(r, 2 * M + 1)
    beta = np.tile(r, 2 * M + 1)
    return alpha, beta


def wavevectors(Q, h1, h2, M):
    """K_ab = (Q1 + alpha) q^1 + (Q2 + beta) q^2, shape (N, 2)."""
    q1, q2 = reciprocal_basis(h1, h2)
    alpha, beta = plane_wave_indices(M)
    return np.outer(Q[0] + alpha, q1) + np.outer(Q[1] + beta, q2)


def quadrature(cell):
    """Centroids x_i (P*P, 2) and weights V_i (P*P,) of the pixel subdomains
    (Sec. III: int F dOmega = sum_i F_i V_i).  Pixel (p, q) has centroid
    ((p + 1/2)/P) h1 + ((q + 1/2)/P) h2 and area |det[h1; h2]| / P^2."""
    P = cell.P
    f = (np.arange(P) + 0.5) / P
    H1, H2 = np.meshgrid(f, f, indexing="ij")
    x = H1.reshape(-1, 1) * cell.h1 + H2.reshape(-1, 1) * cell.h2
    V = abs(np.linalg.det(np.array([cell.h1, cell.h2])))
    return x, np.full(P * P, V / (P * P))


def subdomains(cell):
    """Centroids x_i (nel, 2), areas V_i and phase index of every subdomain
    (Sec. III): the pixels of a pixel cell, or the elements of a mesh cell
    (centroid given in fractional coordinates, x = s h1 + t h2)."""
    if hasattr(cell, "centroid"):
        c = np.asarray(cell.centroid, float)
        x = c[:, :1] * np.asarray(cell.h1, float) + c[:, 1:] * np.asarray(cell.h2, float)
        return x, np.asarray(cell.area, float), np.asarray(cell.phase).astype(np.int64)
    x, w = quadrature(cell)
    return x, w, cell.phase.reshape(-1).astype(np.int64)


def compliance(lam, mu):
    """Isotropic plane-strain compliance D_jkmn (Sec. IV), shape (..., 2,2,2,2):
    D = 1/(2 mu) [ (d_jm d_kn + d_jn d_km)/2 - lam/(2(mu + lam)) d_jk d_mn ]."""
    lam = np.asarray(lam, float)[..., None, None, None, None]
    mu = np.asarray(mu, float)[..., None, None, None, None]
    d = np.eye(2)
    sym = 0.5 * (np.einsum("jm,kn->jkmn", d, d) + np.einsum("jn,km->jkmn", d, d))
    vol = np.einsum("jk,mn->jkmn", d, d)
    return (sym - lam / (2.0 * (mu + lam)) * vol) / (2.0 * mu)


def compliance_from_stiffness(C):
    """D_jkmn (..., 2,2,2,2) of in-plane Voigt stiffness C (..., 3, 3)
    (sigma = C (e11, e22, 2 e12)): with S = C^-1, D1111 = S11, D2222 = S22,
    D1122 = S12, D11_12 = S13 / 2, D22_12 = S23 / 2, D12_12 = S33 / 4 and the
    minor and major symmetries of the compliance tensor (Sec. IV, the general
    constitutive law behind Eq. (ep))."""
    S = np.linalg.inv(np.asarray(C, float))
    D = np.zeros(S.shape[:-2] + (2, 2, 2, 2))
    pairs = [(0, 0), (1, 1), (0, 1)]
    fac = [1.0, 1.0, 0.5]
    for a, (j, k) in enumerate(pairs):
        for b, (m, n) in enumerate(pairs):
            v = S[..., a, b] * fac[a] * fac[b]
            for (jj, kk) in {(j, k), (k, j)}:
                for (mm, nn) in {(m, n), (n, m)}:
                    D[..., jj, kk, mm, nn] = v
    return D


# ---------------------------------------------------------------- integrals
def form_factors(fields, x, w, h1, h2, M, paper_conj=False):
    """ghat[f, da + 2M, db + 2M] = sum_i g_f(x_i) V_i exp(-i G_d . x_i) for
    every difference d = (da, db) in [-2M, 2M]^2, G_d = da q^1 + db q^2.

    This is the centroid rule applied to int g f_a^* f_b dOmega, whose
    integrand depends on the plane-wave pair only through a - b (the k
    part cancels, Sec. IV.A).  paper_conj=True uses exp(+i G_d . x)."""
    fields = np.atleast_2d(np.asarray(fields, float))
    q1, q2 = reciprocal_basis(h1, h2)
    D = 4 * M + 1
    d = np.arange(-2 * M, 2 * M + 1)
    sgn = 1.0 if paper_conj else -1.0
    gw = fields * w                       # (nf, npix)
    out = np.empty((fields.shape[0], D, D), complex)
    xb = x @ q2                           # (npix,)
    xa = x @ q1
    for ia, da in enumerate(d):
        ph = np.exp(sgn * 1j * (da * xa[None, :] + d[:, None] * xb[None, :]))  # (D, npix)
        out[:, ia, :] = gw @ ph.T
    return out


def toeplitz(ghat, M):
    """Expand difference-indexed form factors to the plane-wave matrix
    T[a, b] = ghat[alpha_a - alpha_b, beta_a - beta_b] (Sec. IV.A)."""
    alpha, beta = plane_wave_indices(M)
    ia = alpha[:, None] - alpha[None, :] + 2 * M
    ib = beta[:, None] - beta[None, :] + 2 * M
    return ghat[..., ia, ib]


def integrals_literal(cell, M, Q, g=None):
    """The paper's own GPU formulation of one integral (Sec. V, Eq. (eExp)):
    [f]_ijk = exp([A1(j) - B1(k)] c(i,1) + [A2(j) - B2(k)] c(i,2)),
    I_jk = sum_i g_i [f]_ijk A_i, with A1, A2, B1, B2 built from T = A^-1
    as in that section.  Returns the N x N matrix I (paper sign convention).
    Only for tiny cells: the tensor [f] has N_el * N^2 entries.  The
    elements are the cell's subdomains: pixels, or the elements of a mesh
    (the paper's own case, centroids c(i, :) and areas A_i)."""
    x, w, _ = subdomains(cell)
    if g is None:
        g = np.ones(len(w))
    A = np.array([cell.h1, cell.h2])
    T = np.linalg.inv(A)
    alpha, beta = plane_wave_indices(M)
    A1 = 2j * np.pi * (T[0, 0] * (Q[0] + alpha) + T[0, 1] * (Q[1] + beta))
    A2 = 2j * np.pi * (T[1, 0] * (Q[0] + alpha) + T[1, 1] * (Q[1] + beta))
    B1, B2 = A1, A2                        # theta, eta run over the same set
    f = np.exp((A1[None, :, None] - B1[None, None, :]) * x[:, 0, None, None]
               + (A2[None, :, None] - B2[None, None, :]) * x[:, 1, None, None])
    return np.einsum("ijk,i->jk", f, g * w)


# ---------------------------------------------------------------- matrices
_COMP = [(0, 0), (1, 1), (0, 1)]   # stress components S11, S22, S12 (I1, I2, I3)


class OracleCell:
    """k-independent integrals of one cell, and the per-k pencil."""

    def __init__(self, cell, M, paper_conj=False):
        if not hasattr(cell, "centroid") and 2 * M + 1 > cell.P:
            raise ValueError("truncation needs 2M+1 <= P")
        self.cell, self.M, self.paper_conj = cell, M, paper_conj
        N = (2 * M + 1) ** 2
        self.N = N
        x, w, ph = subdomains(cell)
        rho = cell.rho[ph]
        if getattr(cell, "stiffness", None) is not None:
            D = compliance_from_stiffness(cell.stiffness)[ph]
        else:
            D = compliance(cell.lam, cell.mu)[ph]      # (npix, 2,2,2,2)
        fields = [np.ones_like(rho), rho]
        for (j, k) in _COMP:
            for (m, n) in _COMP:
                fields.append(D[:, j, k, m, n])
        gh = form_factors(np.array(fields), x, w, cell.h1, cell.h2, M, paper_conj)
        self.ghat = gh
        T = toeplitz(gh, M)                             # (nf, N, N)
        self.I1 = T[0]                                  # int f_a^* f_b
        R = T[1]                                        # int rho f_a^* f_b
        self.Omega = np.zeros((2 * N, 2 * N), complex)  # Eq. (eo)
        self.Omega[:N, :N] = R
        self.Omega[N:, N:] = R
        Phi = np.zeros((3 * N, 3 * N), complex)         # Eq. (ep)
        t = 2
        for r, (j, k) in enumerate(_COMP):
            for c, (m, n) in enumerate(_COMP):
                fac = (2.0 if r == 2 else 1.0) * (2.0 if c == 2 else 1.0)
                Phi[r * N:(r + 1) * N, c * N:(c + 1) * N] = fac * T[t]
                t += 1
        self.Phi = Phi
        self._lu = sla.lu_factor(Phi)

    def H(self, Q):
        """Eq. (eh): rows (u1, u2), columns (S11, S22, S12); entry
        i K_{b,l} int f_a^* f_b with b the column plane wave."""
        N = self.N
        K = wavevectors(Q, self.cell.h1, self.cell.h2, self.M)
        H = np.zeros((2 * N, 3 * N), complex)
        for row in range(2):
            for c, (m, n) in enumerate(_COMP):
                coef = np.zeros(N)
                if row == m:
                    coef = coef + K[:, n]
                if row == n and m != n:
                    coef = coef + K[:, m]
                if np.any(coef):
                    H[row * N:(row + 1) * N, c * N:(c + 1) * N] = 1j * self.I1 * coef[None, :]
        return H

    def pencil(self, Q):
        """A = H Phi^-1 H^dagger (Hermitian part) and Omega, Eq. (eigenvalueproblem)."""
        H = self.H(Q)
        Y = sla.lu_solve(self._lu, H.conj().T)
        A = H @ Y
        return 0.5 * (A + A.conj().T), self.Omega

    def eigenvalues(self, Q, nbands=None):
        """Lowest `nbands` lambda = omega^2 of A U = lambda Omega U."""
        A, Om = self.pencil(Q)
        n = A.shape[0]
        nb = n if nbands is None else nbands
        return sla.eigh(A, Om, eigvals_only=True, subset_by_index=[0, nb - 1])

    def omega(self, Q, nbands=None):
        lam = self.eigenvalues(Q, nbands)
        return np.sqrt(np.maximum(lam, 0.0))


def bands(cell, M, Qs, nbands, return_lambda=False):
    """omega (nk, nbands) for every fractional wavevector in Qs."""
    oc = OracleCell(cell, M)
    lam = np.array([oc.eigenvalues(np.asarray(Q, float), nbands) for Q in Qs])
    return lam if return_lambda else np.sqrt(np.maximum(lam, 0.0))
