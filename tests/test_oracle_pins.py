"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these tests re-types the oracle's formulas: each compares it with
an independent fact (a closed form, an invariant, a textbook routine, a
number the paper prints) chosen so that a plausible slip in the oracle (a
dropped term, a wrong sign or index, a transposed operand, a missing
Voigt factor) fails at least one of them.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla
from scipy.optimize import brentq

from oracle import mixed_variational as mv
from paper_1310_6380_gb300 import cells

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------ lattice
@pytest.mark.parametrize("lattice", ["square", "hex"])
def test_reciprocal_basis_duality(lattice):
    """q^i . h^j = 2 pi delta_ij (Eq. (1))."""
    h1, h2 = cells.square(1.7) if lattice == "square" else cells.hexagonal(0.9)
    q1, q2 = mv.reciprocal_basis(h1, h2)
    G = np.array([[q1 @ h1, q1 @ h2], [q2 @ h1, q2 @ h2]])
    assert np.allclose(G, 2 * np.pi * np.eye(2), atol=1e-13)


def test_hex_high_symmetry_points():
    """|k| at M and K of the hexagonal zone: 2 pi/(sqrt3 a) and 4 pi/(3 a)."""
    a = 1.3
    h1, h2 = cells.hexagonal(a)
    Qs = cells.ibz_path("hex", 4, h1, h2)       # G, M, K, G is not uniform; use corners
    KM = mv.wavevectors(np.array([0.5, 0.0]), h1, h2, 0)[0]
    KK = mv.wavevectors(np.array([2 / 3, 1 / 3]), h1, h2, 0)[0]
    assert np.isclose(np.linalg.norm(KM), 2 * np.pi / (np.sqrt(3) * a), rtol=1e-14)
    assert np.isclose(np.linalg.norm(KK), 4 * np.pi / (3 * a), rtol=1e-14)
    assert np.allclose(Qs[0], 0) and np.allclose(Qs[-1], 0)


def test_plane_wave_index_map():
    """I1 = (alpha+M)(2M+1) + (beta+M): alpha-major order (Sec. IV.A)."""
    M = 2
    al, be = mv.plane_wave_indices(M)
    for a in range(-M, M + 1):
        for b in range(-M, M + 1):
            i = (a + M) * (2 * M + 1) + (b + M)
            assert al[i] == a and be[i] == b


# ------------------------------------------------------------ compliance
def test_compliance_inverts_plane_strain_stiffness():
    """D_jkmn C_mnpq = symmetric identity, with C = lam d d + mu (d d + d d)."""
    lam, mu = 3.7, 1.9
    D = mv.compliance(lam, mu)
    d = np.eye(2)
    C = (lam * np.einsum("jk,mn->jkmn", d, d)
         + mu * (np.einsum("jm,kn->jkmn", d, d) + np.einsum("jn,km->jkmn", d, d)))
    I = 0.5 * (np.einsum("jp,kq->jkpq", d, d) + np.einsum("jq,kp->jkpq", d, d))
    assert np.allclose(np.einsum("jkmn,mnpq->jkpq", D, C), I, atol=1e-14)
    # the isotropic values of the plane-strain compliance
    assert np.isclose(D[0, 0, 0, 0], (lam + 2 * mu) / (4 * mu * (lam + mu)))
    assert np.isclose(D[0, 0, 1, 1], -lam / (4 * mu * (lam + mu)))
    assert np.isclose(D[0, 1, 0, 1], 1 / (4 * mu))
    assert D[0, 0, 0, 1] == 0 and D[1, 1, 0, 1] == 0


# ------------------------------------------------------------ form factors
def _ff(cell, field, M, conj=False):
    x, w = mv.quadrature(cell)
    return mv.form_factors(field.reshape(1, -1), x, w, cell.h1, cell.h2, M, conj)[0]


@pytest.mark.parametrize("lattice", ["square", "hex"])
def test_form_factor_mean_and_constant(lattice):
    cell = cells.circle_cell(16, 0.3, lattice=lattice)
    V = abs(np.linalg.det(np.array([cell.h1, cell.h2])))
    g = cell.rho[cell.phase.reshape(-1)]
    M = 3
    gh = _ff(cell, g, M)
    assert np.isclose(gh[2 * M, 2 * M], g.sum() * V / cell.P ** 2, rtol=1e-14)
    gc = _ff(cell, np.full(cell.P ** 2, 2.5), M)
    ref = np.zeros_like(gc)
    ref[2 * M, 2 * M] = 2.5 * V
    assert np.abs(gc - ref).max() < 1e-13 * 2.5 * V


@pytest.mark.parametrize("lattice", ["square", "hex"])
def test_form_factor_rectangle_closed_form(lattice):
    """Indicator of a pixel-aligned block: a product of two geometric series
    (Dirichlet kernels) in exp(-2 pi i d (p+1/2)/P), since G_d . x_p =
    2 pi (da H1 + db H2) for any lattice."""
    P, M = 16, 3
    cell = cells.homogeneous_cell(P, lattice=lattice)
    V = abs(np.linalg.det(np.array([cell.h1, cell.h2])))
    p0, p1, q0, q1 = 3, 11, 5, 8
    g = np.zeros((P, P))
    g[p0:p1, q0:q1] = 1.0
    gh = _ff(cell, g.reshape(-1), M)

    def geo(d, s0, s1):
        z = np.exp(-2j * np.pi * d / P)
        if d % P == 0:
            return complex(s1 - s0) * np.exp(-1j * np.pi * d / P)
        return z ** (s0 + 0.5) * (1 - z ** (s1 - s0)) / (1 - z)

    for da in range(-2 * M, 2 * M + 1):
        for db in range(-2 * M, 2 * M + 1):
            ref = V / P ** 2 * geo(da, p0, p1) * geo(db, q0, q1)
            assert abs(gh[da + 2 * M, db + 2 * M] - ref) < 1e-14 * V


def test_form_factor_hermitian_and_shift():
    P, M = 16, 3
    cell = cells.voronoi_cell(P, 7, seed=5)
    g = cell.mu[cell.phase.reshape(-1)]
    gh = _ff(cell, g, M)
    assert np.allclose(gh[::-1, ::-1], gh.conj(), atol=1e-14 * np.abs(gh).max())
    s1, s2 = 5, 9
    gs = _ff(cell.shifted(s1, s2), cell.mu[cell.shifted(s1, s2).phase.reshape(-1)], M)
    d = np.arange(-2 * M, 2 * M + 1)
    phase = np.exp(-2j * np.pi * (d[:, None] * s1 + d[None, :] * s2) / P)
    assert np.allclose(gs, gh * phase, atol=1e-13 * np.abs(gh).max())


@pytest.mark.parametrize("lattice", ["square", "hex"])
def test_literal_paper_integrals_match(lattice):
    """The paper's own integrand tensor (Eq. (eExp), built from T = A^-1 as
    in Sec. V) summed over elements equals the difference form factors
    expanded to plane-wave pairs (conjugate sign, reading of f)."""
    cell = cells.voronoi_cell(8, 5, seed=2, lattice=lattice)
    M = 2
    Q = np.array([0.31, -0.17])
    rho = cell.rho[cell.phase.reshape(-1)]
    lit = mv.integrals_literal(cell, M, Q, rho)
    T = mv.toeplitz(_ff(cell, rho, M), M)
    assert np.allclose(lit, T.conj(), atol=1e-14 * np.abs(T).max())
    T2 = mv.toeplitz(_ff(cell, rho, M, conj=True), M)
    assert np.allclose(lit, T2, atol=1e-14 * np.abs(T).max())


# ------------------------------------------------------------ eigenvalues
@pytest.mark.parametrize("lattice", ["square", "hex"])
@pytest.mark.parametrize("Q", [(0.2, 0.1), (0.5, 0.0), (0.0, 0.0), (0.37, 0.41)])
def test_homogeneous_full_spectrum(lattice, Q):
    """A homogeneous cell folds the free dispersion: the whole spectrum is
    {c_L^2 |K|^2, c_T^2 |K|^2} over all plane waves K = k + G."""
    lam, mu, rho = 4.0, 1.5, 1.2
    cell = cells.homogeneous_cell(8, lam, mu, rho, lattice=lattice, a=1.3)
    M = 2
    Q = np.array(Q)
    got = mv.OracleCell(cell, M).eigenvalues(Q)
    K = mv.wavevectors(Q, cell.h1, cell.h2, M)
    k2 = np.sum(K ** 2, axis=1)
    ref = np.sort(np.concatenate([(lam + 2 * mu) / rho * k2, mu / rho * k2]))
    scale = ref.max()
    assert np.abs(got - ref).max() < 1e-12 * scale


def test_gamma_two_zero_modes():
    cfg = cells.config0()
    lam = mv.OracleCell(cfg["cell"], cfg["M"]).eigenvalues(np.zeros(2), 4)
    assert abs(lam[0]) < 1e-10 * lam[2] and abs(lam[1]) < 1e-10 * lam[2]
    assert lam[2] > 1.0


def test_translation_invariance():
    cell = cells.voronoi_cell(24, 6, seed=11)
    Q = np.array([0.21, 0.33])
    a = mv.OracleCell(cell, 3).eigenvalues(Q, 12)
    b = mv.OracleCell(cell.shifted(5, 9), 3).eigenvalues(Q, 12)
    assert np.allclose(a, b, rtol=1e-11, atol=1e-12 * a.max())


def test_time_reversal():
    cell = cells.voronoi_cell(16, 5, seed=3, lattice="hex")
    Q = np.array([0.27, 0.13])
    oc = mv.OracleCell(cell, 3)
    assert np.allclose(oc.eigenvalues(Q, 10), oc.eigenvalues(-Q, 10), rtol=1e-11)


def test_scaling_laws():
    cell = cells.voronoi_cell(16, 5, seed=4)
    M, Q = 2, np.array([0.3, 0.2])
    w0 = mv.OracleCell(cell, M).omega(Q, 8)
    s = 2.7
    w1 = mv.OracleCell(cell.with_props(lam=s * cell.lam, mu=s * cell.mu), M).omega(Q, 8)
    w2 = mv.OracleCell(cell.with_props(rho=s * cell.rho), M).omega(Q, 8)
    w3 = mv.OracleCell(cell.with_props(h_scale=s), M).omega(Q, 8)
    assert np.allclose(w1, np.sqrt(s) * w0, rtol=1e-11)
    assert np.allclose(w2, w0 / np.sqrt(s), rtol=1e-11)
    assert np.allclose(w3, w0 / s, rtol=1e-11)


def test_pencil_structure():
    cell = cells.voronoi_cell(16, 6, seed=8, lattice="hex")
    oc = mv.OracleCell(cell, 3)
    N = oc.N
    A, Om = oc.pencil(np.array([0.4, 0.1]))
    H = oc.H(np.array([0.4, 0.1]))
    assert np.allclose(Om, Om.conj().T, atol=0)
    assert np.allclose(oc.Phi, oc.Phi.conj().T, atol=1e-15 * np.abs(oc.Phi).max())
    sla.cholesky(Om, lower=True)           # Omega positive definite
    ev = np.linalg.eigvalsh(A)
    assert ev.min() > -1e-12 * ev.max()     # A positive semidefinite
    V = abs(np.linalg.det(np.array([cell.h1, cell.h2])))
    off = oc.I1 - np.diag(np.diag(oc.I1))
    assert np.abs(off).max() < 1e-13 * V and np.allclose(np.diag(oc.I1), V, rtol=1e-14)
    # isotropy: D_1112 = D_2212 = 0, so these blocks of Phi vanish
    assert np.abs(oc.Phi[:N, 2 * N:]).max() == 0 and np.abs(oc.Phi[N:2 * N, 2 * N:]).max() == 0
    assert H.shape == (2 * N, 3 * N)


def test_paper_conjugation_gives_same_eigenvalues():
    cell = cells.voronoi_cell(16, 6, seed=9)
    Q = np.array([0.12, 0.4])
    a = mv.OracleCell(cell, 3).eigenvalues(Q, 10)
    b = mv.OracleCell(cell, 3, paper_conj=True).eigenvalues(Q, 10)
    assert np.allclose(a, b, rtol=1e-11)


def test_truncation_limit():
    with pytest.raises(ValueError):
        mv.OracleCell(cells.circle_cell(8), 4)   # 2M+1 = 9 > P = 8


# ------------------------------------------------------------ 1-D closed form
def _rytov_roots(k, d1, d2, c1, c2, Z1, Z2, wmax, nroots):
    """Roots in omega of the bilayer dispersion relation
    cos k(d1+d2) = cos(w d1/c1) cos(w d2/c2) - (Z1/Z2 + Z2/Z1)/2 sin(w d1/c1) sin(w d2/c2)."""
    def f(w):
        return (np.cos(w * d1 / c1) * np.cos(w * d2 / c2)
                - 0.5 * (Z1 / Z2 + Z2 / Z1) * np.sin(w * d1 / c1) * np.sin(w * d2 / c2)
                - np.cos(k * (d1 + d2)))
    ws = np.linspace(1e-9, wmax, 200001)
    fs = f(ws)
    out = []
    for i in np.nonzero(np.sign(fs[:-1]) != np.sign(fs[1:]))[0]:
        out.append(brentq(f, ws[i], ws[i + 1], xtol=1e-15, rtol=1e-15))
        if len(out) == nroots:
            break
    return np.array(out)


def test_rytov_bilayer():
    """A cell uniform in x2 with k along x1: the beta = 0 plane waves form an
    exactly decoupled block whose eigenvalues converge, as M grows, to the
    roots of the closed-form P and SV bilayer dispersion relations."""
    l1, l2 = (4.0, 1.5, 1.2), (110.0, 80.0, 7.8)
    P = 64
    cell = cells.bilayer_cell(P, P // 2, l1, l2)
    Q = np.array([0.3, 0.0])
    k = 0.3 * 2 * np.pi
    cL = [np.sqrt((m[0] + 2 * m[1]) / m[2]) for m in (l1, l2)]
    cT = [np.sqrt(m[1] / m[2]) for m in (l1, l2)]
    rP = _rytov_roots(k, 0.5, 0.5, cL[0], cL[1], l1[2] * cL[0], l2[2] * cL[1], 60, 4)
    rS = _rytov_roots(k, 0.5, 0.5, cT[0], cT[1], l1[2] * cT[0], l2[2] * cT[1], 60, 4)
    ref = np.sort(np.concatenate([rP, rS]))[:4]
    errs = {}
    for M in (2, 4, 8, 12):
        oc = mv.OracleCell(cell, M)
        A, Om = oc.pencil(Q)
        _, be = mv.plane_wave_indices(M)
        idx = np.nonzero(be == 0)[0]
        sel = np.concatenate([idx, oc.N + idx])
        rest = np.setdiff1d(np.arange(2 * oc.N), sel)
        assert np.abs(A[np.ix_(sel, rest)]).max() < 1e-13 * np.abs(A).max()
        lam = sla.eigh(A[np.ix_(sel, sel)], Om[np.ix_(sel, sel)], eigvals_only=True)[:4]
        errs[M] = np.abs(np.sqrt(lam) - ref) / ref
    assert errs[2].max() > 3 * errs[8].max()
    assert errs[8].max() < 1.5e-3
    assert errs[12].max() < 3e-4


# ------------------------------------------------------------ the paper's numbers
def test_golden_hex_steel_epoxy_stop_bands():
    """The paper's worked example: stop bands at 120-262 kHz and 427-473 kHz
    (first 12 branches, M = 5).  Pixel quadrature stands in for the paper's
    964-triangle mesh, so the edges agree to about 1 %."""
    ref = np.loadtxt(os.path.join(GOLDEN, "hex_steel_epoxy_stop_bands.txt"))
    cell = cells.steel_epoxy_hex_cell(48)
    Qs = cells.ibz_path("hex", 46, cell.h1, cell.h2)
    f = mv.bands(cell, 5, Qs, 12) / (2 * np.pi) / 1e3
    gaps = []
    for i in range(11):
        lo, hi = f[:, i].max(), f[:, i + 1].min()
        if hi - lo > 10.0:                  # ignore sub-10 kHz sampling artefacts
            gaps.append((lo, hi))
    gaps = np.array(gaps)
    assert gaps.shape == ref.shape
    assert np.allclose(gaps, ref, rtol=0.015)


def test_convergence_envelope():
    """The lowest four branches approach the M = 12 solution as M grows
    (the envelope shrinks; step-by-step monotonicity is not required)."""
    cfg = cells.config0()
    Q = np.array([0.25, 0.0])
    ref = mv.OracleCell(cfg["cell"], 12).omega(Q, 4)
    err = [np.abs(mv.OracleCell(cfg["cell"], M).omega(Q, 4) - ref).max() / ref.max()
           for M in (1, 2, 4, 8)]
    assert err[0] > err[1] > err[2] > err[3]
    assert err[3] < err[1] / 2
