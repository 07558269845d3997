"""Pins of the oracle with a general in-plane stiffness per phase (the full
D_jkmn of Eq. (ep)): the isotropic special case, the Christoffel closed form
of a homogeneous anisotropic cell, rotation covariance, and a planted Voigt
factor that the pins catch."""
import numpy as np
import pytest

from oracle import mixed_variational as mv
from paper_1310_6380_gb300 import cells

Q = np.array([0.23, 0.11])


def test_isotropic_stiffness_gives_isotropic_compliance():
    lam, mu = np.array([4.0, 110.0, 2.5]), np.array([1.5, 80.0, 7.0])
    D1 = mv.compliance_from_stiffness(cells.isotropic_stiffness(lam, mu))
    D2 = mv.compliance(lam, mu)
    assert np.abs(D1 - D2).max() <= 1e-15 * np.abs(D2).max() * 10


def test_isotropic_stiffness_gives_isotropic_bands():
    cell = cells.config0()["cell"]
    iso = cells.with_stiffness(cell, cells.isotropic_stiffness(cell.lam, cell.mu))
    a = mv.OracleCell(cell, 3).omega(Q, 8)
    b = mv.OracleCell(iso, 3).omega(Q, 8)
    assert np.abs(a - b).max() <= 1e-13 * a.max()


def christoffel_bands(C, rho, K, nb):
    """rho omega^2 = eigenvalues of Gamma(K) = N(K)^T C N(K), N = [[K1, 0], [0, K2], [K2, K1]]
    (strain (e11, e22, 2 e12) of a plane wave u e^{i K.x}), for every plane wave K."""
    w = []
    for k1, k2 in K:
        Nk = np.array([[k1, 0.0], [0.0, k2], [k2, k1]])
        w.extend(np.linalg.eigvalsh(Nk.T @ C @ Nk) / rho)
    return np.sqrt(np.maximum(np.sort(w), 0.0))[:nb]


@pytest.mark.parametrize("lattice", ["square", "hex"])
def test_homogeneous_anisotropic_is_christoffel(lattice):
    M, nb = 3, 12
    C = cells.rotated_orthotropic(120.0, 40.0, 25.0, 18.0, 0.61)
    base = cells.homogeneous_cell(16, 4.0, 1.5, 1.3, lattice=lattice)
    cell = cells.with_stiffness(base, C[None])
    oc = mv.OracleCell(cell, M)
    for q in ([0.23, 0.11], [0.5, 0.0], [0.31, -0.4]):
        q = np.array(q)
        K = mv.wavevectors(q, cell.h1, cell.h2, M)
        ref = christoffel_bands(C, 1.3, K, nb)
        got = oc.omega(q, nb)
        assert np.abs(got - ref).max() <= 1e-12 * ref.max(), q


@pytest.mark.parametrize("sign", [1, -1])
def test_rotation_covariance(sign):
    """Turning the pixel map, every phase's stiffness and the wavevector by
    +-90 degrees on a square lattice leaves the bands unchanged."""
    base = cells.voronoi_cell(16, 5, seed=3)
    a = cells.anisotropic_cell(base, seed=1)
    P = base.P
    p, q = np.meshgrid(np.arange(P), np.arange(P), indexing="ij")
    th = sign * np.pi / 2
    newph = base.phase[q, P - 1 - p] if sign == 1 else base.phase[P - 1 - q, p]
    rotated = cells.Cell(base.h1, base.h2, newph.astype(np.uint16), base.lam, base.mu, base.rho)
    b = cells.with_stiffness(rotated, np.array([cells.rotate_stiffness(C, th)
                                                for C in a.stiffness]))
    Qr = np.array([-Q[1], Q[0]]) if sign == 1 else np.array([Q[1], -Q[0]])
    w1 = mv.OracleCell(a, 2).omega(Q, 8)
    w2 = mv.OracleCell(b, 2).omega(Qr, 8)
    assert np.abs(w1 - w2).max() <= 1e-12 * w1.max()


def test_anisotropic_pencil_structure():
    cell = cells.anisotropic_cell(cells.voronoi_cell(16, 4, seed=2, lattice="hex"), seed=4)
    oc = mv.OracleCell(cell, 2)
    assert np.abs(oc.Phi - oc.Phi.conj().T).max() <= 1e-14 * np.abs(oc.Phi).max()
    assert np.linalg.eigvalsh(oc.Phi).min() > 0
    A, Om = oc.pencil(Q)
    assert np.linalg.eigvalsh(A).min() >= -1e-10 * np.abs(A).max()


def test_planted_voigt_factor_fails_christoffel(monkeypatch):
    """D12_12 = S33 instead of S33 / 4 (a plausible Voigt slip) breaks the pin."""
    C = cells.rotated_orthotropic(120.0, 40.0, 25.0, 18.0, 0.61)
    cell = cells.with_stiffness(cells.homogeneous_cell(16, 4.0, 1.5, 1.3), C[None])
    M = 2
    K = mv.wavevectors(Q, cell.h1, cell.h2, M)
    ref = christoffel_bands(C, 1.3, K, 8)
    good = mv.compliance_from_stiffness

    def bad(Cs):
        D = good(Cs)
        S33 = np.linalg.inv(Cs)[..., 2, 2]
        for (j, k, m, n) in [(0, 1, 0, 1), (1, 0, 0, 1), (0, 1, 1, 0), (1, 0, 1, 0)]:
            D[..., j, k, m, n] = S33
        return D

    monkeypatch.setattr(mv, "compliance_from_stiffness", bad)
    got = mv.OracleCell(cell, M).omega(Q, 8)
    assert np.abs(got - ref).max() > 1e-2 * ref.max()
