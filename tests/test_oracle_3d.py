"""Pins of the 3-D oracle (voxel cells, three displacement and six stress
components): the homogeneous closed form, three zero modes at Gamma, a cell
uniform along x3 reproducing the 2-D oracle's in-plane bands, translation
invariance, scaling, and a planted shear factor that the pins catch."""
import numpy as np
import pytest

from oracle import mixed_variational as mv
from oracle import mixed_variational_3d as mv3
from paper_1310_6380_gb300 import cells

LAM, MU, RHO = 4.0, 1.5, 1.2


def homogeneous3(P=6, h=None):
    h1, h2, h3 = h if h is not None else (np.eye(3)[0], np.eye(3)[1], np.eye(3)[2])
    return cells.Cell3(h1, h2, h3, np.zeros((P, P, P), np.uint16), np.array([LAM]),
                       np.array([MU]), np.array([RHO]))


@pytest.mark.parametrize("shear", [False, True])
def test_homogeneous_closed_form(shear):
    h = None
    if shear:
        h = (np.array([1.0, 0.0, 0.0]), np.array([0.3, 0.9, 0.0]), np.array([0.2, -0.1, 1.1]))
    cell = homogeneous3(6, h)
    M = 1
    oc = mv3.OracleCell3(cell, M)
    for Q in ([0.21, 0.07, -0.13], [0.5, 0.5, 0.5]):
        Q = np.array(Q)
        lam = oc.eigenvalues(Q)
        K = np.linalg.norm(mv3.wavevectors3(Q, cell.h1, cell.h2, cell.h3, M), axis=1) ** 2
        ref = np.sort(np.concatenate([(LAM + 2 * MU) / RHO * K, MU / RHO * K, MU / RHO * K]))
        assert np.abs(lam - ref).max() <= 1e-11 * ref.max(), Q


def test_three_zero_modes_at_gamma():
    cell = cells.sphere_cell3(6, 0.3)
    lam = mv3.OracleCell3(cell, 1).eigenvalues(np.zeros(3))
    assert np.abs(lam[:3]).max() <= 1e-10 * lam.max()
    assert lam[3] > 1e-3 * lam.max()


def test_extruded_cell_contains_the_2d_bands():
    """A cell uniform along x3 at k3 = 0: the plane waves with gamma = 0 and
    u3 = 0 decouple, and the s33 rows of Phi S + H^* U = 0 enforce e33 = 0.
    When every phase has the same Poisson ratio (lam = 2 mu here) the
    Toeplitz blocks of D3311 and D3333 are proportional, so eliminating s33
    gives exactly the Toeplitz blocks of the plane-strain compliance: every
    in-plane eigenvalue of the (pinned) 2-D oracle is one of the 3-D pencil."""
    base = cells.voronoi_cell(6, 3, seed=4)
    c2 = base.with_props(lam=2.0 * base.mu)
    c3 = cells.extruded_cell3(c2)
    M = 1
    Q2 = np.array([0.31, 0.12])
    lam2 = mv.OracleCell(c2, M).eigenvalues(Q2)
    lam3 = mv3.OracleCell3(c3, M).eigenvalues(np.array([Q2[0], Q2[1], 0.0]))
    gap = np.array([np.abs(lam3 - v).min() for v in lam2])
    assert gap.max() <= 1e-9 * lam2.max(), gap.max()


def test_translation_and_scaling():
    cell = cells.voronoi_cell3(6, 4, seed=2)
    M = 1
    Q = np.array([0.2, -0.1, 0.3])
    a = mv3.OracleCell3(cell, M).omega(Q, 8)
    shifted = cells.Cell3(cell.h1, cell.h2, cell.h3, np.roll(cell.phase, (1, 2, 3), (0, 1, 2)),
                          cell.lam, cell.mu, cell.rho)
    b = mv3.OracleCell3(shifted, M).omega(Q, 8)
    assert np.abs(a - b).max() <= 1e-11 * a.max()
    heavy = cells.Cell3(cell.h1, cell.h2, cell.h3, cell.phase, cell.lam, cell.mu, 4 * cell.rho)
    c = mv3.OracleCell3(heavy, M).omega(Q, 8)
    assert np.allclose(c, a / 2, rtol=1e-12, atol=1e-12 * a.max())


def test_planted_shear_factor_fails(monkeypatch):
    """Dropping the Voigt factor 2 of the shear stresses in Phi breaks the
    homogeneous pin."""
    cell = homogeneous3(6)
    M = 1
    Q = np.array([0.21, 0.07, -0.13])
    K = np.linalg.norm(mv3.wavevectors3(Q, cell.h1, cell.h2, cell.h3, M), axis=1) ** 2
    ref = np.sort(np.concatenate([(LAM + 2 * MU) / RHO * K, MU / RHO * K, MU / RHO * K]))
    real = mv3.compliance3

    def halved_shear(lam, mu):
        D = real(lam, mu)
        for (i, j) in [(0, 1), (1, 0), (0, 2), (2, 0), (1, 2), (2, 1)]:
            D[..., i, j, i, j] *= 0.5
            D[..., i, j, j, i] *= 0.5
        return D

    monkeypatch.setattr(mv3, "compliance3", halved_shear)
    lam = mv3.OracleCell3(cell, M).eigenvalues(Q)
    assert np.abs(lam - ref).max() > 1e-2 * ref.max()
