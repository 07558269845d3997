"""Pins of the oracle on mesh cells (centroid quadrature over triangles,
Sec. III): the pixel mesh reduces to the pinned pixel path, translation
invariance, the homogeneous closed form approached as the mesh refines, the
density scaling law, and a planted centroid error that the pins catch."""
import os

import numpy as np
import pytest

from oracle import mixed_variational as mv
from paper_1310_6380_gb300 import cells

Q = np.array([0.23, 0.11])
LAM, MU, RHO = 4.0, 1.5, 1.2


def homogeneous_error(mesh, M, nb=10):
    w = mv.OracleCell(mesh, M).omega(Q, nb)
    K = mv.wavevectors(Q, mesh.h1, mesh.h2, M)
    kn = np.linalg.norm(K, axis=1)
    ref = np.sort(np.concatenate([np.sqrt((LAM + 2 * MU) / RHO) * kn, np.sqrt(MU / RHO) * kn]))
    return np.abs(w - ref[:nb]).max() / ref[nb - 1]


def test_mesh_generator_tiles_the_cell():
    for lat in ("square", "hex"):
        m = cells.mesh_voronoi_cell(12, 7, seed=2, lattice=lat)
        V = abs(np.linalg.det(np.array([m.h1, m.h2])))
        assert m.nel == 2 * 12 * 12
        assert abs(m.area.sum() - V) <= 1e-14 * V
        assert (m.area > 0).all()


@pytest.mark.parametrize("mk, M", [
    (lambda: cells.circle_cell(32, 0.3), 3),
    (lambda: cells.voronoi_cell(24, 6, seed=8, lattice="hex"), 4),
])
def test_pixel_mesh_equals_pixel_cell(mk, M):
    """Square elements at the pixel centres with area V/P^2 are the pixel
    quadrature itself, so the pencil and its eigenvalues are the same."""
    cell = mk()
    a = mv.OracleCell(cell, M).omega(Q, 8)
    b = mv.OracleCell(cells.pixel_mesh(cell), M).omega(Q, 8)
    assert np.abs(a - b).max() <= 1e-13 * a.max()


def test_mesh_translation_invariance():
    """Moving every centroid by the same (non-grid) vector multiplies the
    form factors by exp(-i G . s): a unitary similarity of the pencil."""
    m = cells.mesh_voronoi_cell(16, 10, seed=3, lattice="hex")
    a = mv.OracleCell(m, 3).omega(Q, 8)
    b = mv.OracleCell(m.translated(0.137, -0.291), 3).omega(Q, 8)
    assert np.abs(a - b).max() <= 1e-11 * a.max()


def test_homogeneous_mesh_converges_to_closed_form():
    """A homogeneous cell meshed ever finer approaches omega = c_L |K|, c_T |K|
    (the centroid rule integrates the plane waves better as the elements shrink)."""
    errs = [homogeneous_error(cells.mesh_circle_cell(n, matrix=(LAM, MU, RHO),
                                                     inclusion=(LAM, MU, RHO)), 2)
            for n in (6, 12, 24)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] <= 1e-3 and errs[2] <= 1e-5, errs


def test_mesh_density_scaling():
    m = cells.mesh_circle_cell(10)
    a = mv.OracleCell(m, 2).omega(Q, 8)
    b = mv.OracleCell(m.with_props(rho=4.0 * m.rho), 2).omega(Q, 8)
    assert np.allclose(b, a / 2.0, rtol=1e-12, atol=1e-12 * a.max())


def test_planted_vertex_for_centroid_fails():
    """Evaluating the plane waves at a vertex instead of the centroid (a
    plausible mistake) is caught by the convergence pin."""
    n = 24
    tris = cells.jittered_triangles(n, 0.3, 0)
    good = cells.mesh_circle_cell(n, matrix=(LAM, MU, RHO), inclusion=(LAM, MU, RHO))
    bad = cells.MeshCell(good.h1, good.h2, tris[:, 0, :].copy(), good.area, good.phase,
                         good.lam, good.mu, good.rho)
    assert homogeneous_error(good, 2) <= 1e-5
    assert homogeneous_error(bad, 2) > 1e-4


def test_paper_integrand_on_a_mesh():
    """The paper's own GPU formulation (Eq. (eExp): the integrand tensor from
    element centroids and areas, T = A^-1) on a triangle mesh equals the
    mesh form factors expanded to plane-wave pairs (paper sign convention)."""
    m = cells.mesh_voronoi_cell(6, 4, seed=3, lattice="hex")
    M = 2
    Q = np.array([0.31, -0.17])
    x, w, ph = mv.subdomains(m)
    rho = m.rho[ph]
    lit = mv.integrals_literal(m, M, Q, rho)
    T = mv.toeplitz(mv.form_factors(rho[None], x, w, m.h1, m.h2, M, paper_conj=True)[0], M)
    assert np.allclose(lit, T, atol=1e-14 * np.abs(T).max())


def test_golden_stop_bands_on_the_papers_kind_of_mesh():
    """The paper's worked example (Sec. IV.B) on a 968-triangle mesh, close to
    its 964-triangle one: the oracle's stop bands (first 12 branches, M = 5)
    match the printed 120-262 kHz and 427-473 kHz to 1 %."""
    ref = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden",
                                  "hex_steel_epoxy_stop_bands.txt"))
    cell = cells.steel_epoxy_hex_mesh(22)
    Qs = cells.ibz_path("hex", 46, cell.h1, cell.h2)
    f = mv.bands(cell, 5, Qs, 12) / (2 * np.pi) / 1e3
    gaps = [(f[:, i].max(), f[:, i + 1].min()) for i in range(11)
            if f[:, i + 1].min() - f[:, i].max() > 10.0]
    assert np.array(gaps).shape == ref.shape
    assert np.allclose(gaps, ref, rtol=0.01)
