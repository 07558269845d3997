"""Mesh cells (centroid rule over triangles, Sec. III) through the C ABI
against the oracle: form factors, the reduced matrix, frequencies on the
FP64, mixed and LOBPCG paths, stress coefficients, the pixel mesh against
the pixel path, and argument errors."""
import os

import numpy as np
import pytest

from oracle import mixed_variational as mv
from oracle import mode_shapes as ms
from paper_1310_6380_gb300 import cells

from _helpers import omega_floor, omega_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1310_6380_gb300 import binding as bs  # noqa: E402

QS = np.array([[0.0, 0.0], [0.21, 0.07], [0.5, 0.0], [0.4, 0.3], [2 / 3, 1 / 3]])

MESHES = [
    ("circle_square", lambda: cells.mesh_circle_cell(16), 3),
    ("steel_epoxy_hex_968", lambda: cells.steel_epoxy_hex_mesh(22), 5),
    ("voronoi_hex", lambda: cells.mesh_voronoi_cell(20, 12, seed=9, lattice="hex"), 4),
]


def make(m, M, prec=bs.BS_PREC_FP64, assemble=True):
    h = bs.bs_create_cell_mesh(m.h1, m.h2, np.ascontiguousarray(m.centroid),
                               np.ascontiguousarray(m.area),
                               np.ascontiguousarray(m.phase, np.uint16), m.lam.copy(),
                               m.mu.copy(), m.rho.copy(), M, prec)
    if assemble:
        bs.bs_assemble(h)
    return h


@pytest.mark.parametrize("name, mk, M", MESHES)
def test_mesh_form_factors(name, mk, M):
    m = mk()
    h = make(m, M)
    D = 4 * M + 1
    out = np.empty(3 * D * D * 2)
    try:
        bs.bs_form_factors(h, out)
    finally:
        bs.bs_destroy_cell(h)
    got = out.view(np.complex128).reshape(3, D, D)
    x, w, ph = mv.subdomains(m)
    fields = np.array([1.0 / (m.lam + m.mu), 1.0 / m.mu, m.rho])[:, ph]
    ref = mv.form_factors(fields, x, w, m.h1, m.h2, M)
    for f in range(3):
        assert np.abs(got[f] - ref[f]).max() <= 1e-13 * np.abs(ref[f]).max(), (name, f)


@pytest.mark.parametrize("name, mk, M", MESHES)
def test_mesh_reduced_matrix(name, mk, M):
    m = mk()
    h = make(m, M)
    N, n = bs.bs_cell_dims(h)
    oc = mv.OracleCell(m, M)
    try:
        for Q in QS[1:4]:
            out = np.empty(n * n * 2)
            bs.bs_reduced_matrix(h, Q, out)
            got = out.view(np.complex128).reshape(n, n).T
            A, Om = oc.pencil(Q)
            Li = np.linalg.inv(np.linalg.cholesky(Om))
            ref = Li @ A @ Li.conj().T
            low = np.tril_indices(n)
            assert np.abs(got[low] - ref[low]).max() <= 1e-11 * np.abs(ref).max(), (name, Q)
    finally:
        bs.bs_destroy_cell(h)


@pytest.mark.parametrize("name, mk, M", MESHES)
def test_mesh_frequencies_all_paths(name, mk, M):
    """FP64 path to 1e-8, mixed path and LOBPCG to 1e-6 of the oracle."""
    m = mk()
    nb = 12
    oc = mv.OracleCell(m, M)
    ref = np.array([oc.omega(q, nb) for q in QS])
    fl = omega_floor(m)
    h = make(m, M)
    try:
        w = np.empty((len(QS), nb))
        st = np.empty(len(QS), np.int32)
        bs.bs_solve_k(h, QS, nb, w, st)
        assert not st.any()
        assert omega_rel_err(w, ref, fl).max() <= 1e-8, name
    finally:
        bs.bs_destroy_cell(h)
    h = make(m, M, bs.BS_PREC_MIXED)
    try:
        w = np.empty((len(QS), nb))
        bs.bs_solve_k(h, QS, nb, w, st)
        assert not st.any()
        assert omega_rel_err(w, ref, fl).max() <= 1e-6, name
        w2 = np.empty((len(QS), nb))
        bs.bs_solve_k_lobpcg(h, QS, nb, w2, status_out=st)
        assert not st.any()
        assert omega_rel_err(w2, ref, fl).max() <= 1e-6, name
    finally:
        bs.bs_destroy_cell(h)


def test_mesh_stress_matches_oracle():
    m = cells.mesh_voronoi_cell(16, 8, seed=4)
    M, nvec = 3, 4
    oc = mv.OracleCell(m, M)
    rng = np.random.default_rng(2)
    U = rng.standard_normal((3, nvec, 2 * oc.N)) + 1j * rng.standard_normal((3, nvec, 2 * oc.N))
    S = np.empty((3, nvec, 3 * oc.N), np.complex128)
    h = make(m, M)
    try:
        bs.bs_stress_coefficients(h, QS[1:4], U, S)
    finally:
        bs.bs_destroy_cell(h)
    for i, q in enumerate(QS[1:4]):
        ref = ms.stress_coefficients(oc, q, U[i])
        # one scale per wavevector: at Gamma the rigid translations have S = 0 exactly,
        # and their rounding follows the size of the other modes' terms
        scale = np.abs(ref).max()
        assert (np.abs(S[i] - ref) <= 1e-10 * scale).all(), i


def test_pixel_mesh_matches_pixel_path():
    """The same subdomains through the mesh kernels (FP64 CUDA cores) and the
    pixel kernels (tcgen05 exact slices): the same frequencies."""
    cell = cells.voronoi_cell(24, 6, seed=8, lattice="hex")
    M, nb = 4, 10
    pm = cells.pixel_mesh(cell)
    hp = bs.bs_create_cell(cell.h1, cell.h2, np.ascontiguousarray(cell.phase, np.uint16),
                           cell.lam.copy(), cell.mu.copy(), cell.rho.copy(), M, bs.BS_PREC_FP64)
    hm = make(pm, M)
    try:
        bs.bs_assemble(hp)
        wp = np.empty((len(QS), nb))
        wm = np.empty((len(QS), nb))
        bs.bs_solve_k(hp, QS, nb, wp)
        bs.bs_solve_k(hm, QS, nb, wm)
    finally:
        bs.bs_destroy_cell(hp)
        bs.bs_destroy_cell(hm)
    assert omega_rel_err(wm, wp, omega_floor(cell)).max() <= 1e-10


def test_mesh_argument_errors():
    m = cells.mesh_circle_cell(6)                  # 72 elements
    args = lambda **kw: dict(dict(centroid=np.ascontiguousarray(m.centroid),
                                  area=np.ascontiguousarray(m.area),
                                  phase=np.ascontiguousarray(m.phase, np.uint16)), **kw)

    def create(M=2, **kw):
        a = args(**kw)
        return bs.bs_create_cell_mesh(m.h1, m.h2, a["centroid"], a["area"], a["phase"],
                                      m.lam.copy(), m.mu.copy(), m.rho.copy(), M)

    for kw, M in [({}, 5),                                      # (2M+1)^2 = 121 > 72 elements
                  ({"area": -np.ascontiguousarray(m.area)}, 2),
                  ({"phase": np.full(m.nel, 7, np.uint16)}, 2)]:
        with pytest.raises(bs.BSError) as ei:
            create(M, **kw)
        assert ei.value.code == bs.BS_EINVAL
    # every element at one point: the Gram matrices are singular -> BS_ENOTPD
    h = create(2, centroid=np.zeros((m.nel, 2)))
    try:
        bs.bs_assemble(h)
        with pytest.raises(bs.BSError) as ei:
            bs.bs_solve_k(h, QS[1:2], 4, np.empty((1, 4)))
        assert ei.value.code == bs.BS_ENOTPD
    finally:
        bs.bs_destroy_cell(h)


def test_gpu_mesh_reproduces_the_papers_stop_bands():
    """The paper's worked example on a 968-triangle mesh through the GPU FP64
    path: the stop bands of the first 12 branches (M = 5) match the printed
    120-262 kHz and 427-473 kHz to 1 % (tests/golden, Sec. IV.B)."""
    ref = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden",
                                  "hex_steel_epoxy_stop_bands.txt"))
    m = cells.steel_epoxy_hex_mesh(22)
    Qs = np.ascontiguousarray(cells.ibz_path("hex", 46, m.h1, m.h2))
    h = make(m, 5)
    try:
        w = np.empty((len(Qs), 12))
        st = np.empty(len(Qs), np.int32)
        bs.bs_solve_k(h, Qs, 12, w, st)
    finally:
        bs.bs_destroy_cell(h)
    assert not st.any()
    f = w / (2 * np.pi) / 1e3
    gaps = [(f[:, i].max(), f[:, i + 1].min()) for i in range(11)
            if f[:, i + 1].min() - f[:, i].max() > 10.0]
    assert np.array(gaps).shape == ref.shape
    assert np.allclose(gaps, ref, rtol=0.01)
