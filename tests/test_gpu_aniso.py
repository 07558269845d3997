"""General in-plane stiffness per phase (the full Phi of Eq. (ep)) through the
C ABI against the oracle: form factors of the seven fields, the reduced
matrix, frequencies on the FP64, mixed and LOBPCG paths, stress, pixel and
mesh cells, the isotropic special case against the isotropic path, and
argument errors."""
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


def c6(cell):
    C = cell.stiffness
    return np.ascontiguousarray(np.stack([C[:, 0, 0], C[:, 1, 1], C[:, 0, 1], C[:, 0, 2],
                                          C[:, 1, 2], C[:, 2, 2]], axis=1))


def make(cell, M, prec=bs.BS_PREC_FP64, assemble=True):
    if hasattr(cell, "centroid"):
        h = bs.bs_create_cell_mesh(cell.h1, cell.h2, np.ascontiguousarray(cell.centroid),
                                   np.ascontiguousarray(cell.area),
                                   np.ascontiguousarray(cell.phase, np.uint16), cell.lam.copy(),
                                   cell.mu.copy(), cell.rho.copy(), M, prec)
    else:
        h = bs.bs_create_cell(cell.h1, cell.h2, np.ascontiguousarray(cell.phase, np.uint16),
                              cell.lam.copy(), cell.mu.copy(), cell.rho.copy(), M, prec)
    if getattr(cell, "stiffness", None) is not None:
        bs.bs_set_stiffness(h, c6(cell))
    if assemble:
        bs.bs_assemble(h)
    return h


CELLS = [
    ("voronoi_hex", lambda: cells.anisotropic_cell(
        cells.voronoi_cell(24, 6, seed=8, lattice="hex"), seed=3), 4),
    ("ellipses_square", lambda: cells.anisotropic_cell(cells.ellipse_cell(32, 3, seed=2),
                                                       seed=5), 3),
    ("mesh_voronoi", lambda: cells.anisotropic_cell(
        cells.mesh_voronoi_cell(16, 8, seed=4, lattice="hex"), seed=7), 3),
]


@pytest.mark.parametrize("name, mk, M", CELLS[:2])
def test_aniso_form_factors(name, mk, M):
    cell = mk()
    h = make(cell, M)
    D = 4 * M + 1
    out = np.empty(7 * D * D * 2)
    try:
        bs.bs_form_factors(h, out)
    finally:
        bs.bs_destroy_cell(h)
    got = out.view(np.complex128).reshape(7, D, D)
    S = np.linalg.inv(cell.stiffness)
    x, w, ph = mv.subdomains(cell)
    fields = np.array([S[:, 0, 0], S[:, 1, 1], cell.rho, S[:, 0, 1], S[:, 0, 2], S[:, 1, 2],
                       S[:, 2, 2]])[:, ph]
    ref = mv.form_factors(fields, x, w, cell.h1, cell.h2, M)
    for f in range(7):
        assert np.abs(got[f] - ref[f]).max() <= 1e-13 * np.abs(ref[f]).max(), (name, f)


@pytest.mark.parametrize("name, mk, M", CELLS)
def test_aniso_reduced_matrix(name, mk, M):
    cell = mk()
    h = make(cell, M)
    N, n = bs.bs_cell_dims(h)
    oc = mv.OracleCell(cell, M)
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


@pytest.mark.parametrize("name, mk, M", CELLS)
def test_aniso_frequencies_all_paths(name, mk, M):
    cell = mk()
    nb = 12
    oc = mv.OracleCell(cell, M)
    ref = np.array([oc.omega(q, nb) for q in QS])
    fl = omega_floor(cell)
    st = np.empty(len(QS), np.int32)
    h = make(cell, M)
    try:
        w = np.empty((len(QS), nb))
        bs.bs_solve_k(h, QS, nb, w, st)
        assert not st.any()
        assert omega_rel_err(w, ref, fl).max() <= 1e-8, name
    finally:
        bs.bs_destroy_cell(h)
    h = make(cell, M, bs.BS_PREC_MIXED)
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


def test_isotropic_stiffness_matches_isotropic_path():
    """The isotropic materials given as general stiffnesses take the full-Phi
    path; the bands equal those of the block-diagonal isotropic path."""
    base = cells.config0()["cell"]
    iso = cells.with_stiffness(base, cells.isotropic_stiffness(base.lam, base.mu))
    M, nb = 3, 8
    hb, hi = make(base, M), make(iso, M)
    try:
        wb = np.empty((len(QS), nb))
        wi = np.empty((len(QS), nb))
        bs.bs_solve_k(hb, QS, nb, wb)
        bs.bs_solve_k(hi, QS, nb, wi)
    finally:
        bs.bs_destroy_cell(hb)
        bs.bs_destroy_cell(hi)
    assert omega_rel_err(wi, wb, omega_floor(base)).max() <= 1e-10


def test_homogeneous_aniso_is_christoffel():
    C = cells.rotated_orthotropic(120.0, 40.0, 25.0, 18.0, 0.61)
    cell = cells.with_stiffness(cells.homogeneous_cell(16, 4.0, 1.5, 1.3, lattice="hex"), C[None])
    M, nb = 3, 12
    h = make(cell, M)
    try:
        w = np.empty((len(QS), nb))
        bs.bs_solve_k(h, QS, nb, w)
    finally:
        bs.bs_destroy_cell(h)
    for i, q in enumerate(QS):
        K = mv.wavevectors(q, cell.h1, cell.h2, M)
        ref = []
        for k1, k2 in K:
            Nk = np.array([[k1, 0.0], [0.0, k2], [k2, k1]])
            ref.extend(np.linalg.eigvalsh(Nk.T @ C @ Nk) / 1.3)
        ref = np.sqrt(np.maximum(np.sort(ref)[:nb], 0.0))
        assert omega_rel_err(w[i], ref, omega_floor(cell)).max() <= 1e-9, i


@pytest.mark.parametrize("which", [0, 2])
def test_aniso_stress_matches_oracle(which):
    name, mk, M = CELLS[which]
    cell = mk()
    oc = mv.OracleCell(cell, M)
    nvec = 4
    rng = np.random.default_rng(which)
    U = rng.standard_normal((3, nvec, 2 * oc.N)) + 1j * rng.standard_normal((3, nvec, 2 * oc.N))
    S = np.empty((3, nvec, 3 * oc.N), np.complex128)
    h = make(cell, M)
    try:
        bs.bs_stress_coefficients(h, QS[1:4], U, S)
    finally:
        bs.bs_destroy_cell(h)
    for i, q in enumerate(QS[1:4]):
        ref = ms.stress_coefficients(oc, q, U[i])
        assert np.abs(S[i] - ref).max() <= 1e-10 * np.abs(ref).max(), (name, i)


def test_aniso_argument_errors():
    base = cells.config0()["cell"]
    h = make(base, 2, assemble=False)
    try:
        bad = np.tile([1.0, 1.0, 2.0, 0.0, 0.0, 1.0], (base.nphase, 1))   # C12 > sqrt(C11 C22)
        with pytest.raises(bs.BSError) as ei:
            bs.bs_set_stiffness(h, bad)
        assert ei.value.code == bs.BS_EINVAL
        good = np.tile([10.0, 8.0, 2.0, 0.5, -0.3, 3.0], (base.nphase, 1))
        bs.bs_set_stiffness(h, good)
        with pytest.raises(bs.BSError) as ei:                        # not assembled since
            bs.bs_solve_k(h, QS[1:2], 4, np.empty((1, 4)))
        assert ei.value.code == bs.BS_ESTATE
        bs.bs_assemble(h)
        w = np.empty((1, 4))
        bs.bs_solve_k(h, QS[1:2], 4, w)
        assert np.isfinite(w).all()
    finally:
        bs.bs_destroy_cell(h)


def test_aniso_c1_cell_full_size():
    """The c1 cell with rotated orthotropic phases at M = 10 (n = 882), as the
    benchmark solves it: the W and monomial products run on the exact-slice
    tensor path (6N = 2646 <= 4096); sampled wavevectors against the oracle."""
    cfg = cells.config1()
    cell = cells.anisotropic_cell(cfg["cell"], seed=6380)
    M, nb = cfg["M"], cfg["nbands"]
    Q = cfg["Q"][[0, 37, 71]]
    h = make(cell, M)
    try:
        w = np.empty((len(Q), nb))
        st = np.empty(len(Q), np.int32)
        bs.bs_solve_k(h, np.ascontiguousarray(Q), nb, w, st)
        assert not st.any()
    finally:
        bs.bs_destroy_cell(h)
    oc = mv.OracleCell(cell, M)
    fl = omega_floor(cell)
    for i, q in enumerate(Q):
        assert omega_rel_err(w[i], oc.omega(q, nb), fl).max() <= 1e-8, i


def test_aniso_products_beyond_the_exact_slice_limit():
    """M = 13 (N = 729, 6N = 4374 > 4096): the W and monomial products fall
    back to FP64 complex GEMMs on the CUDA cores; one wavevector against the
    oracle."""
    cell = cells.anisotropic_cell(cells.voronoi_cell(40, 8, seed=13), seed=11)
    M, nb = 13, 8
    q = np.array([[0.31, 0.12]])
    h = make(cell, M)
    try:
        w = np.empty((1, nb))
        st = np.empty(1, np.int32)
        bs.bs_solve_k(h, q, nb, w, st)
        assert not st.any()
    finally:
        bs.bs_destroy_cell(h)
    ref = mv.OracleCell(cell, M).omega(q[0], nb)
    assert omega_rel_err(w[0], ref, omega_floor(cell)).max() <= 1e-8


def test_aniso_reduced_matrix_full_size():
    """C(k) of the c1 cell with orthotropic phases at M = 10 (n = 882): the
    3N = 1323 factor of Phi is inverted by doubling and the W_i and
    monomial products run on the exact-slice tensor path; against the
    oracle's literal pencil."""
    cell = cells.anisotropic_cell(cells.config1()["cell"], seed=6380)
    M = 10
    h = make(cell, M)
    N, n = bs.bs_cell_dims(h)
    oc = mv.OracleCell(cell, M)
    try:
        Q = np.array([0.37, 0.11])
        out = np.empty(n * n * 2)
        bs.bs_reduced_matrix(h, Q, out)
    finally:
        bs.bs_destroy_cell(h)
    got = out.view(np.complex128).reshape(n, n).T
    A, Om = oc.pencil(Q)
    Li = np.linalg.inv(np.linalg.cholesky(Om))
    ref = Li @ A @ Li.conj().T
    low = np.tril_indices(n)
    assert np.abs(got[low] - ref[low]).max() <= 1e-11 * np.abs(ref).max()
