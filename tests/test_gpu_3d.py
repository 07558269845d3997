"""3-D voxel cells through the C ABI against the 3-D oracle: form factors,
the reduced matrix, frequencies (FP64 path, 1e-8), the homogeneous closed
form at the largest tested truncation, an extruded cell against the 2-D
path, and argument errors."""
import numpy as np
import pytest

from oracle import mixed_variational_3d as mv3
from paper_1310_6380_gb300 import cells

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1310_6380_gb300 import binding as bs  # noqa: E402

QS = np.array([[0.0, 0.0, 0.0], [0.21, 0.07, -0.13], [0.5, 0.0, 0.0], [0.5, 0.5, 0.5],
               [0.3, -0.4, 0.1]])


def make(cell, M, assemble=True):
    h = bs.bs_create_cell3(cell.h1, cell.h2, cell.h3, np.ascontiguousarray(cell.phase, np.uint16),
                           cell.lam.copy(), cell.mu.copy(), cell.rho.copy(), M)
    if assemble:
        bs.bs_assemble3(h)
    return h


def floor3(cell):
    A = np.array([cell.h1, cell.h2, cell.h3])
    qm = 2 * np.pi * np.linalg.inv(A)
    return np.sqrt(np.min(cell.mu / cell.rho)) * min(np.linalg.norm(qm[:, i]) for i in range(3)) / 2


def rel3(w, ref, fl):
    return np.abs(w ** 2 - ref ** 2) / (2 * np.maximum(ref ** 2, fl ** 2))


def triclinic_voronoi():
    c = cells.voronoi_cell3(10, 6, seed=5)
    return cells.Cell3(np.array([1.0, 0.0, 0.0]), np.array([0.3, 0.9, 0.0]),
                       np.array([0.2, -0.1, 1.1]), c.phase, c.lam, c.mu, c.rho, "triclinic")


CASES = [
    ("sphere", lambda: cells.sphere_cell3(8, 0.3), 2),
    ("voronoi", lambda: cells.voronoi_cell3(10, 8, seed=3), 2),
    ("triclinic", triclinic_voronoi, 2),
    ("sphere_M1", lambda: cells.sphere_cell3(6, 0.35), 1),
]


@pytest.mark.parametrize("name, mk, M", CASES[:2])
def test_form_factors3(name, mk, M):
    cell = mk()
    h = make(cell, M)
    D = 4 * M + 1
    out = np.empty(3 * D ** 3 * 2)
    try:
        bs.bs_form_factors3(h, out)
    finally:
        bs.bs_destroy_cell3(h)
    got = out.view(np.complex128).reshape(3, D, D, D)
    x, w = mv3.quadrature3(cell)
    ph = cell.phase.reshape(-1).astype(np.int64)
    fields = np.array([1.0 / (3 * cell.lam + 2 * cell.mu), 1.0 / cell.mu, cell.rho])[:, ph]
    q = mv3.reciprocal_basis3(cell.h1, cell.h2, cell.h3)
    ref = mv3.form_factors3(fields, x, w, q, M)
    for f in range(3):
        assert np.abs(got[f] - ref[f]).max() <= 1e-13 * np.abs(ref[f]).max(), (name, f)


@pytest.mark.parametrize("name, mk, M", CASES[:3])
def test_reduced_matrix3(name, mk, M):
    cell = mk()
    h = make(cell, M)
    N, n = bs.bs_cell3_dims(h)
    oc = mv3.OracleCell3(cell, M)
    try:
        for Q in QS[1:4]:
            out = np.empty(n * n * 2)
            bs.bs_reduced_matrix3(h, Q, out)
            got = out.view(np.complex128).reshape(n, n).T
            A, Om = oc.pencil(Q)
            Li = np.linalg.inv(np.linalg.cholesky(Om))
            ref = Li @ A @ Li.conj().T
            low = np.tril_indices(n)
            assert np.abs(got[low] - ref[low]).max() <= 1e-11 * np.abs(ref).max(), (name, Q)
    finally:
        bs.bs_destroy_cell3(h)


@pytest.mark.parametrize("name, mk, M", CASES)
def test_frequencies3(name, mk, M):
    cell = mk()
    nb = 12
    oc = mv3.OracleCell3(cell, M)
    ref = np.array([oc.omega(q, nb) for q in QS])
    h = make(cell, M)
    try:
        w = np.empty((len(QS), nb))
        st = np.empty(len(QS), np.int32)
        bs.bs_solve_k3(h, QS, nb, w, st)
    finally:
        bs.bs_destroy_cell3(h)
    assert not st.any()
    assert rel3(w, ref, floor3(cell)).max() <= 1e-8, name


def test_homogeneous_closed_form_M4():
    """n = 3 (2M+1)^3 = 2187: every band of a homogeneous cell is c_L |K| or c_T |K|."""
    lam, mu, rho = 4.0, 1.5, 1.2
    P, M, nb = 10, 4, 40
    h1, h2, h3 = np.eye(3)
    h = bs.bs_create_cell3(h1, h2, h3, np.zeros((P, P, P), np.uint16), np.array([lam]),
                           np.array([mu]), np.array([rho]), M)
    try:
        bs.bs_assemble3(h)
        Q = QS[1:3]
        w = np.empty((len(Q), nb))
        bs.bs_solve_k3(h, Q, nb, w)
    finally:
        bs.bs_destroy_cell3(h)
    for i, q in enumerate(Q):
        K = np.linalg.norm(mv3.wavevectors3(q, h1, h2, h3, M), axis=1)
        ref = np.sort(np.concatenate([np.sqrt((lam + 2 * mu) / rho) * K, np.sqrt(mu / rho) * K,
                                      np.sqrt(mu / rho) * K]))[:nb]
        assert np.abs(w[i] - ref).max() <= 1e-9 * ref.max(), i


def test_extruded_cell_contains_the_2d_gpu_bands():
    """Two GPU paths against each other: an extruded cell with one Poisson
    ratio (lam = 2 mu) at k3 = 0 has every in-plane band of the 2-D path."""
    base = cells.voronoi_cell(8, 3, seed=4)
    c2 = base.with_props(lam=2.0 * base.mu)
    c3 = cells.extruded_cell3(c2)
    M, nb2 = 1, 8
    h2 = bs.bs_create_cell(c2.h1, c2.h2, np.ascontiguousarray(c2.phase, np.uint16), c2.lam.copy(),
                           c2.mu.copy(), c2.rho.copy(), M, bs.BS_PREC_FP64)
    h3 = make(c3, M)
    try:
        bs.bs_assemble(h2)
        Q2 = np.array([[0.31, 0.12]])
        w2 = np.empty((1, nb2))
        bs.bs_solve_k(h2, Q2, nb2, w2)
        n3 = bs.bs_cell3_dims(h3)[1]
        w3 = np.empty((1, n3))
        bs.bs_solve_k3(h3, np.array([[0.31, 0.12, 0.0]]), n3, w3)
    finally:
        bs.bs_destroy_cell(h2)
        bs.bs_destroy_cell3(h3)
    gap = np.array([np.abs(w3[0] ** 2 - v ** 2).min() for v in w2[0]])
    assert gap.max() <= 1e-9 * w2[0].max() ** 2


def test_3d_argument_errors():
    c = cells.sphere_cell3(6, 0.3)
    with pytest.raises(bs.BSError) as ei:
        make(c, 3)                                  # 2M + 1 = 7 > P = 6
    assert ei.value.code == bs.BS_EINVAL
    with pytest.raises(bs.BSError) as ei:
        bs.bs_create_cell3(c.h1, c.h2, c.h3, np.ascontiguousarray(c.phase, np.uint16),
                           c.lam.copy(), np.array([1.5, -1.0]), c.rho.copy(), 1)
    assert ei.value.code == bs.BS_EINVAL
    h = make(c, 1, assemble=False)
    try:
        with pytest.raises(bs.BSError) as ei:
            bs.bs_solve_k3(h, QS[1:2], 4, np.empty((1, 4)))
        assert ei.value.code == bs.BS_ESTATE
        bs.bs_assemble3(h)
        bs.bs_solve_k3(h, np.zeros((0, 3)), 4, np.empty((0, 4)))
        with pytest.raises(bs.BSError) as ei:
            bs.bs_solve_k3(h, QS[1:2], 82, np.empty((1, 82)))          # n = 81
        assert ei.value.code == bs.BS_EINVAL
    finally:
        bs.bs_destroy_cell3(h)
