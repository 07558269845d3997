"""Mode shapes through the C ABI against the FP64 oracle: stress coefficients
S = -Phi^-1 H^* U (FP64, to 1e-10 of the largest |S| at each k) and plane-wave fields on a grid
(FP32, within the documented bound (2(2M+1) + 4) 2^-24 sum |coef| per point)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import mixed_variational as mv
from oracle import mode_shapes as ms
from paper_1310_6380_gb300 import cells

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1310_6380_gb300 import binding as bs  # noqa: E402

QS = np.array([[0.0, 0.0], [0.21, 0.07], [0.5, 0.5], [0.33, -0.29]])
U32 = 2.0 ** -24


def make(cell, M, prec=bs.BS_PREC_FP64, assemble=True):
    h = bs.bs_create_cell(cell.h1, cell.h2, np.ascontiguousarray(cell.phase, np.uint16),
                          cell.lam.copy(), cell.mu.copy(), cell.rho.copy(), M, prec)
    if assemble:
        bs.bs_assemble(h)
    return h


def oracle_modes(oc, Q, nvec):
    A, Om = oc.pencil(Q)
    lam, V = sla.eigh(A, Om, subset_by_index=[0, nvec - 1])
    return lam, np.ascontiguousarray(V.T)


def field_bound(M, coef):
    return (2 * (2 * M + 1) + 4) * U32 * np.abs(coef).sum(axis=-1)


@pytest.mark.parametrize("name, mk, M, prec", [
    ("c0_circle", lambda: cells.config0()["cell"], 3, bs.BS_PREC_FP64),
    ("hex_voronoi_mixed", lambda: cells.voronoi_cell(48, 9, seed=21, lattice="hex"), 5,
     bs.BS_PREC_MIXED),
    ("c3_cell", lambda: cells.config3_cell(2)["cell"], 6, bs.BS_PREC_MIXED),
])
def test_stress_matches_oracle(name, mk, M, prec):
    cell = mk()
    oc = mv.OracleCell(cell, M)
    nvec = 6
    U = np.stack([oracle_modes(oc, q, nvec)[1] for q in QS])          # (nk, nvec, 2N)
    rng = np.random.default_rng(7)
    U[-1, -1] = rng.standard_normal(2 * oc.N) + 1j * rng.standard_normal(2 * oc.N)
    U = np.ascontiguousarray(U)
    S = np.empty((len(QS), nvec, 3 * oc.N), np.complex128)
    h = make(cell, M, prec)
    try:
        bs.bs_stress_coefficients(h, QS, U, S)
    finally:
        bs.bs_destroy_cell(h)
    for i, q in enumerate(QS):
        ref = ms.stress_coefficients(oc, q, U[i])
        # one scale per wavevector: at Gamma the rigid translations have S = 0 exactly,
        # and their rounding follows the size of the other modes' terms
        scale = np.abs(ref).max()
        assert (np.abs(S[i] - ref) <= 1e-10 * scale).all(), (name, i, np.abs(S[i] - ref).max())


def test_stress_of_lobpcg_vectors_satisfies_first_block_row():
    """End to end: LOBPCG modes (complex64) -> GPU stress -> H S + lambda Omega U = 0
    of the oracle to the FP32 level of the vectors."""
    cell = cells.config3_cell(5)["cell"]
    M, nb = 5, 8
    h = make(cell, M, bs.BS_PREC_MIXED)
    try:
        Q = QS[1:]
        nk = len(Q)
        N, n = bs.bs_cell_dims(h)
        w = np.empty((nk, nb))
        fb = np.empty(nk, np.int32)
        vec = np.empty((nk, nb, n), np.complex64)
        bs.bs_solve_k_lobpcg(h, Q, nb, w, fallback_out=fb, vec_out=vec)
        U = np.ascontiguousarray(vec.astype(np.complex128))
        S = np.empty((nk, nb, 3 * N), np.complex128)
        bs.bs_stress_coefficients(h, Q, U, S)
    finally:
        bs.bs_destroy_cell(h)
    oc = mv.OracleCell(cell, M)
    for i, q in enumerate(Q):
        if fb[i]:
            continue
        H = oc.H(q)
        A2 = np.linalg.norm(oc.pencil(q)[0], 2)
        for j in range(nb):
            lam = w[i, j] ** 2
            r = H @ S[i, j] + lam * (oc.Omega @ U[i, j])
            assert np.linalg.norm(r) <= 1e-5 * A2 * np.linalg.norm(U[i, j]), (i, j)


@pytest.mark.parametrize("M, G", [(3, 37), (5, 64), (6, 300), (15, 40)])
def test_mode_field_matches_oracle(M, G):
    """Ragged grids (G = 37, 300 spans two column passes of 150), the largest
    truncation (2M + 1 = 31), displacement and stress fields of oracle modes."""
    cell = cells.voronoi_cell(64, 10, seed=M, lattice="hex" if M % 2 else "square")
    oc = mv.OracleCell(cell, M)
    N = oc.N
    Q = QS[1:3]
    nvec = 2
    coef = []
    for q in Q:
        lam, U = oracle_modes(oc, q, nvec)
        S = ms.stress_coefficients(oc, q, U)
        coef.append(np.concatenate([U.reshape(2 * nvec, N), S.reshape(3 * nvec, N)]))
    coef = np.ascontiguousarray(np.stack(coef))                         # (nk, 5 nvec, N)
    out = np.empty((len(Q), coef.shape[1], G, G), np.complex64)
    h = make(cell, M, assemble=False)
    try:
        bs.bs_mode_field(h, Q, coef, G, out)
    finally:
        bs.bs_destroy_cell(h)
    for i, q in enumerate(Q):
        ref = ms.field_on_grid(cell, M, q, coef[i], G)
        err = np.abs(out[i].astype(np.complex128) - ref).max(axis=(1, 2))
        assert (err <= field_bound(M, coef[i])).all(), (err, field_bound(M, coef[i]))


def test_mode_field_large_grid_host_chunks_sampled():
    """G = 2100 with host output: the fields are staged in chunks that split a
    wavevector's fields; sampled points against the oracle one by one."""
    cell = cells.config0()["cell"]
    M, G = 3, 2100
    N = (2 * M + 1) ** 2
    rng = np.random.default_rng(11)
    Q = rng.uniform(-0.5, 0.5, (6, 2))
    coef = rng.standard_normal((6, 2, N)) + 1j * rng.standard_normal((6, 2, N))
    out = np.empty((6, 2, G, G), np.complex64)
    h = make(cell, M, assemble=False)
    try:
        bs.bs_mode_field(h, Q, coef, G, out)
    finally:
        bs.bs_destroy_cell(h)
    pts = rng.integers(0, G, (64, 2))
    pts = np.vstack([pts, [[0, 0], [G - 1, G - 1], [0, G - 1], [G - 1, 0]]])
    x = ((pts[:, :1] + 0.5) / G) * cell.h1 + ((pts[:, 1:] + 0.5) / G) * cell.h2
    for i in range(6):
        ref = ms.plane_wave_sum(cell, M, Q[i], coef[i], x)               # (2, npts)
        got = out[i][:, pts[:, 0], pts[:, 1]]
        err = np.abs(got - ref).max(axis=1)
        assert (err <= field_bound(M, coef[i])).all(), (i, err)


def test_mode_paths_device_pointers_equal_host():
    cell = cells.voronoi_cell(32, 6, seed=4)
    M, G, nvec = 4, 48, 3
    oc = mv.OracleCell(cell, M)
    N = oc.N
    rng = np.random.default_rng(5)
    U = rng.standard_normal((3, nvec, 2 * N)) + 1j * rng.standard_normal((3, nvec, 2 * N))
    Q = QS[1:]
    h = make(cell, M)
    try:
        S = np.empty((3, nvec, 3 * N), np.complex128)
        bs.bs_stress_coefficients(h, Q, U, S)
        Sd = torch.empty((3, nvec, 3 * N), dtype=torch.complex128, device="cuda")
        bs.bs_stress_coefficients(h, torch.tensor(Q, device="cuda"),
                                  torch.tensor(U, device="cuda"), Sd)
        F = np.empty((3, 3 * nvec, G, G), np.complex64)
        coef = np.ascontiguousarray(S.reshape(3, 3 * nvec, N))
        bs.bs_mode_field(h, Q, coef, G, F)
        Fd = torch.empty((3, 3 * nvec, G, G), dtype=torch.complex64, device="cuda")
        bs.bs_mode_field(h, torch.tensor(Q, device="cuda"), torch.tensor(coef, device="cuda"), G,
                         Fd)
        torch.cuda.synchronize()
    finally:
        bs.bs_destroy_cell(h)
    assert np.array_equal(Sd.cpu().numpy(), S)
    assert np.array_equal(Fd.cpu().numpy(), F)


def test_mode_edge_cases_and_errors():
    cell = cells.config0()["cell"]
    # M = 0: one plane wave per component, the field is coef * exp(i k . x)
    h0 = make(cell, 0, assemble=False)
    try:
        Q = np.array([[0.3, -0.2]])
        coef = np.array([[[1.5 - 0.5j]]])
        out = np.empty((1, 1, 5, 5), np.complex64)
        bs.bs_mode_field(h0, Q, coef, 5, out)
        ref = ms.field_on_grid(cell, 0, Q[0], coef[0], 5)
        assert np.abs(out[0] - ref).max() <= field_bound(0, coef[0]).max()
        one = np.empty((1, 1, 1, 1), np.complex64)                       # G = 1: the centre
        bs.bs_mode_field(h0, Q, coef, 1, one)
        assert np.abs(one[0, 0, 0, 0] - ms.field_on_grid(cell, 0, Q[0], coef[0], 1)[0, 0, 0]) \
            <= field_bound(0, coef[0]).max()
        with pytest.raises(bs.BSError) as ei:
            bs.bs_stress_coefficients(h0, Q, np.zeros((1, 1, 2), np.complex128),
                                      np.zeros((1, 1, 3), np.complex128))
        assert ei.value.code == bs.BS_ESTATE
        with pytest.raises(bs.BSError) as ei:
            bs.bs_mode_field(h0, Q, coef, 0, out)
        assert ei.value.code == bs.BS_EINVAL
    finally:
        bs.bs_destroy_cell(h0)
    h = make(cell, 2)
    try:
        N = 25
        bs.bs_stress_coefficients(h, np.zeros((0, 2)), np.zeros((0, 1, 2 * N), np.complex128),
                                  np.zeros((0, 1, 3 * N), np.complex128))
        bs.bs_mode_field(h, np.zeros((0, 2)), np.zeros((0, 1, N), np.complex128), 8,
                         np.zeros((0, 1, 8, 8), np.complex64))
        with pytest.raises(bs.BSError) as ei:
            bs.bs_stress_coefficients(h, QS, np.zeros((4, 0, 2 * N), np.complex128),
                                      np.zeros((4, 0, 3 * N), np.complex128))
        assert ei.value.code == bs.BS_EINVAL
    finally:
        bs.bs_destroy_cell(h)
