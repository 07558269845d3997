"""Block LOBPCG path (FP32 iterations + FP64 Rayleigh-Ritz, dense FP64
fallback) against the FP64 oracle: relative frequency error <= 1e-6 on
every wavevector, eigenvectors that satisfy the oracle's pencil, and a warm
start that needs fewer iterations than the cold one."""
import numpy as np
import pytest

from oracle import mixed_variational as mv
from paper_1310_6380_gb300 import cells

from _helpers import omega_floor, omega_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1310_6380_gb300 import binding as bs  # noqa: E402

TOL = 1e-6
QS = np.array([[0.0, 0.0], [0.21, 0.07], [0.5, 0.0], [0.5, 0.5], [0.33, 0.29], [0.05, 0.0]])


def make(cell, M):
    h = bs.bs_create_cell(cell.h1, cell.h2, np.ascontiguousarray(cell.phase, np.uint16),
                          cell.lam.copy(), cell.mu.copy(), cell.rho.copy(), M, bs.BS_PREC_MIXED)
    bs.bs_assemble(h)
    return h


def lobpcg(h, Q, nb, X0=None, vectors=False):
    Q = np.ascontiguousarray(Q, np.float64).reshape(-1, 2)
    nk = len(Q)
    w = np.empty((nk, nb))
    st = np.empty(nk, np.int32)
    it = np.empty(nk, np.int32)
    fb = np.empty(nk, np.int32)
    N, n = bs.bs_cell_dims(h)
    vec = np.empty((nk, nb, n), np.complex64) if vectors else None
    bs.bs_solve_k_lobpcg(h, Q, nb, w, X0=X0, status_out=st, iters_out=it, fallback_out=fb,
                         vec_out=vec)
    return w, st, it, fb, vec


@pytest.mark.parametrize("name, mk, M, nb", [
    ("c0_circle", lambda: cells.config0()["cell"], 3, 8),
    ("hex_voronoi", lambda: cells.voronoi_cell(48, 9, seed=21, lattice="hex"), 5, 10),
    ("homogeneous_degenerate", lambda: cells.homogeneous_cell(12, 4.0, 1.5, 1.2), 3, 12),
    ("c3_cell_3", lambda: cells.config3_cell(3)["cell"], 6, 10),
])
def test_lobpcg_matches_oracle(name, mk, M, nb):
    cell = mk()
    h = make(cell, M)
    try:
        w, st, it, fb, _ = lobpcg(h, QS, nb)
    finally:
        bs.bs_destroy_cell(h)
    oc = mv.OracleCell(cell, M)
    ref = np.array([oc.omega(q, nb) for q in QS])
    err = omega_rel_err(w, ref, omega_floor(cell))
    assert err.max() <= TOL, (name, err.max(), it, fb)
    assert not st.any(), st
    assert (it >= 1).all() and (it <= bs.BS_LOB_MAXIT).all(), it
    # the FP32 iterations, not the dense fallback, carry the solves; a cell
    # whose spectrum is a ladder of exactly degenerate multiplets leaves the
    # certificate no gap inside the block at some wavevectors, and those take
    # the dense FP64 path (which the error check above covers)
    assert fb.sum() <= (len(QS) if name == "homogeneous_degenerate" else 1), (name, fb, it)


def test_lobpcg_vectors_satisfy_pencil():
    """Returned u solve A u = lambda Omega u of the oracle to FP32 level."""
    cell = cells.config3_cell(5)["cell"]
    M, nb = 5, 10
    h = make(cell, M)
    try:
        w, st, it, fb, vec = lobpcg(h, QS[1:4], nb, vectors=True)
    finally:
        bs.bs_destroy_cell(h)
    oc = mv.OracleCell(cell, M)
    for i, q in enumerate(QS[1:4]):
        if fb[i]:
            continue
        A, Om = oc.pencil(q)
        U = vec[i].astype(np.complex128).T          # n x nb
        lam = w[i] ** 2
        R = A @ U - (Om @ U) * lam[None, :]
        rel = np.linalg.norm(R, axis=0) / (np.linalg.norm(A, 2) * np.linalg.norm(U, axis=0))
        assert rel.max() < 1e-5, rel
        # Omega-orthonormal up to the constant scale of Omega
        G = U.conj().T @ Om @ U
        d = np.real(np.diag(G))
        assert np.allclose(G / d.mean(), np.eye(nb), atol=1e-4)


def test_lobpcg_warm_start_saves_iterations():
    """Starting from the solution's own vectors (plus the cold columns) the
    iteration count drops well below the cold start's, same answers."""
    cell = cells.config3_cell(7)["cell"]
    M, nb = 6, 10
    h = make(cell, M)
    try:
        Q = QS[1:5]
        w0, st0, it0, fb0, vec = lobpcg(h, Q, nb, vectors=True)
        X0 = np.ascontiguousarray(vec[:, :nb, :])
        w1, st1, it1, fb1, _ = lobpcg(h, Q, nb, X0=X0)
    finally:
        bs.bs_destroy_cell(h)
    fl = omega_floor(cell)
    assert omega_rel_err(w1, w0, fl).max() <= TOL
    assert not st1.any()
    # the iteration counts are those of the LOBPCG solve, also where the
    # certificate then sent a wavevector to the dense fallback
    assert it1.max() < it0.min(), (it0, it1, fb0, fb1)


def test_lobpcg_device_pointers_and_chunks():
    """Device tensors in and out; results equal to the host-pointer call."""
    cell = cells.config0()["cell"]
    M, nb = 3, 8
    h = make(cell, M)
    try:
        rng = np.random.default_rng(4)
        Q = rng.uniform(0, 0.5, (40, 2))
        w_h, st_h, it_h, fb_h, _ = lobpcg(h, Q, nb)
        Qd = torch.tensor(Q, device="cuda")
        wd = torch.empty((40, nb), dtype=torch.float64, device="cuda")
        sd = torch.empty(40, dtype=torch.int32, device="cuda")
        itd = torch.empty(40, dtype=torch.int32, device="cuda")
        bs.bs_solve_k_lobpcg(h, Qd, nb, wd, status_out=sd, iters_out=itd)
        torch.cuda.synchronize()
    finally:
        bs.bs_destroy_cell(h)
    assert np.array_equal(wd.cpu().numpy(), w_h)
    assert np.array_equal(itd.cpu().numpy(), it_h)
    assert not sd.cpu().numpy().any()


def test_lobpcg_rejects_bad_arguments():
    cell = cells.config0()["cell"]
    h = make(cell, 3)
    try:
        w = np.empty((1, 13))
        with pytest.raises(bs.BSError) as ei:
            bs.bs_solve_k_lobpcg(h, np.zeros((1, 2)), 13, w)
        assert ei.value.code == bs.BS_EINVAL
        X0 = np.zeros((1, 17, 98), np.complex64)
        with pytest.raises(bs.BSError) as ei:
            bs.bs_solve_k_lobpcg(h, np.zeros((1, 2)), 8, np.empty((1, 8)), X0=X0)
        assert ei.value.code == bs.BS_EINVAL
    finally:
        bs.bs_destroy_cell(h)
    h = bs.bs_create_cell(cell.h1, cell.h2, np.ascontiguousarray(cell.phase, np.uint16),
                          cell.lam.copy(), cell.mu.copy(), cell.rho.copy(), 3, bs.BS_PREC_FP64)
    try:
        bs.bs_assemble(h)
        with pytest.raises(bs.BSError) as ei:
            bs.bs_solve_k_lobpcg(h, np.zeros((1, 2)), 8, np.empty((1, 8)))
        assert ei.value.code == bs.BS_EINVAL
    finally:
        bs.bs_destroy_cell(h)


def test_lobpcg_edge_cases():
    """No wavevectors; a single band; the smallest cell (M = 1, n = 18)."""
    cell = cells.voronoi_cell(8, 3, seed=3)
    h = make(cell, 1)
    try:
        w0 = np.empty((0, 4))
        bs.bs_solve_k_lobpcg(h, np.zeros((0, 2)), 4, w0)          # nk = 0: nothing to do
        Q = QS[:4]
        for nb in (1, 4, 12):                                    # 3b = 48 > n = 18
            w, st, it, fb, _ = lobpcg(h, Q, nb)
            oc = mv.OracleCell(cell, 1)
            ref = np.array([oc.omega(q, nb) for q in Q])
            assert omega_rel_err(w, ref, omega_floor(cell)).max() <= TOL, nb
            assert not st.any()
        with pytest.raises(bs.BSError) as ei:                    # above BS_LOB_MAX_BANDS
            bs.bs_solve_k_lobpcg(h, Q, 13, np.empty((4, 13)))
        assert ei.value.code == bs.BS_EINVAL
    finally:
        bs.bs_destroy_cell(h)


@pytest.mark.slow
def test_lobpcg_largest_truncation():
    """M = 15 (n = 1922, the largest the library takes) on a 64 x 64 Voronoi cell."""
    cell = cells.voronoi_cell(64, 12, seed=77)
    M, nb = 15, 10
    h = make(cell, M)
    try:
        Q = QS[1:3]
        w, st, it, fb, _ = lobpcg(h, Q, nb)
    finally:
        bs.bs_destroy_cell(h)
    assert not st.any()
    oc = mv.OracleCell(cell, M)
    ref = np.array([oc.omega(q, nb) for q in Q])
    assert omega_rel_err(w, ref, omega_floor(cell)).max() <= TOL
