"""The two-stage reduction of the FP64 path (dense -> band on the tensor
cores, band -> tridiagonal by bulge chasing), called through the C ABI.

Both reductions are unitary similarities of the same C(k), so the two-stage
frequencies must match the oracle to the FP64 path's tolerance (1e-8
relative, on omega^2 with the acoustic floor) and the one-stage reduction
to 1e-9 (both FP64; the difference is the rounding of the two reductions
and of the exact-slice products, a few 2^-53 of the matrix norm, which at
the acoustic zero modes of Gamma is seen against the floor).
"""
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

TOL_W = 1e-8
TOL_PATHS = 1e-9


@pytest.fixture(autouse=True)
def restore_reduction():
    yield
    bs.bs_set_reduction(bs.BS_REDUCE_AUTO)


def solve(cell, M, Q, nb, mode):
    bs.bs_set_reduction(mode)
    h = bs.bs_create_cell(cell.h1, cell.h2, np.ascontiguousarray(cell.phase, np.uint16),
                          cell.lam.copy(), cell.mu.copy(), cell.rho.copy(), M, bs.BS_PREC_FP64)
    try:
        bs.bs_assemble(h)
        Q = np.ascontiguousarray(Q, np.float64).reshape(-1, 2)
        n = bs.bs_cell_dims(h)[1]
        nb = min(nb, n)
        w = np.empty((len(Q), nb))
        st = np.empty(len(Q), np.int32)
        bs.bs_solve_k(h, Q, nb, w, st)
        assert not st.any()
    finally:
        bs.bs_destroy_cell(h)
    return w


CASES = [
    # name, cell, M: n = 2 (2M+1)^2 from 2 (no band step, the bulge chase
    # alone) through panels that end in a partial one and band ragged tails
    ("single_wave", lambda: cells.circle_cell(4, 0.3), 0),            # n = 2
    ("tiny_exact_grid", lambda: cells.voronoi_cell(5, 3, seed=4), 1), # n = 18
    ("c0_circle", lambda: cells.config0()["cell"], 3),                # n = 98
    ("hex_voronoi", lambda: cells.voronoi_cell(48, 9, seed=21, lattice="hex"), 5),   # n = 242
    ("square_voronoi_m7", lambda: cells.voronoi_cell(40, 12, seed=5), 7),            # n = 450
]


@pytest.mark.parametrize("name, make, M", CASES)
def test_two_stage_against_oracle_and_one_stage(name, make, M):
    cell = make()
    Q = np.array([[0.0, 0.0], [0.31, 0.17], [0.5, 0.0], [0.5, 0.5]])
    nb = 10
    w2 = solve(cell, M, Q, nb, bs.BS_REDUCE_TWOSTAGE)
    w1 = solve(cell, M, Q, nb, bs.BS_REDUCE_ONESTAGE)
    fl = omega_floor(cell)
    assert omega_rel_err(w2, w1, fl).max() <= TOL_PATHS, name
    oc = mv.OracleCell(cell, M)
    for i in (1, 3):
        ref = oc.omega(Q[i], w2.shape[1])
        assert omega_rel_err(w2[i], ref, fl).max() <= TOL_W, (name, i)
    assert np.all(np.diff(w2, axis=1) >= 0)


@pytest.mark.parametrize("name, make, M", CASES[1:4])
def test_two_stage_whole_spectrum(name, make, M):
    """nbands = n: every eigenvalue survives the band and bulge stages."""
    cell = make()
    Q = np.array([0.3, 0.1])
    w = solve(cell, M, Q, 10 ** 6, bs.BS_REDUCE_TWOSTAGE)[0]
    ref = mv.OracleCell(cell, M).omega(Q)
    assert omega_rel_err(w, ref, omega_floor(cell)).max() <= TOL_W


def test_two_stage_c1_full_size():
    """Config 1 at full size (n = 882, all 90 k in one batch, as the
    benchmark solves it): every wavevector against the one-stage reduction,
    sampled ones against the oracle."""
    cfg = cells.config1()
    w2 = solve(cfg["cell"], cfg["M"], cfg["Q"], cfg["nbands"], bs.BS_REDUCE_TWOSTAGE)
    w1 = solve(cfg["cell"], cfg["M"], cfg["Q"], cfg["nbands"], bs.BS_REDUCE_ONESTAGE)
    fl = omega_floor(cfg["cell"])
    assert omega_rel_err(w2, w1, fl).max() <= TOL_PATHS
    oc = mv.OracleCell(cfg["cell"], cfg["M"])
    for i in (0, 30, 61, 89):
        ref = oc.omega(cfg["Q"][i], cfg["nbands"])
        assert omega_rel_err(w2[i], ref, fl).max() <= TOL_W, i


def test_set_reduction_rejects_unknown_mode():
    with pytest.raises(bs.BSError):
        bs.bs_set_reduction(7)


# ---- the other FP64 solvers that take the two-stage reduction, forced on
# small cells (BS_REDUCE_AUTO takes it from n = 400 on, where the tests
# above and the benches reach it)

def _aniso_cell():
    return cells.anisotropic_cell(cells.voronoi_cell(24, 6, seed=8, lattice="hex"), seed=3)


def _solve_aniso(cell, M, Q, nb, mode):
    bs.bs_set_reduction(mode)
    C = cell.stiffness
    c6 = np.ascontiguousarray(np.stack([C[:, 0, 0], C[:, 1, 1], C[:, 0, 1], C[:, 0, 2],
                                        C[:, 1, 2], C[:, 2, 2]], axis=1))
    h = bs.bs_create_cell(cell.h1, cell.h2, np.ascontiguousarray(cell.phase, np.uint16),
                          cell.lam.copy(), cell.mu.copy(), cell.rho.copy(), M, bs.BS_PREC_FP64)
    try:
        bs.bs_set_stiffness(h, c6)
        bs.bs_assemble(h)
        w = np.empty((len(Q), nb))
        st = np.empty(len(Q), np.int32)
        bs.bs_solve_k(h, np.ascontiguousarray(Q), nb, w, st)
        assert not st.any()
    finally:
        bs.bs_destroy_cell(h)
    return w


def test_two_stage_anisotropic_cell():
    cell, M, nb = _aniso_cell(), 4, 10                     # n = 162
    Q = np.array([[0.21, 0.07], [2 / 3, 1 / 3]])
    w2 = _solve_aniso(cell, M, Q, nb, bs.BS_REDUCE_TWOSTAGE)
    w1 = _solve_aniso(cell, M, Q, nb, bs.BS_REDUCE_ONESTAGE)
    fl = omega_floor(cell)
    assert omega_rel_err(w2, w1, fl).max() <= TOL_PATHS
    oc = mv.OracleCell(cell, M)
    for i in range(len(Q)):
        assert omega_rel_err(w2[i], oc.omega(Q[i], nb), fl).max() <= TOL_W


def _solve3(cell, M, Q, nb, mode):
    bs.bs_set_reduction(mode)
    h = bs.bs_create_cell3(cell.h1, cell.h2, cell.h3, np.ascontiguousarray(cell.phase, np.uint16),
                           cell.lam.copy(), cell.mu.copy(), cell.rho.copy(), M)
    try:
        bs.bs_assemble3(h)
        w = np.empty((len(Q), nb))
        st = np.empty(len(Q), np.int32)
        bs.bs_solve_k3(h, np.ascontiguousarray(Q), nb, w, st)
        assert not st.any()
    finally:
        bs.bs_destroy_cell3(h)
    return w


def test_two_stage_3d_cell():
    from oracle import mixed_variational_3d as mv3
    cell, M, nb = cells.sphere_cell3(8, 0.3), 2, 12         # n = 375
    Q = np.array([[0.21, 0.07, -0.13], [0.5, 0.5, 0.5]])
    w2 = _solve3(cell, M, Q, nb, bs.BS_REDUCE_TWOSTAGE)
    w1 = _solve3(cell, M, Q, nb, bs.BS_REDUCE_ONESTAGE)
    A = np.array([cell.h1, cell.h2, cell.h3])
    qm = 2 * np.pi * np.linalg.inv(A)
    fl = np.sqrt(np.min(cell.mu / cell.rho)) * min(np.linalg.norm(qm[:, i]) for i in range(3)) / 2
    assert omega_rel_err(w2, w1, fl).max() <= TOL_PATHS
    oc = mv3.OracleCell3(cell, M)
    for i in range(len(Q)):
        assert omega_rel_err(w2[i], oc.omega(Q[i], nb), fl).max() <= TOL_W


def test_two_stage_batch_fp64_solver():
    """BS_SOLVER_FP64 of a ragged batch (two truncation groups, M = 6 and 7,
    n = 338 and 450) with the two-stage reduction forced, against single-cell
    one-stage solves."""
    cfgs = [cells.config3_cell(i) for i in range(40, 44)]
    nk, nb = 3, 10
    Qs = np.ascontiguousarray(np.stack([c["Q"][::9][:nk] for c in cfgs]))
    args = lambda c, p: (c["cell"].h1, c["cell"].h2,
                         np.ascontiguousarray(c["cell"].phase, np.uint16), c["cell"].lam.copy(),
                         c["cell"].mu.copy(), c["cell"].rho.copy(), c["M"], p)
    bs.bs_set_reduction(bs.BS_REDUCE_TWOSTAGE)
    b = bs.bs_batch_create([args(c, bs.BS_PREC_MIXED) for c in cfgs], nk, nb)
    try:
        bs.bs_batch_set_solver(b, bs.BS_SOLVER_FP64)
        w = np.empty((len(cfgs), nk, nb))
        st = np.empty((len(cfgs), nk), np.int32)
        bs.bs_batch_solve(b, Qs, w, st)
    finally:
        bs.bs_batch_destroy(b)
    assert not st.any()
    for i, c in enumerate(cfgs):
        ref = solve(c["cell"], c["M"], Qs[i], nb, bs.BS_REDUCE_ONESTAGE)
        assert omega_rel_err(w[i], ref, omega_floor(c["cell"])).max() <= TOL_PATHS, i


def test_two_stage_mesh_cell():
    m, M, nb = cells.mesh_voronoi_cell(16, 8, seed=4, lattice="hex"), 3, 10   # n = 98
    Q = np.array([[0.21, 0.07], [0.5, 0.0]])
    out = {}
    for mode in (bs.BS_REDUCE_TWOSTAGE, bs.BS_REDUCE_ONESTAGE):
        bs.bs_set_reduction(mode)
        h = bs.bs_create_cell_mesh(m.h1, m.h2, np.ascontiguousarray(m.centroid),
                                   np.ascontiguousarray(m.area),
                                   np.ascontiguousarray(m.phase, np.uint16), m.lam.copy(),
                                   m.mu.copy(), m.rho.copy(), M, bs.BS_PREC_FP64)
        try:
            bs.bs_assemble(h)
            w = np.empty((len(Q), nb))
            st = np.empty(len(Q), np.int32)
            bs.bs_solve_k(h, np.ascontiguousarray(Q), nb, w, st)
            assert not st.any()
        finally:
            bs.bs_destroy_cell(h)
        out[mode] = w
    fl = omega_floor(m)
    assert omega_rel_err(out[bs.BS_REDUCE_TWOSTAGE], out[bs.BS_REDUCE_ONESTAGE],
                         fl).max() <= TOL_PATHS
