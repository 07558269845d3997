"""The ragged batch of cells (config-3 style: square and hexagonal lattices,
ellipse and Voronoi maps, 2-16 phases, M = 5..8) on the mixed path, through
the C ABI: against single-cell solves, against the oracle, and with the
solve recorded and replayed as a CUDA graph."""
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


def _args(cell, M):
    return (cell.h1, cell.h2, np.ascontiguousarray(cell.phase, np.uint16), cell.lam.copy(),
            cell.mu.copy(), cell.rho.copy(), M, bs.BS_PREC_MIXED)


def _single(cell, M, Q, nb):
    h = bs.bs_create_cell(*_args(cell, M))
    try:
        bs.bs_assemble(h)
        w = np.empty((len(Q), nb))
        bs.bs_solve_k(h, np.ascontiguousarray(Q), nb, w)
    finally:
        bs.bs_destroy_cell(h)
    return w


@pytest.fixture(scope="module")
def small_batch():
    cfgs = [cells.config3_cell(i) for i in range(12)]
    nk, nb = 5, 10
    Qs = np.stack([c["Q"][::6][:nk] for c in cfgs])          # 5 k per cell along its path
    args = [_args(c["cell"], c["M"]) for c in cfgs]
    b = bs.bs_batch_create(args, nk, nb)
    w = np.empty((len(cfgs), nk, nb))
    st = np.empty((len(cfgs), nk), np.int32)
    bs.bs_batch_solve(b, np.ascontiguousarray(Qs), w, st)
    tiles = bs.bs_batch_tiles(b)
    yield cfgs, Qs, w, st, b, tiles
    bs.bs_batch_destroy(b)


def test_batch_matches_single_cells(small_batch):
    cfgs, Qs, w, st, _, tiles = small_batch
    assert not st.any()
    assert set(tiles.values()) <= {32, 64} and len(tiles) >= 2   # ragged: several truncations
    for i, c in enumerate(cfgs):
        ref = _single(c["cell"], c["M"], Qs[i], w.shape[2])
        assert omega_rel_err(w[i], ref, omega_floor(c["cell"])).max() <= TOL, i


def test_batch_matches_oracle(small_batch):
    cfgs, Qs, w, _, _, _ = small_batch
    for i in (0, 5, 11):
        c = cfgs[i]
        oc = mv.OracleCell(c["cell"], c["M"])
        ref = np.array([oc.omega(q, w.shape[2]) for q in Qs[i]])
        assert omega_rel_err(w[i], ref, omega_floor(c["cell"])).max() <= TOL, i


def test_batch_graph_replay(small_batch):
    cfgs, Qs, w, _, b, _ = small_batch
    Qd = torch.tensor(Qs, device="cuda")
    wd = torch.empty(w.shape, dtype=torch.float64, device="cuda")
    sd = torch.empty(w.shape[:2], dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream()
    bs.bs_batch_set_graph(b, True)
    try:
        for _ in range(2):                       # record, then replay
            wd.zero_()
            bs.bs_batch_solve(b, Qd, wd, sd, s)
            s.synchronize()
            assert np.array_equal(wd.cpu().numpy(), w)
            assert not sd.cpu().numpy().any()
    finally:
        bs.bs_batch_set_graph(b, False)


def test_batch_rejects_mixed_grids_and_fp64():
    a = cells.config3_cell(0)
    b64 = cells.circle_cell(32)
    with pytest.raises(bs.BSError) as ei:
        bs.bs_batch_create([_args(a["cell"], a["M"]), _args(b64, 3)], 2, 4)
    assert ei.value.code == bs.BS_EINVAL and "same P" in str(ei.value)
    fp64 = list(_args(a["cell"], a["M"]))
    fp64[-1] = bs.BS_PREC_FP64
    with pytest.raises(bs.BSError):
        bs.bs_batch_create([tuple(fp64)], 2, 4)


def test_batch_tile_edges_agree():
    """Both tile edges of the per-step FP32 reduction (32 and 64) give the
    same certified bands on every (cell, k); other tile values are refused."""
    cfgs = [cells.config3_cell(i) for i in range(20, 28)]
    nk, nb = 6, 10
    Qs = np.ascontiguousarray(np.stack([c["Q"][::5][:nk] for c in cfgs]))
    b = bs.bs_batch_create([_args(c["cell"], c["M"]) for c in cfgs], nk, nb)
    try:
        with pytest.raises(bs.BSError) as ei:
            bs.bs_batch_set_tile(b, 0)
        assert ei.value.code == bs.BS_EINVAL
        out = {}
        for tile in (32, 64):
            bs.bs_batch_set_tile(b, tile)
            w = np.empty((len(cfgs), nk, nb))
            st = np.empty((len(cfgs), nk), np.int32)
            bs.bs_batch_solve(b, Qs, w, st)
            _, fb = bs.bs_batch_stats(b, len(cfgs) * nk)
            out[tile] = (w, st, fb, bs.bs_batch_tiles(b))
    finally:
        bs.bs_batch_destroy(b)
    assert set(out[32][3].values()) == {32} and set(out[64][3].values()) == {64}
    for i, c in enumerate(cfgs):
        assert omega_rel_err(out[32][0][i], out[64][0][i], omega_floor(c["cell"])).max() <= 2 * TOL
    assert not out[32][1].any() and not out[64][1].any()


def test_batch_fp64_solver_matches_single_cell_fp64():
    """BS_SOLVER_FP64 runs the plain FP64 path of bs_solve_k for every
    (cell, k) of a chunk at once: the same numbers as single-cell FP64 solves
    to the rounding of two FP64 evaluation orders, and the oracle to 1e-8.

    A single cell inverts its Gram factors by doubling, a batch of many cells
    diagonal by diagonal; the two inverses differ by a few n eps, which moves
    the eigenvalues by about n eps ||C||.  At the acoustic zero modes of Gamma
    that is ~1e-13 ||C|| against the floor squared (||C|| / floor^2 ~ 60
    here), hence 1e-10 on the floored relative error."""
    cfgs = [cells.config3_cell(i) for i in range(30, 36)]
    nk, nb = 4, 10
    Qs = np.ascontiguousarray(np.stack([c["Q"][::7][:nk] for c in cfgs]))
    b = bs.bs_batch_create([_args(c["cell"], c["M"]) for c in cfgs], nk, nb)
    try:
        bs.bs_batch_set_solver(b, bs.BS_SOLVER_FP64)
        w = np.empty((len(cfgs), nk, nb))
        st = np.empty((len(cfgs), nk), np.int32)
        bs.bs_batch_solve(b, Qs, w, st)
    finally:
        bs.bs_batch_destroy(b)
    assert not st.any()
    for i, c in enumerate(cfgs):
        h = bs.bs_create_cell(*(_args(c["cell"], c["M"])[:-1] + (bs.BS_PREC_FP64,)))
        try:
            bs.bs_assemble(h)
            ref = np.empty((nk, nb))
            bs.bs_solve_k(h, np.ascontiguousarray(Qs[i]), nb, ref)
        finally:
            bs.bs_destroy_cell(h)
        assert omega_rel_err(w[i], ref, omega_floor(c["cell"])).max() <= 1e-10, i
    oc = mv.OracleCell(cfgs[0]["cell"], cfgs[0]["M"])
    ref = np.array([oc.omega(q, nb) for q in Qs[0]])
    assert omega_rel_err(w[0], ref, omega_floor(cfgs[0]["cell"])).max() <= 1e-8
