"""Bitwise reproducibility of the ragged batch on the iterative path.

Identical inputs must give identical results: every (cell, k) of a batch
of held-out cells is solved by block LOBPCG (from the trained network's
starting subspaces and from the cold start) several times, each time in a
freshly created batch, and omega, the status, the iteration counts and the
fallback flags must agree bit for bit.  The cells are assembled on 16
worker streams at once, so this also guards the blocked factorisations
(Cholesky of the Gram matrices, LDL of the count certificate) against
races between the CTAs of one launch.
"""
import json
import os

import numpy as np
import pytest

from paper_1310_6380_gb300 import cells, warmstart as ws

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1310_6380_gb300 import binding as bs  # noqa: E402

WEIGHTS = os.path.join(os.path.dirname(ws.__file__), "data", "warmstart.npz")
REPEATS = 5


@pytest.fixture(scope="module")
def held_out():
    saved = np.load(WEIGHTS)
    meta = json.loads(str(saved["meta"]))
    cfgs = [cells.config4_eval_cell(i) for i in range(1100, 1164)]
    cl = [c["cell"] for c in cfgs]
    Ms = [c["M"] for c in cfgs]
    Q = np.ascontiguousarray(np.stack([c["Q"] for c in cfgs]))
    net = ws.WarmStartNet(meta["nvec"], meta["Mp"], max_cells=64, max_samples=64 * 30)
    try:
        net.set_params(saved["params"])
        U = net.predict(ws.CellPack(cl), Q)
    finally:
        net.close()
    return cl, Ms, Q, U, meta["Mp"]


@pytest.mark.parametrize("warm", [True, False])
def test_lobpcg_batch_is_bitwise_reproducible(held_out, warm):
    cl, Ms, Q, U, Mp = held_out
    runs = [ws.solve_batch(cl, Ms, Q, 10, bs.BS_SOLVER_LOBPCG, start=U if warm else None, Mp=Mp)
            for _ in range(REPEATS)]
    w0, st0, it0, fb0, _ = runs[0]
    assert not st0.any()
    for r, (w, st, it, fb, _) in enumerate(runs[1:], 1):
        diff = sorted(set(np.argwhere((w != w0).any(-1))[:, 0].tolist()))
        assert np.array_equal(w, w0), f"run {r}: omega differs in cells {diff}"
        assert np.array_equal(st, st0) and np.array_equal(it, it0) and np.array_equal(fb, fb0), r


def test_dense_mixed_batch_is_bitwise_reproducible():
    """The dense mixed batch (FP32 reduction + FP64 refinement) on the same
    cells, with the reduction tile fixed (the autotuner may pick either
    edge, and the two round differently): bitwise equal over repeated
    solves in fresh batches."""
    cfgs = [cells.config3_cell(i) for i in range(200, 248)]
    args = [(c["cell"].h1, c["cell"].h2, np.ascontiguousarray(c["cell"].phase, np.uint16),
             c["cell"].lam.copy(), c["cell"].mu.copy(), c["cell"].rho.copy(), c["M"],
             bs.BS_PREC_MIXED) for c in cfgs]
    Q = np.ascontiguousarray(np.stack([c["Q"][::3] for c in cfgs]))
    out = []
    for _ in range(3):
        b = bs.bs_batch_create(args, Q.shape[1], 10)
        try:
            bs.bs_batch_set_tile(b, 64)
            w = np.empty((len(cfgs), Q.shape[1], 10))
            st = np.empty((len(cfgs), Q.shape[1]), np.int32)
            bs.bs_batch_solve(b, Q, w, st)
        finally:
            bs.bs_batch_destroy(b)
        out.append((w, st))
    assert not out[0][1].any()
    for w, st in out[1:]:
        assert np.array_equal(w, out[0][0]) and np.array_equal(st, out[0][1])
