"""Mixed-precision path (FP32 reduction + FP64 Rayleigh-Ritz) against the
FP64 oracle and against the FP64 GPU path: relative frequency error
<= 1e-6 (measured on omega^2 with the acoustic floor)."""
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


def solve(cell, M, Q, nb, precision):
    h = bs.bs_create_cell(cell.h1, cell.h2, np.ascontiguousarray(cell.phase, np.uint16),
                          cell.lam.copy(), cell.mu.copy(), cell.rho.copy(), M, precision)
    try:
        bs.bs_assemble(h)
        Q = np.ascontiguousarray(Q, np.float64).reshape(-1, 2)
        w = np.empty((len(Q), nb))
        st = np.empty(len(Q), np.int32)
        bs.bs_solve_k(h, Q, nb, w, st)
    finally:
        bs.bs_destroy_cell(h)
    return w, st


@pytest.mark.parametrize("name, make, M, nb", [
    ("c0_circle", lambda: cells.config0()["cell"], 3, 8),
    ("hex_voronoi", lambda: cells.voronoi_cell(48, 9, seed=21, lattice="hex"), 5, 12),
    ("homogeneous_degenerate", lambda: cells.homogeneous_cell(12, 4.0, 1.5, 1.2), 3, 16),
    ("small_n", lambda: cells.voronoi_cell(8, 3, seed=3), 1, 10),      # n = 18
])
def test_mixed_matches_oracle(name, make, M, nb):
    cell = make()
    Q = np.array([[0.0, 0.0], [0.21, 0.07], [0.5, 0.0], [0.5, 0.5], [0.33, 0.29]])
    w, st = solve(cell, M, Q, nb, bs.BS_PREC_MIXED)
    oc = mv.OracleCell(cell, M)
    ref = np.array([oc.omega(q, nb) for q in Q])
    err = omega_rel_err(w, ref, omega_floor(cell))
    assert err.max() <= TOL, (name, err.max())
    assert not st.any(), st


@pytest.mark.slow
def test_mixed_c2_full_size():
    """Config 2: the config-1 cell on the mixed path, all 90 k in one batch;
    every k against the FP64 GPU path, sampled k against the oracle."""
    cfg = cells.config1()
    cell, M, Q, nb = cfg["cell"], cfg["M"], cfg["Q"], cfg["nbands"]
    wm, st = solve(cell, M, Q, nb, bs.BS_PREC_MIXED)
    w64, _ = solve(cell, M, Q, nb, bs.BS_PREC_FP64)
    fl = omega_floor(cell)
    assert omega_rel_err(wm, w64, fl).max() <= TOL
    assert not st.any()
    oc = mv.OracleCell(cell, M)
    for i in (0, 30, 61, 89):
        assert omega_rel_err(wm[i], oc.omega(Q[i], nb), fl).max() <= TOL, i


def test_mixed_band_limit():
    cell = cells.config0()["cell"]
    with pytest.raises(bs.BSError) as ei:
        solve(cell, 3, np.zeros((1, 2)), 25, bs.BS_PREC_MIXED)
    assert ei.value.code == bs.BS_EINVAL
