"""The iteration caps of the iterative steps run out: the solvers return
(without hanging) with the per-wavevector status and fallback flags set.

The caps are lowered with bs_set_iteration_limits (a process-wide test and
diagnostic setting) and restored afterwards:
  * LOBPCG capped at one iteration: no wavevector can be certified from its
    FP32 iterations, so every one goes to the dense fallback (single cell:
    the dense FP64 path; batch: the dense mixed rescue), and the bands still
    match the plain FP64 path;
  * the Sturm bisection capped at one sweep: its brackets cannot reach FP64
    accuracy, so the FP64 path reports BS_ENOCONV for every wavevector, as
    does the single-cell LOBPCG path whose fallback is that FP64 path.
"""
import numpy as np
import pytest

from paper_1310_6380_gb300 import cells

from _helpers import omega_floor, omega_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1310_6380_gb300 import binding as bs  # noqa: E402

NB = 10


@pytest.fixture
def caps():
    yield bs.bs_set_iteration_limits
    bs.bs_set_iteration_limits(0, 0)


def _cell(i):
    c = cells.config3_cell(i)
    cl = c["cell"]
    return c, (cl.h1, cl.h2, np.ascontiguousarray(cl.phase, np.uint16), cl.lam.copy(),
               cl.mu.copy(), cl.rho.copy(), c["M"])


def _fp64_reference(args, Q):
    h = bs.bs_create_cell(*args, bs.BS_PREC_FP64)
    try:
        bs.bs_assemble(h)
        w = np.empty((len(Q), NB))
        bs.bs_solve_k(h, Q, NB, w)
    finally:
        bs.bs_destroy_cell(h)
    return w


def test_limits_are_validated(caps):
    for bad in ((1001, 0), (0, 129)):
        with pytest.raises(bs.BSError) as ei:
            caps(*bad)
        assert ei.value.code == bs.BS_EINVAL


def test_lobpcg_cap_sends_every_wavevector_to_the_fallback(caps):
    c, args = _cell(5)
    Q = np.ascontiguousarray(c["Q"][1:7])
    ref = _fp64_reference(args, Q)
    caps(1, 0)
    h = bs.bs_create_cell(*args, bs.BS_PREC_MIXED)
    try:
        bs.bs_assemble(h)
        w = np.empty((len(Q), NB))
        st = np.empty(len(Q), np.int32)
        it = np.empty(len(Q), np.int32)
        fb = np.empty(len(Q), np.int32)
        bs.bs_solve_k_lobpcg(h, Q, NB, w, status_out=st, iters_out=it, fallback_out=fb)
    finally:
        bs.bs_destroy_cell(h)
    assert (it <= 1).all(), it
    assert fb.all(), fb
    assert not st.any(), st
    assert omega_rel_err(w, ref, omega_floor(c["cell"])).max() <= 1e-8


def test_lobpcg_cap_in_a_batch_goes_to_the_rescue(caps):
    sel = [_cell(i) for i in range(8, 14)]
    Q = np.ascontiguousarray(np.stack([c["Q"][::6][:5] for c, _ in sel]))
    caps(1, 0)
    b = bs.bs_batch_create([a + (bs.BS_PREC_MIXED,) for _, a in sel], Q.shape[1], NB)
    try:
        bs.bs_batch_set_solver(b, bs.BS_SOLVER_LOBPCG)
        w = np.empty((len(sel), Q.shape[1], NB))
        st = np.empty((len(sel), Q.shape[1]), np.int32)
        bs.bs_batch_solve(b, Q, w, st)
        it, fb = bs.bs_batch_stats(b, w.shape[0] * w.shape[1])
    finally:
        bs.bs_batch_destroy(b)
    assert (it <= 1).all(), it
    assert (fb > 0).all(), fb
    assert not st.any(), st
    for i, (c, a) in enumerate(sel):
        ref = _fp64_reference(a, np.ascontiguousarray(Q[i]))
        assert omega_rel_err(w[i], ref, omega_floor(c["cell"])).max() <= 1e-6, i


def test_bisection_cap_reports_no_convergence(caps):
    c, args = _cell(5)
    Q = np.ascontiguousarray(c["Q"][1:5])
    caps(0, 1)
    h = bs.bs_create_cell(*args, bs.BS_PREC_FP64)
    try:
        bs.bs_assemble(h)
        w = np.empty((len(Q), NB))
        st = np.empty(len(Q), np.int32)
        with pytest.raises(bs.BSError) as ei:
            bs.bs_solve_k(h, Q, NB, w)
        assert ei.value.code == bs.BS_ENOCONV
        with pytest.raises(bs.BSError) as ei:
            bs.bs_solve_k(h, Q, NB, w, st)
        assert ei.value.code == bs.BS_ENOCONV
        assert (st == bs.BS_ENOCONV).all(), st
    finally:
        bs.bs_destroy_cell(h)
    # the LOBPCG path with both caps low: its FP64 fallback cannot converge either
    caps(1, 1)
    h = bs.bs_create_cell(*args, bs.BS_PREC_MIXED)
    try:
        bs.bs_assemble(h)
        st = np.empty(len(Q), np.int32)
        fb = np.empty(len(Q), np.int32)
        bs.bs_solve_k_lobpcg(h, Q, NB, w, status_out=st, fallback_out=fb)
        assert fb.all() and (st == bs.BS_ENOCONV).all(), (st, fb)
    finally:
        bs.bs_destroy_cell(h)
