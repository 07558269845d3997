"""Parity of the CUDA path (called through the C ABI) with the FP64 oracle.

Tolerances (FP64 path): form factors 1e-13 of their largest magnitude;
reduced matrix 1e-11 of its largest entry; frequencies 1e-8 relative
(measured on omega^2 with the acoustic floor, see _helpers.omega_rel_err).
"""
import numpy as np
import pytest

from oracle import mixed_variational as mv
from paper_1310_6380_gb300 import cells

from _helpers import field_tables, omega_floor, omega_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1310_6380_gb300 import binding as bs  # noqa: E402

TOL_W = 1e-8


class GpuCell:
    def __init__(self, cell, M, precision=bs.BS_PREC_FP64, assemble=True):
        self.cell, self.M = cell, M
        self.h = bs.bs_create_cell(cell.h1, cell.h2, np.ascontiguousarray(cell.phase, np.uint16),
                                   cell.lam.copy(), cell.mu.copy(), cell.rho.copy(), M, precision)
        self.N, self.n = bs.bs_cell_dims(self.h)
        if assemble:
            bs.bs_assemble(self.h)
            bs.bs_sync(self.h)

    def omega(self, Q, nb):
        Q = np.ascontiguousarray(Q, np.float64).reshape(-1, 2)
        w = np.empty((len(Q), nb))
        st = np.empty(len(Q), np.int32)
        bs.bs_solve_k(self.h, Q, nb, w, st)
        assert not st.any()
        return w

    def close(self):
        bs.bs_destroy_cell(self.h)


@pytest.fixture(scope="module")
def c0():
    cfg = cells.config0()
    g = GpuCell(cfg["cell"], cfg["M"])
    yield cfg, g
    g.close()


CASES = [
    ("c0_circle", lambda: cells.config0()["cell"], 3),
    ("hex_voronoi_ragged", lambda: cells.voronoi_cell(48, 9, seed=21, lattice="hex"), 5),
    ("tiny_exact_grid", lambda: cells.voronoi_cell(5, 3, seed=4), 2),      # P = 2M+1
    ("single_wave", lambda: cells.circle_cell(4, 0.3), 0),                 # M = 0, n = 2
]


@pytest.mark.parametrize("name, make, M", CASES)
def test_form_factors(name, make, M):
    cell = make()
    g = GpuCell(cell, M)
    D = 4 * M + 1
    out = np.empty(3 * D * D * 2)
    bs.bs_form_factors(g.h, out)
    g.close()
    got = out.view(np.complex128).reshape(3, D, D)
    x, w = mv.quadrature(cell)
    ref = mv.form_factors(field_tables(cell), x, w, cell.h1, cell.h2, M)
    for f in range(3):
        assert np.abs(got[f] - ref[f]).max() <= 1e-13 * np.abs(ref[f]).max(), (name, f)


@pytest.mark.parametrize("name, make, M", CASES)
def test_reduced_matrix(name, make, M):
    """C(k) = L^-1 A L^-dagger with L the Cholesky factor of Omega."""
    cell = make()
    g = GpuCell(cell, M)
    oc = mv.OracleCell(cell, M)
    for Q in ([0.21, -0.13], [0.0, 0.0], [0.5, 0.5]):
        Q = np.array(Q)
        out = np.empty(g.n * g.n * 2)
        bs.bs_reduced_matrix(g.h, Q, out)
        got = out.view(np.complex128).reshape(g.n, g.n).T      # column-major -> [r, c]
        A, Om = oc.pencil(Q)
        L = np.linalg.cholesky(Om)
        Li = np.linalg.inv(L)
        ref = Li @ A @ Li.conj().T
        low = np.tril_indices(g.n)
        assert np.abs(got[low] - ref[low]).max() <= 1e-11 * np.abs(ref).max(), (name, Q)
    g.close()


def test_c0_bands_full(c0):
    """Config 0 end to end: 30 k on G-X-M-G, 8 branches, FP64."""
    cfg, g = c0
    w = g.omega(cfg["Q"], cfg["nbands"])
    ref = mv.bands(cfg["cell"], cfg["M"], cfg["Q"], cfg["nbands"])
    err = omega_rel_err(w, ref, omega_floor(cfg["cell"]))
    assert err.max() <= TOL_W, err.max()


@pytest.mark.parametrize("name, make, M", CASES[1:])
def test_all_eigenvalues(name, make, M):
    """nbands = n: the whole spectrum, checked against the oracle."""
    cell = make()
    g = GpuCell(cell, M)
    Q = np.array([0.3, 0.1])
    w = g.omega(Q, g.n)[0]
    g.close()
    ref = mv.OracleCell(cell, M).omega(Q)
    assert omega_rel_err(w, ref, omega_floor(cell)).max() <= TOL_W


def test_homogeneous_closed_form():
    """The GPU path folds the free dispersion of a homogeneous cell."""
    cell = cells.homogeneous_cell(12, 4.0, 1.5, 1.2, lattice="hex", a=1.3)
    M = 3
    g = GpuCell(cell, M)
    Q = np.array([0.2, 0.1])
    w = g.omega(Q, g.n)[0]
    g.close()
    K = mv.wavevectors(Q, cell.h1, cell.h2, M)
    k2 = np.sum(K ** 2, axis=1)
    ref = np.sqrt(np.sort(np.concatenate([(4.0 + 3.0) / 1.2 * k2, 1.5 / 1.2 * k2])))
    assert omega_rel_err(w, ref, omega_floor(cell)).max() <= TOL_W


def test_gamma_and_time_reversal(c0):
    cfg, g = c0
    w = g.omega(np.array([[0.0, 0.0], [0.31, 0.17], [-0.31, -0.17]]), 4)
    assert w[0, 0] < 1e-3 and w[0, 1] < 1e-3 and w[0, 2] > 1.0
    assert omega_rel_err(w[1], w[2], omega_floor(cfg["cell"])).max() <= TOL_W


def test_edge_counts(c0):
    cfg, g = c0
    empty = np.empty((0, 8))
    bs.bs_solve_k(g.h, np.empty((0, 2)), 8, empty)       # nk = 0 is a no-op
    with pytest.raises(bs.BSError) as ei:
        g.omega(np.zeros(2), g.n + 1)
    assert ei.value.code == bs.BS_EINVAL
    one = g.omega(np.array([0.1, 0.0]), 1)
    assert one.shape == (1, 1) and one[0, 0] > 0


def test_solve_before_assemble():
    cell = cells.circle_cell(8, 0.3)
    g = GpuCell(cell, 2, assemble=False)
    with pytest.raises(bs.BSError) as ei:
        g.omega(np.zeros(2), 2)
    g.close()
    assert ei.value.code == bs.BS_ESTATE


def test_k_chunking():
    """More wavevectors than one k batch holds (4096): chunks agree."""
    cell = cells.voronoi_cell(8, 4, seed=7)
    g = GpuCell(cell, 1)
    rng = np.random.default_rng(0)
    Q = rng.uniform(-0.5, 0.5, (4100, 2))
    w = g.omega(Q, 6)
    g.close()
    oc = mv.OracleCell(cell, 1)
    for i in (0, 4095, 4096, 4099):
        ref = oc.omega(Q[i], 6)
        assert omega_rel_err(w[i], ref, omega_floor(cell)).max() <= TOL_W


def test_device_pointers_match_host(c0):
    cfg, g = c0
    Qd = torch.tensor(cfg["Q"], dtype=torch.float64, device="cuda")
    wd = torch.empty((len(cfg["Q"]), 8), dtype=torch.float64, device="cuda")
    sd = torch.empty(len(cfg["Q"]), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    bs.bs_solve_k(g.h, Qd, 8, wd, sd, stream=stream)
    stream.synchronize()
    wh = g.omega(cfg["Q"], 8)
    assert np.array_equal(wd.cpu().numpy(), wh)
    assert not sd.cpu().numpy().any()


def test_device_resident_cell_inputs():
    cell = cells.config0()["cell"]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    h = bs.bs_create_cell(cell.h1, cell.h2, dev(cell.phase.astype(np.uint16)), dev(cell.lam),
                          dev(cell.mu), dev(cell.rho), 3)
    bs.bs_assemble(h)
    w = np.empty((1, 8))
    bs.bs_solve_k(h, np.array([[0.25, 0.0]]), 8, w)
    bs.bs_destroy_cell(h)
    g = GpuCell(cell, 3)
    ref = g.omega(np.array([0.25, 0.0]), 8)
    g.close()
    assert np.array_equal(w, ref)


@pytest.mark.parametrize("lattice, path", [("square", 0), ("hex", 1)])
def test_bands_path(lattice, path):
    cell = cells.voronoi_cell(16, 5, seed=2, lattice=lattice)
    g = GpuCell(cell, 2)
    nk = 17
    Qo = np.empty((nk, 2))
    wo = np.empty((nk, 6))
    bs.bs_bands(g.h, path, nk, 6, Qo, wo)
    g.close()
    Qr = cells.ibz_path(lattice, nk, cell.h1, cell.h2)
    assert np.allclose(Qo, Qr, atol=1e-14)
    ref = mv.bands(cell, 2, Qr, 6)
    assert omega_rel_err(wo, ref, omega_floor(cell)).max() <= TOL_W


@pytest.mark.slow
def test_c1_full_size_sampled():
    """Config 1 at full size, solved as the benchmark solves it (all 90 k in
    one batch); sampled wavevectors checked against the oracle one by one."""
    cfg = cells.config1()
    g = GpuCell(cfg["cell"], cfg["M"])
    w = g.omega(cfg["Q"], cfg["nbands"])
    g.close()
    oc = mv.OracleCell(cfg["cell"], cfg["M"])
    fl = omega_floor(cfg["cell"])
    for i in (0, 17, 30, 44, 61, 89):
        ref = oc.omega(cfg["Q"][i], cfg["nbands"])
        assert omega_rel_err(w[i], ref, fl).max() <= TOL_W, i
    assert np.all(np.diff(w, axis=1) >= 0)


def test_reduced_matrix_doubling_inverse():
    """M = 11 (N = 529): the three N x N Gram factors are inverted by
    doubling (levels of batched products with a ragged last pair) instead of
    diagonal by diagonal; C(k) against the oracle's literal pencil."""
    cell = cells.voronoi_cell(64, 24, seed=29)
    M = 11
    g = GpuCell(cell, M)
    oc = mv.OracleCell(cell, M)
    try:
        Q = np.array([0.29, 0.17])
        out = np.empty(g.n * g.n * 2)
        bs.bs_reduced_matrix(g.h, Q, out)
    finally:
        g.close()
    got = out.view(np.complex128).reshape(g.n, g.n).T
    A, Om = oc.pencil(Q)
    Li = np.linalg.inv(np.linalg.cholesky(Om))
    ref = Li @ A @ Li.conj().T
    low = np.tril_indices(g.n)
    assert np.abs(got[low] - ref[low]).max() <= 1e-11 * np.abs(ref).max()
