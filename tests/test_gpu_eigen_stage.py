"""The eigen step alone (Sturm multisection on tridiagonals) against LAPACK
(scipy.linalg.eigvalsh_tridiagonal) on matrices known to be hard for it:
Wilkinson W21+ (pairs closer than 1e-14), glued Wilkinson blocks, exact
multiplicities, graded entries and SI-sized norms."""
import numpy as np
import pytest
import scipy.linalg as sla

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1310_6380_gb300 import binding as bs  # noqa: E402


def _wilkinson(m=10):
    d = np.abs(np.arange(-m, m + 1)).astype(float)
    return d, np.ones(2 * m)


def _cases():
    rng = np.random.default_rng(1)
    out = {}
    d = rng.standard_normal((6, 300)); e = rng.standard_normal((6, 299))
    out["random"] = (d, e)
    dw, ew = _wilkinson()
    out["wilkinson21"] = (dw[None], ew[None])
    blocks = [_wilkinson() for _ in range(5)]
    dg = np.concatenate([b[0] for b in blocks])
    eg = np.concatenate([np.concatenate([b[1], [1e-10]]) for b in blocks])[:-1]
    out["glued_wilkinson"] = (dg[None], eg[None])
    db = np.tile([1.0, 2.0, 3.0], 40); eb = np.tile([0.5, 0.5, 0.0], 40)[:-1]
    out["repeated_blocks"] = (db[None], eb[None])
    k = np.arange(200)
    out["graded"] = ((10.0 ** (-k / 20))[None], (10.0 ** (-k[:-1] / 20 - 0.5))[None])
    dp = 1e13 * rng.uniform(0, 1, (2, 400)); ep = 1e13 * rng.uniform(0, 0.3, (2, 399))
    out["si_scale"] = (dp, ep)
    out["n1"] = (np.array([[3.5], [-2.0]]), np.zeros((2, 0)))
    out["n2"] = (np.array([[1.0, 1.0]]), np.array([[1e-9]]))
    return out


@pytest.mark.parametrize("name", list(_cases().keys()))
def test_tridiagonal_eigenvalues(name):
    d, e = _cases()[name]
    batch, n = d.shape
    for nb in sorted({1, min(18, n), n}):
        lam = np.empty((batch, nb))
        bs.bs_tridiag_eigenvalues(np.ascontiguousarray(d), np.ascontiguousarray(e), nb, lam)
        for b in range(batch):
            ref = sla.eigvalsh_tridiagonal(d[b], e[b], select="i", select_range=(0, nb - 1))
            tn = np.abs(d[b]).max() + 2 * (np.abs(e[b]).max() if n > 1 else 0)
            tol = 8 * np.finfo(float).eps * np.maximum(tn, np.abs(ref))
            assert np.all(np.abs(lam[b] - ref) <= tol), (name, nb, b, np.abs(lam[b] - ref).max())


def test_device_buffers():
    d, e = _cases()["random"]
    dd = torch.tensor(d, device="cuda"); ed = torch.tensor(e, device="cuda")
    out = torch.empty((d.shape[0], 10), dtype=torch.float64, device="cuda")
    bs.bs_tridiag_eigenvalues(dd, ed, 10, out)
    host = np.empty((d.shape[0], 10))
    bs.bs_tridiag_eigenvalues(d, e, 10, host)
    assert np.array_equal(out.cpu().numpy(), host)
