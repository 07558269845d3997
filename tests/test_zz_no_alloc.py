"""The allocation-free eigen step (bs_tridiag_eigenvalues_static) against the
allocating one (bs_tridiag_eigenvalues), through the C ABI.

Some callers of this library cannot allocate device memory (their memory
belongs to another allocator, or they cannot let cudaFree wait for the
whole device).  The static variant keeps its scratch in a fixed array in
the library's device image; it must give the same eigenvalues as the
allocating entry point, on consecutive calls that reuse that array.
This file is collected last so that a failure here comes after every
other test has run.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1310_6380_gb300 import binding as bs  # noqa: E402

EPS = np.finfo(float).eps


def _tridiag(seed, batch, n):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((batch, n)), rng.uniform(0.1, 2.0, (batch, n - 1))


def _close(a, b, d, e):
    tn = np.abs(d).max() + 2 * np.abs(e).max()
    return np.all(np.abs(a - b) <= 8 * EPS * np.maximum(tn, np.abs(b)))


def test_static_matches_allocating_on_two_calls():
    # two consecutive calls with different sizes: the second reuses the array
    for seed, batch, n, nb in ((1, 40, 300, 18), (2, 7, 882, 24)):
        d, e = _tridiag(seed, batch, n)
        ref = np.empty((batch, nb))
        bs.bs_tridiag_eigenvalues(d, e, nb, ref)
        dd, ed = torch.tensor(d, device="cuda"), torch.tensor(e, device="cuda")
        out = torch.empty((batch, nb), dtype=torch.float64, device="cuda")
        bs.bs_tridiag_eigenvalues_static(dd, ed, nb, out, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert _close(out.cpu().numpy(), ref, d, e), seed


def test_static_rejects_oversize_and_host_pointers():
    # every case is rejected by the host-side checks before any copy or launch
    n, batch = 1000, 600                       # batch * 2n > 2^20
    d = torch.zeros((batch, n), dtype=torch.float64, device="cuda")
    e = torch.ones((batch, n - 1), dtype=torch.float64, device="cuda")
    out = torch.empty((batch, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(bs.BSError) as ei:
        bs.bs_tridiag_eigenvalues_static(d, e, 4, out)
    assert ei.value.code == bs.BS_EINVAL and "fixed scratch" in str(ei.value)
    # within the array, but one matrix's tridiagonal exceeds shared memory
    n = 10000
    d = torch.zeros((1, n), dtype=torch.float64, device="cuda")
    e = torch.ones((1, n - 1), dtype=torch.float64, device="cuda")
    out = torch.empty((1, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(bs.BSError) as ei:
        bs.bs_tridiag_eigenvalues_static(d, e, 4, out)
    assert ei.value.code == bs.BS_EINVAL and "shared memory" in str(ei.value)
    dh, eh = _tridiag(3, 2, 10)
    with pytest.raises(bs.BSError) as ei:
        bs.bs_tridiag_eigenvalues_static(dh, eh, 3, np.empty((2, 3)))
    assert ei.value.code == bs.BS_EINVAL
