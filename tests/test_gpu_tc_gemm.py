"""The tcgen05 contraction primitive through the C ABI: with small-integer
BF16 operands every product and partial sum is exact in FP32, so the
result must equal the integer matrix product bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1310_6380_gb300 import binding as bs  # noqa: E402


def _bf16_bits(x):
    """Exact BF16 bit patterns of small integers (|x| <= 256)."""
    return (np.asarray(x, np.float32).view(np.uint32) >> 16).astype(np.uint16)


@pytest.mark.parametrize("batch, M, N, K", [
    (1, 128, 128, 64),       # one tile, one k-block
    (1, 300, 200, 1768),     # ragged M, N; many k-blocks; K not a multiple of 64
    (3, 97, 56, 8),          # K smaller than a block
    (2, 5292, 336, 1768),    # the Rayleigh-Ritz product of the n = 882 workload
])
def test_integer_exact(batch, M, N, K):
    rng = np.random.default_rng(M + N + K)
    a = rng.integers(-64, 65, (batch, M, K))
    b = rng.integers(-64, 65, (batch, N, K))
    D = np.empty((batch, N, M), np.float32)
    bs.bs_gemm_bf16(_bf16_bits(a), _bf16_bits(b), D)
    ref = np.einsum("zmk,znk->znm", a, b)
    assert np.abs(ref).max() < 2 ** 24
    assert np.array_equal(D.astype(np.int64), ref)


def test_device_operands():
    rng = np.random.default_rng(5)
    a = rng.integers(-64, 65, (1, 256, 512))
    b = rng.integers(-64, 65, (1, 192, 512))
    Ad = torch.from_numpy(_bf16_bits(a)).cuda()
    Bd = torch.from_numpy(_bf16_bits(b)).cuda()
    Dd = torch.empty((1, 192, 256), dtype=torch.float32, device="cuda")
    bs.bs_gemm_bf16(Ad, Bd, Dd)
    assert np.array_equal(Dd.cpu().numpy().astype(np.int64), np.einsum("zmk,znk->znm", a, b))


def test_rejects_bad_k():
    z = np.zeros((1, 8, 12), np.uint16)
    with pytest.raises(bs.BSError) as ei:
        bs.bs_gemm_bf16(z, z, np.zeros((1, 8, 8), np.float32))
    assert ei.value.code == bs.BS_EINVAL
