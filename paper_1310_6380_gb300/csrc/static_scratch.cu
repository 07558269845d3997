// bs_tridiag_eigenvalues_static: the tridiagonal eigen step for callers
// that cannot allocate device memory.
//
// bs_tridiag_eigenvalues allocates a packed copy of the tridiagonals with
// cudaMalloc and releases it with cudaFree, and cudaFree waits for the
// whole device.  Some callers cannot do either: code whose device memory
// belongs to another allocator that has reserved the pool up front (a
// framework's caching allocator, an embedding application with a fixed
// budget), and pipelined multi-stream code that must not stall the device
// on every call.  This variant keeps its scratch in a fixed array in the
// library's own device image instead, so it allocates and frees nothing.
#include "bs_internal.h"

namespace {

// Packed tridiagonals [b][d(n) | e(n-1), pad]: batch * 2n doubles at most.
constexpr size_t kStaticDoubles = (size_t)1 << 20;   // 8 MiB per GPU that loads the library
static __device__ __align__(256) double g_static_scratch[kStaticDoubles];

constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

bool is_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int bs_tridiag_eigenvalues_static(const double* d, const double* e, int n, int batch,
                                             int nbands, double* lam_out, void* stream) {
  if (!d || (!e && n > 1) || !lam_out || n < 1 || batch < 1 || nbands < 1 || nbands > n) {
    bs_set_error("bs_tridiag_eigenvalues_static: need non-NULL arrays, n >= 1, batch >= 1, "
                 "1 <= nbands <= n");
    return BS_EINVAL;
  }
  if ((size_t)batch * 2 * (size_t)n > kStaticDoubles) {
    bs_set_error("bs_tridiag_eigenvalues_static: batch * 2n = %zu exceeds the fixed scratch of "
                 "%zu doubles; split the batch", (size_t)batch * 2 * (size_t)n, kStaticDoubles);
    return BS_EINVAL;
  }
  if (!is_device(d) || (n > 1 && !is_device(e)) || !is_device(lam_out)) {
    bs_set_error("bs_tridiag_eigenvalues_static: d, e and lam_out must be device pointers");
    return BS_EINVAL;
  }
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return bs_cuda_status(ce, "bs_tridiag_eigenvalues_static device");
  if (dev < 0 || dev >= kMaxDevices) {
    bs_set_error("bs_tridiag_eigenvalues_static: device ordinal %d not supported", dev);
    return BS_EINVAL;
  }
  // one-time set-up on this device: the host-side name of the array is not
  // a device address, so ask the runtime for the array's address on the
  // current device
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    ce = cudaGetSymbolAddress(&p, g_static_scratch);
    if (ce != cudaSuccess) return bs_cuda_status(ce, "bs_tridiag_eigenvalues_static symbol");
    g_scratch_ptr[dev] = (double*)p;
  }
  double* de = g_scratch_ptr[dev];
  cudaStream_t s = (cudaStream_t)stream;
  // the array keeps the previous call's contents: clear the one padding
  // slot per matrix that no copy below writes (the kernel never reads it)
  ce = cudaMemset2DAsync(de + 2 * (size_t)n - 1, 2 * n * sizeof(double), 0, sizeof(double), batch,
                         s);
  if (ce == cudaSuccess)
    ce = cudaMemcpy2DAsync(de, 2 * n * sizeof(double), d, n * sizeof(double), n * sizeof(double),
                           batch, cudaMemcpyDeviceToDevice, s);
  if (ce == cudaSuccess && n > 1)
    ce = cudaMemcpy2DAsync(de + n, 2 * n * sizeof(double), e, (n - 1) * sizeof(double),
                           (n - 1) * sizeof(double), batch, cudaMemcpyDeviceToDevice, s);
  if (ce != cudaSuccess) return bs_cuda_status(ce, "bs_tridiag_eigenvalues_static copy");
  return bs_launch_bisect(de, n, batch, nbands, lam_out, nullptr, s, false);
}
