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
#include <atomic>

#include "bs_internal.h"

namespace {

// Packed tridiagonals [b][d(n) | e(n-1), pad]: batch * 2n doubles at most.
constexpr size_t kStaticDoubles = (size_t)1 << 20;   // 8 MiB per GPU that loads the library
static __device__ __align__(256) double g_static_scratch[kStaticDoubles];

constexpr int kMaxDevices = 64;
// Device address of the array on each device, looked up once per device.
// Atomic so that host threads making their first calls at the same time
// (on one device or on several) do not race on the cache; the lookup
// itself is idempotent, so two threads that both miss store the same value.
std::atomic<double*> g_scratch_ptr[kMaxDevices];

// The eigen step keeps the packed tridiagonal of one matrix in shared
// memory: 2n doubles and 2n floats per block.
constexpr size_t kSmemPerOrder = 2 * sizeof(double) + 2 * sizeof(float);

// A device pointer usable by a kernel launched on device `dev`: device
// memory that lives on `dev` itself, or managed memory.  Device memory of
// another GPU is rejected (a kernel on `dev` would otherwise write a peer's
// memory, which faults without peer access).
bool on_device(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
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
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return bs_cuda_status(ce, "bs_tridiag_eigenvalues_static device");
  if (dev < 0 || dev >= kMaxDevices) {
    bs_set_error("bs_tridiag_eigenvalues_static: device ordinal %d not supported", dev);
    return BS_EINVAL;
  }
  if (!on_device(d, dev) || (n > 1 && !on_device(e, dev)) || !on_device(lam_out, dev)) {
    bs_set_error("bs_tridiag_eigenvalues_static: d, e and lam_out must be device pointers on "
                 "the current device (%d)", dev);
    return BS_EINVAL;
  }
  int smem_max = 0;
  ce = cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (ce != cudaSuccess) return bs_cuda_status(ce, "bs_tridiag_eigenvalues_static attribute");
  if ((size_t)n * kSmemPerOrder > (size_t)smem_max) {
    bs_set_error("bs_tridiag_eigenvalues_static: n = %d needs %zu bytes of shared memory per "
                 "block, above this device's %d (n <= %zu)", n, (size_t)n * kSmemPerOrder,
                 smem_max, (size_t)smem_max / kSmemPerOrder);
    return BS_EINVAL;
  }
  // one-time set-up on this device: the host-side name of the array is not
  // a device address, so ask the runtime for the array's address on the
  // current device
  double* de = g_scratch_ptr[dev].load(std::memory_order_acquire);
  if (!de) {
    void* p = nullptr;
    ce = cudaGetSymbolAddress(&p, g_static_scratch);
    if (ce != cudaSuccess) return bs_cuda_status(ce, "bs_tridiag_eigenvalues_static symbol");
    de = (double*)p;
    g_scratch_ptr[dev].store(de, std::memory_order_release);
  }
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
