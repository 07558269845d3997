// Lowest eigenvalues of the real symmetric tridiagonal matrices left by the
// Householder reduction, by Sturm-sequence bisection (FP64), and the
// angular frequencies omega = sqrt(max(lambda, 0)) of Eq. (eigenvalueproblem).
//
// One thread per (matrix, eigenvalue index i): the interval [lo, hi] keeps
// count(lo) <= i < count(hi), where count(x) is the number of negative
// pivots of T - x I (Sylvester inertia), until it is as narrow as FP64
// allows relative to the Gershgorin bound of the matrix.
#include <float.h>
#include <math.h>

#include "bs_internal.h"

namespace {

__device__ __forceinline__ int sturm_count(const double* __restrict__ d,
                                           const double* __restrict__ e2, int n, double x,
                                           double pivmin) {
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  int cnt = q <= 0.0;
  for (int k = 1; k < n; ++k) {
    q = (d[k] - x) - e2[k - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += q <= 0.0;
  }
  return cnt;
}

__global__ void bisect_kernel(const double* __restrict__ de, int n, int nbands,
                              double* __restrict__ omega, int* __restrict__ stat) {
  extern __shared__ double sm[];
  double* d = sm;
  double* e2 = sm + n;
  __shared__ double red[3];
  const int b = blockIdx.x;
  const double* dg = de + (size_t)b * 2 * n;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    d[k] = dg[k];
    const double e = k + 1 < n ? dg[n + k] : 0.0;
    e2[k] = e * e;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double gl = d[0], gu = d[0], emax = 0.0;
    for (int k = 0; k < n; ++k) {
      const double el = k > 0 ? sqrt(e2[k - 1]) : 0.0, er = k + 1 < n ? sqrt(e2[k]) : 0.0;
      gl = fmin(gl, d[k] - el - er);
      gu = fmax(gu, d[k] + el + er);
      emax = fmax(emax, e2[k]);
    }
    const double tnorm = fmax(fabs(gl), fabs(gu));
    gl -= 2.0 * DBL_EPSILON * tnorm * n + DBL_MIN;
    gu += 2.0 * DBL_EPSILON * tnorm * n + DBL_MIN;
    red[0] = gl;
    red[1] = gu;
    red[2] = DBL_MIN * fmax(1.0, emax);
  }
  __syncthreads();
  const double gl = red[0], gu = red[1], pivmin = red[2];
  const double atol = 4.0 * DBL_EPSILON * fmax(fabs(gl), fabs(gu));
  int bad = 0;
  for (int i = threadIdx.x; i < nbands; i += blockDim.x) {
    double lo = gl, hi = gu;
    for (int it = 0; it < 256; ++it) {
      const double tol = fmax(atol, 4.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)));
      if (hi - lo <= tol) break;
      const double mid = 0.5 * (lo + hi);
      if (sturm_count(d, e2, n, mid, pivmin) > i) hi = mid;
      else lo = mid;
    }
    const double lam = 0.5 * (lo + hi);
    if (!isfinite(lam)) bad = 1;
    omega[(size_t)b * nbands + i] = sqrt(fmax(lam, 0.0));
  }
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0 && stat) stat[b] = bad ? BS_ENOCONV : 0;
}

}  // namespace

int bs_launch_bisect(const double* de, int n, int batch, int nbands, double* omega, int* stat,
                     cudaStream_t s) {
  const size_t smem = 2 * (size_t)n * sizeof(double);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(bisect_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return bs_cuda_status(e, "bisect smem");
  }
  bisect_kernel<<<batch, 64, smem, s>>>(de, n, nbands, omega, stat);
  BS_CHECK_LAUNCH("bisect_kernel");
  return BS_OK;
}
