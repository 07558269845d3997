// Lowest eigenvalues of the real symmetric tridiagonal matrices left by the
// Householder reduction, by Sturm-sequence multisection, and the angular
// frequencies omega = sqrt(max(lambda, 0)) of Eq. (eigenvalueproblem).
//
// count(x) = number of non-positive pivots of the LDL^T factorisation of
// T - x I (Sylvester inertia) = number of eigenvalues <= x.  Each eigenvalue
// index i keeps a bracket lo < lambda_i <= hi with count(lo) <= i < count(hi);
// a group of L lanes evaluates count at L interior points per sweep.
//
// GB300 executes FP64 (and above all FP64 division) far slower than FP32,
// so the bracket is first narrowed with FP32 counts to a width of
// 64 eps32 ||T|| (an FP32 count is exact for a matrix within a few eps32
// ||T|| of T), then widened by that margin, verified with FP64 counts and
// finished in FP64 to 4 eps64 max(||T||, |lambda|).  In the FP64 pivot
// recurrence q_k = (d_k - x) - e_k^2 / q_{k-1} the reciprocal of q is an
// FP32 seed refined by one cubic correction (rcp64 below), with an exact
// division when q lies outside the FP32 normal range.
// stop_rel > 4 eps ends the FP64 phase at stop_rel ||T||: the mixed path
// needs the eigenvalues of its FP32-reduced T only as inverse-iteration
// shifts, for which 1e-9 ||T|| is ample.
#include <float.h>
#include <math.h>

#include "bs_internal.h"

namespace {

constexpr int L = 4;        // lanes per eigenvalue
constexpr int NTB = 32;     // threads per block: one warp, EPC eigenvalues
constexpr int EPC = NTB / L;  // eigenvalues per CTA (a matrix's bands spread over CTAs)

// 1/q from the FP32 hardware approximation r0 (relative error e = 1 - q r0
// below 2^-22) and the series 1/q = r0 / (1 - e) = r0 (1 + e + e^2 + ...),
// cut after e^2 (what remains is below 2^-66); exact division when q lies
// outside [2^-119, 2^120), where the FP32 approximation is not normal.  The
// range test reads the exponent field, so no FP64 comparison lengthens the
// recurrence's dependency chain.
__device__ __forceinline__ double rcp64(double q) {
  const unsigned ex = ((unsigned)__double2hiint(q) >> 20) & 0x7ffu;
  if (ex - 904u <= 238u) {
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"((float)q));
    const double r0 = (double)rf;
    const double e = fma(-q, r0, 1.0);
    return fma(fma(e, e, e), r0, r0);
  }
  return 1.0 / q;
}

__device__ __forceinline__ float rcp32(float q) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(q));
  return r;
}

// |q| < pivmin as an integer comparison of the magnitude bits
__device__ __forceinline__ bool tiny64(double q, long long pivbits) {
  return (__double_as_longlong(q) & 0x7fffffffffffffffLL) < pivbits;
}
__device__ __forceinline__ bool tiny32(float q, int pivbits) {
  return (__float_as_int(q) & 0x7fffffff) < pivbits;
}

__device__ int count64(const double* __restrict__ d, const double* __restrict__ e2, int n,
                       double x, double pivmin) {
  const long long pb = __double_as_longlong(pivmin);
  double q = d[0] - x;
  if (tiny64(q, pb)) q = -pivmin;
  int cnt = q <= 0.0;
  for (int k = 1; k < n; ++k) {
    q = fma(-e2[k - 1], rcp64(q), d[k] - x);
    if (tiny64(q, pb)) q = -pivmin;
    cnt += q <= 0.0;
  }
  return cnt;
}

// The FP32 pivots take e^2 / q as e^2 times the approximate reciprocal (a
// few FP32 ulps of e^2: the count stays exact for a matrix within a few
// eps32 ||T|| of T, the margin the FP32 phase allows for)
__device__ int count32(const float* __restrict__ d, const float* __restrict__ e2, int n, float x,
                       float pivmin) {
  const int pb = __float_as_int(pivmin);
  float q = d[0] - x;
  if (tiny32(q, pb)) q = -pivmin;
  int cnt = q <= 0.0f;
  for (int k = 1; k < n; ++k) {
    q = fmaf(-e2[k - 1], rcp32(q), d[k] - x);
    if (tiny32(q, pb)) q = -pivmin;
    cnt += q <= 0.0f;
  }
  return cnt;
}

__device__ __forceinline__ double vmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ double vmin(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }

// one multisection sweep of the group: lanes evaluate L interior points
template <typename T, typename CountFn>
__device__ void sweep(T& lo, T& hi, int i, int l, unsigned mask, CountFn cnt) {
  const T x = lo + (hi - lo) * (T)(l + 1) / (T)(L + 1);
  const int c = cnt(x);
  T xl = c <= i ? x : lo;
  T xh = c > i ? x : hi;
#pragma unroll
  for (int o = 1; o < L; o <<= 1) {
    xl = vmax(xl, __shfl_xor_sync(mask, xl, o, L));
    xh = vmin(xh, __shfl_xor_sync(mask, xh, o, L));
  }
  lo = xl;
  hi = xh;
}

__global__ void __launch_bounds__(NTB) bisect_kernel(const double* __restrict__ de, int n,
                                                     int nbands, double* __restrict__ omega,
                                                     int* __restrict__ stat, int want_omega,
                                                     double stop_rel, int maxsweep) {
  extern __shared__ double sm[];
  double* d = sm;
  double* e2 = sm + n;
  float* d32 = reinterpret_cast<float*>(sm + 2 * n);
  float* e32 = d32 + n;
  __shared__ double red[4];
  const int b = blockIdx.x, tid = threadIdx.x;
  const double* dg = de + (size_t)b * 2 * n;
  for (int k = tid; k < n; k += NTB) {
    d[k] = dg[k];
    const double e = k + 1 < n ? dg[n + k] : 0.0;
    e2[k] = e * e;
    d32[k] = (float)d[k];
    e32[k] = (float)e2[k];
  }
  __syncwarp();
  {
    // Gershgorin bounds and the largest e^2, reduced over the warp
    double gl = INFINITY, gu = -INFINITY, emax = 0.0;
    for (int k = tid; k < n; k += NTB) {
      const double el = k > 0 ? sqrt(e2[k - 1]) : 0.0, er = k + 1 < n ? sqrt(e2[k]) : 0.0;
      gl = fmin(gl, d[k] - el - er);
      gu = fmax(gu, d[k] + el + er);
      emax = fmax(emax, e2[k]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      gl = fmin(gl, __shfl_xor_sync(0xffffffffu, gl, o));
      gu = fmax(gu, __shfl_xor_sync(0xffffffffu, gu, o));
      emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    }
    if (tid == 0) {
      const double tnorm = fmax(fabs(gl), fabs(gu));
      gl -= 2.0 * DBL_EPSILON * tnorm * n + DBL_MIN;
      gu += 2.0 * DBL_EPSILON * tnorm * n + DBL_MIN;
      red[0] = gl;
      red[1] = gu;
      red[2] = DBL_MIN * fmax(1.0, emax);
      red[3] = tnorm;
    }
  }
  __syncwarp();
  const double gl = red[0], gu = red[1], pivmin = red[2], tnorm = red[3];
  const double atol = fmax(4.0 * DBL_EPSILON, stop_rel) * tnorm;
  // FP32 counts need the matrix inside the FP32 range with headroom
  const bool use32 = tnorm < 1e18 && tnorm > 1e-18;
  const float pivmin32 = FLT_MIN * fmaxf(1.0f, (float)(tnorm * tnorm));
  const double w32 = 64.0 * FLT_EPSILON * tnorm;

  const int lane = tid & 31, l = tid % L;
  const unsigned mask = 0xFu << (lane & ~(L - 1));
  auto c64 = [&](double x) { return count64(d, e2, n, x, pivmin); };
  auto c32 = [&](float x) { return count32(d32, e32, n, x, pivmin32); };
  int bad = 0;
  const int iend = min(nbands, (int)(blockIdx.y + 1) * EPC);
  for (int i = blockIdx.y * EPC + tid / L; i < iend; i += NTB / L) {
    double lo = gl, hi = gu;
    if (use32) {
      float flo = (float)gl, fhi = (float)gu;
      flo = fminf(flo, (float)gl - (float)w32);
      fhi = fmaxf(fhi, (float)gu + (float)w32);
      for (int it = 0; it < min(64, maxsweep) && (double)fhi - (double)flo > w32; ++it)
        sweep(flo, fhi, i, l, mask, c32);
      // widen by the FP32 count margin and verify in FP64
      double vlo = fmax(gl, (double)flo - w32), vhi = fmin(gu, (double)fhi + w32);
      const double x = l == 0 ? vlo : vhi;
      const int c = (l < 2) ? c64(x) : 0;
      const int clo = __shfl_sync(mask, c, 0, L), chi = __shfl_sync(mask, c, 1, L);
      if (clo <= i && chi > i) {
        lo = vlo;
        hi = vhi;
      }
    }
    bool conv = false;
    for (int it = 0; it <= maxsweep; ++it) {
      const double tol = fmax(atol, 4.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)));
      conv = hi - lo <= tol;
      if (conv || it == maxsweep) break;
      sweep(lo, hi, i, l, mask, c64);
    }
    const double lam = 0.5 * (lo + hi);
    if (!isfinite(lam) || !conv) bad = 1;   // sweep limit reached: not converged
    if (l == 0) omega[(size_t)b * nbands + i] = want_omega ? sqrt(fmax(lam, 0.0)) : lam;
  }
  // the status of a matrix is zeroed before the launch; any CTA of it that
  // ran out of sweeps marks it
  bad = __any_sync(0xffffffffu, bad);
  if (tid == 0 && stat && bad) atomicMin(stat + b, BS_ENOCONV);
}

}  // namespace

int bs_launch_bisect(const double* de, int n, int batch, int nbands, double* omega, int* stat,
                     cudaStream_t s, bool want_omega, double stop_rel) {
  if (batch < 1 || nbands < 1) return BS_OK;
  const size_t smem = 2 * (size_t)n * sizeof(double) + 2 * (size_t)n * sizeof(float);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(bisect_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return bs_cuda_status(e, "bisect smem");
  }
  if (stat) {
    const cudaError_t e = cudaMemsetAsync(stat, 0, (size_t)batch * sizeof(int), s);
    if (e != cudaSuccess) return bs_cuda_status(e, "bisect status");
  }
  bisect_kernel<<<dim3(batch, (nbands + EPC - 1) / EPC), NTB, smem, s>>>(
      de, n, nbands, omega, stat, want_omega ? 1 : 0, stop_rel, bs_bisect_sweeps());
  BS_CHECK_LAUNCH("bisect_kernel");
  return BS_OK;
}
