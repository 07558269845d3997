// Per-k builder of the reduced Hermitian matrix.
//
// C(k) = L^-1 H(k) Phi^-1 H(k)^* L^-dagger is quadratic in the Cartesian
// wavevector k = Q1 q^1 + Q2 q^2 because H(k) of Eq. (eh) is linear in
// K = k + G.  With the six coefficient matrices assembled once per cell,
//   C(k) = C_1 + k1 C_k1 + k2 C_k2 + k1^2 C_k11 + k1 k2 C_k12 + k2^2 C_k22,
// so the per-k build is a streaming linear combination (HBM bound) of the
// lower triangles, written for a whole batch of wavevectors at once so each
// coefficient element is read once per batch.
#include "bs_internal.h"

namespace {

constexpr int KB = 32;   // wavevectors per pass over the coefficients

__global__ void builder_kernel(const zd* __restrict__ Cm, int n, const double* __restrict__ Q,
                               int nk, double q1x, double q1y, double q2x, double q2y,
                               zd* __restrict__ C) {
  __shared__ double coef[KB][6];
  const size_t nn = (size_t)n * n;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = e < nn && (int)(e % n) >= (int)(e / n);
  zd m[6];
  if (live) {
#pragma unroll
    for (int t = 0; t < 6; ++t) m[t] = Cm[t * nn + e];
  }
  for (int k0 = 0; k0 < nk; k0 += KB) {
    const int kb = min(KB, nk - k0);
    __syncthreads();
    if (threadIdx.x < kb) {
      const double Q1 = Q[2 * (k0 + threadIdx.x)], Q2 = Q[2 * (k0 + threadIdx.x) + 1];
      const double k1 = Q1 * q1x + Q2 * q2x, k2 = Q1 * q1y + Q2 * q2y;
      coef[threadIdx.x][0] = 1.0;
      coef[threadIdx.x][1] = k1;
      coef[threadIdx.x][2] = k2;
      coef[threadIdx.x][3] = k1 * k1;
      coef[threadIdx.x][4] = k1 * k2;
      coef[threadIdx.x][5] = k2 * k2;
    }
    __syncthreads();
    if (!live) continue;
    for (int b = 0; b < kb; ++b) {
      double re = m[0].x, im = m[0].y;
#pragma unroll
      for (int t = 1; t < 6; ++t) {
        re = fma(coef[b][t], m[t].x, re);
        im = fma(coef[b][t], m[t].y, im);
      }
      C[(size_t)(k0 + b) * nn + e] = zmake(re, im);
    }
  }
}

}  // namespace

int bs_launch_builder(const zd* Cm, int n, const double* Q, int nk, double q1x, double q1y,
                      double q2x, double q2y, zd* C, cudaStream_t s) {
  const size_t nn = (size_t)n * n;
  builder_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(Cm, n, Q, nk, q1x, q1y, q2x, q2y, C);
  BS_CHECK_LAUNCH("builder_kernel");
  return BS_OK;
}
