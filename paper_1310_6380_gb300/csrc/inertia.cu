// Eigenvalue-count certificate for the iterative eigen path.
//
// A residual bound tells that each Ritz value lies near SOME eigenvalue of
// C(k); it cannot tell that no eigenvalue was skipped.  Sylvester's law of
// inertia can: the number of negative pivots of an LDL^dagger factorisation
// of C - sigma I equals the number of eigenvalues below sigma.  With sigma in
// a gap just above the wanted Ritz values, a count larger than the number of
// Ritz values below sigma exposes a missed eigenvalue.
//
// The factorisation runs in FP32 without pivoting on the congruent, diagonally
// scaled matrix S (C - sigma I) S, S = diag(C)^-1/2 (congruence keeps the
// inertia; the scaling evens out the rows).  A pivot smaller than 1e-5 of the
// scaled unit diagonal makes the count unreliable and is reported as such.
// Blocked right-looking, panels of 32: a panel kernel for the block rows
// below each diagonal block and a trailing-update kernel over the
// lower-triangular tiles (whose first tile's CTA also factors the next
// diagonal block), for a batch of matrices.
#include <float.h>
#include <math.h>

#include "bs_internal.h"

namespace {

constexpr int NB = 32;
constexpr float TINY_PIVOT = 1e-5f;

// sigma and the expected count per k (bs_count_shift); no usable gap: flag
// (count unreliable)
__global__ void inertia_shift_kernel(const double* __restrict__ theta, int b, int nb, int kb,
                                     double floor2, float* __restrict__ sigma,
                                     int* __restrict__ expect, int* __restrict__ flag,
                                     bool given) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kb) return;
  if (given)
    flag[k] = expect[k] < 0 ? 1 : 0;
  else
    flag[k] = bs_count_shift(theta + (size_t)k * b, b, nb, floor2, sigma + k, expect + k) ? 0 : 1;
}

// sc[k][r] = diag(C)_r^-1/2
__global__ void inertia_diag_kernel(const zf* __restrict__ C, int n, int kb, float* __restrict__ sc) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)n * kb) return;
  const size_t k = e / n, r = e % n;
  sc[e] = rsqrtf(fmaxf(C[k * n * n + r * n + r].x, FLT_MIN));
}

// A <- S (A - sigma I) S in place on the lower triangle (FP32), S = diag(sc)
__global__ void inertia_scale_kernel(zf* __restrict__ A, int n, const float* __restrict__ sigma,
                                     const float* __restrict__ sc) {
  const size_t nn = (size_t)n * n;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (e >= nn) return;
  const int r = (int)(e % n), c = (int)(e / n);
  if (r < c) return;
  const float s = sc[(size_t)k * n + r] * sc[(size_t)k * n + c];
  zf* ak = A + (size_t)k * nn;
  zf v = ak[e];
  if (r == c) v = make_float2(v.x - sigma[k], 0.f);
  ak[e] = make_float2(v.x * s, v.y * s);
}

// Blocked right-looking LDL^dagger, panels of NB columns.  As in the FP64
// Cholesky, each diagonal block is factored and stored by exactly one CTA,
// in a launch whose other CTAs do not read it: the first by
// ldl_diag_kernel, block j + 1 by the CTA of ldl_update_kernel(j) that
// owns it.  That CTA also counts the block's negative pivots.

// In-place A11 = L11 D1 L11^dagger of the jb x jb lower triangle in shared
// memory (unit L11 below the diagonal, D1 in d); a pivot below TINY_PIVOT
// in magnitude flags the count of matrix k as unreliable.
__device__ void ldl_block_smem(zf (*L)[NB + 1], float* d, int jb, int* flag) {
  const int tid = threadIdx.x;
  for (int c = 0; c < jb; ++c) {
    if (tid == 0) {
      float p = L[c][c].x;
      if (!(fabsf(p) >= TINY_PIVOT)) {
        *flag = 1;
        p = p < 0.f ? -TINY_PIVOT : TINY_PIVOT;
      }
      d[c] = p;
      L[c][c] = make_float2(1.f, 0.f);
    }
    __syncthreads();
    const float inv = 1.f / d[c];
    // column c of L below the diagonal
    for (int r = c + 1 + tid; r < jb; r += blockDim.x) L[r][c] = zscale(L[r][c], inv);
    __syncthreads();
    // right-looking update of the remaining lower part: A_rs -= l_rc d_c conj(l_sc)
    const int m = jb - c - 1;
    for (int e = tid; e < m * m; e += blockDim.x) {
      const int r = c + 1 + e % m, s = c + 1 + e / m;
      if (r >= s) {
        const zf lr = L[r][c], ls = L[s][c];
        const float dc = d[c];
        zf v = L[r][s];
        v.x -= dc * (lr.x * ls.x + lr.y * ls.y);
        v.y -= dc * (lr.y * ls.x - lr.x * ls.y);
        L[r][s] = v;
      }
    }
    __syncthreads();
  }
}

// load the lower triangle of the diagonal block at (j0, j0), factor it,
// store L (strictly lower) and D (on the diagonal), add its negative pivots
__device__ void ldl_diag(zf* a, int n, int j0, int k, zf (*L)[NB + 1], float* d, int* neg,
                         int* flag) {
  const int jb = min(NB, n - j0);
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e % NB, c = e / NB;
    L[r][c] = (r < jb && c < jb && r >= c) ? a[(size_t)(j0 + r) + (size_t)(j0 + c) * n]
                                           : make_float2(0.f, 0.f);
  }
  __syncthreads();
  ldl_block_smem(L, d, jb, flag + k);
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e % NB, c = e / NB;
    if (r < jb && c < jb && r >= c)
      a[(size_t)(j0 + r) + (size_t)(j0 + c) * n] = r == c ? make_float2(d[r], 0.f) : L[r][c];
  }
  if (threadIdx.x == 0) {
    int cnt = 0;
    for (int c = 0; c < jb; ++c) cnt += d[c] < 0.f;
    atomicAdd(neg + k, cnt);
  }
}

__global__ void ldl_diag_kernel(zf* __restrict__ A, int n, int* __restrict__ neg,
                                int* __restrict__ flag) {
  __shared__ zf L[NB][NB + 1];
  __shared__ float d[NB];
  const int k = blockIdx.x;
  ldl_diag(A + (size_t)k * n * n, n, 0, k, L, d, neg, flag);
}

// block row i = j + 1 + blockIdx.x of panel j0: L_i1 = A_i1 L11^-dagger D1^-1
// from the stored factor of the diagonal block
__global__ void ldl_panel_kernel(zf* __restrict__ A, int n, int j0) {
  __shared__ zf L[NB][NB + 1];
  __shared__ zf X[NB][NB + 1];
  __shared__ float d[NB];
  zf* a = A + (size_t)blockIdx.y * n * n;
  const int tid = threadIdx.x;
  const int jb = min(NB, n - j0);
  const int i0 = j0 + NB * (blockIdx.x + 1);
  if (i0 >= n) return;
  const int ib = min(NB, n - i0);
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    const int r = e % NB, c = e / NB;
    L[r][c] = (r < jb && c < jb && r > c) ? a[(size_t)(j0 + r) + (size_t)(j0 + c) * n]
                                          : make_float2(0.f, 0.f);
    X[r][c] = (r < ib && c < jb) ? a[(size_t)(i0 + r) + (size_t)(j0 + c) * n]
                                 : make_float2(0.f, 0.f);
  }
  if (tid < NB) d[tid] = tid < jb ? a[(size_t)(j0 + tid) * (n + 1)].x : 1.f;
  __syncthreads();
  // Y L11^dagger = A_i1 (unit L11), then L_i1 = Y D1^-1
  if (tid < ib) {
    const int r = tid;
    for (int c = 0; c < jb; ++c) {
      zf y = X[r][c];
      for (int t = 0; t < c; ++t) y = zfnmac(X[r][t], L[c][t], y);
      X[r][c] = y;
    }
    for (int c = 0; c < jb; ++c) X[r][c] = zscale(X[r][c], 1.f / d[c]);
  }
  __syncthreads();
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    const int r = e % NB, c = e / NB;
    if (r < ib && c < jb) a[(size_t)(i0 + r) + (size_t)(j0 + c) * n] = X[r][c];
  }
}

// (bi, bk), bi >= bk, of the l-th lower-triangular tile (row-major order)
__device__ __forceinline__ void tile_of(int l, int& bi, int& bk) {
  int r = (int)((sqrtf(8.0f * (float)l + 1.0f) - 1.0f) * 0.5f);
  while ((r + 1) * (r + 2) / 2 <= l) ++r;
  while (r * (r + 1) / 2 > l) --r;
  bi = r;
  bk = l - r * (r + 1) / 2;
}

// trailing update A_ik -= L_i1 D1 L_k1^dagger for block rows i >= k > panel;
// the CTA of the first trailing diagonal block then factors that block
__global__ void ldl_update_kernel(zf* __restrict__ A, int n, int j0, int* __restrict__ neg,
                                  int* __restrict__ flag) {
  __shared__ zf Li[NB][NB + 1];
  __shared__ zf Lk[NB][NB + 1];
  __shared__ float d[NB];
  zf* a = A + (size_t)blockIdx.y * n * n;
  int bi, bk;
  tile_of(blockIdx.x, bi, bk);
  const int t0 = j0 / NB + 1;
  const int i0 = (t0 + bi) * NB, k0 = (t0 + bk) * NB;
  const int jb = min(NB, n - j0);
  const int tid = threadIdx.x;
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    const int r = e % NB, c = e / NB;
    const bool ok = c < jb;
    Li[r][c] = (ok && i0 + r < n) ? a[(size_t)(i0 + r) + (size_t)(j0 + c) * n] : make_float2(0.f, 0.f);
    Lk[r][c] = (ok && k0 + r < n) ? a[(size_t)(k0 + r) + (size_t)(j0 + c) * n] : make_float2(0.f, 0.f);
  }
  if (tid < NB) d[tid] = tid < jb ? a[(size_t)(j0 + tid) * (n + 1)].x : 0.f;
  __syncthreads();
  const int r = tid % NB;
  for (int cc = tid / NB; cc < NB; cc += blockDim.x / NB) {
    float ax = 0.f, ay = 0.f;
    for (int t = 0; t < jb; ++t) {
      const zf li = Li[r][t], lk = Lk[cc][t];
      const float dt = d[t];
      ax += dt * (li.x * lk.x + li.y * lk.y);
      ay += dt * (li.y * lk.x - li.x * lk.y);
    }
    if (i0 + r < n && k0 + cc < n && i0 + r >= k0 + cc) {
      const size_t o = (size_t)(i0 + r) + (size_t)(k0 + cc) * n;
      a[o].x -= ax;
      a[o].y -= ay;
    }
  }
  if (bi == 0 && bk == 0) {
    __syncthreads();   // the block's updated entries, written by this CTA
    ldl_diag(a, n, i0, blockIdx.y, Li, d, neg, flag);
  }
}

__global__ void inertia_decide_kernel(const int* __restrict__ neg, const int* __restrict__ expect,
                                     const int* __restrict__ flag, int kb, int* __restrict__ stat,
                                     int* __restrict__ outcome) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kb) return;
  const int bad = flag[k] || neg[k] != expect[k];
  if (outcome) outcome[k] = flag[k] ? 2 : (neg[k] != expect[k] ? 1 : 0);
  if (bad && stat[k] == 0) stat[k] = BS_ENOCONV;
}

}  // namespace

// Count check of kb problems: A (kb x n x n FP32, lower triangle of C(k)) is
// overwritten with the factors; theta (kb x b FP64 Ritz values); sigma (kb)
// and sc (kb x n) floats and iwork (3 kb ints) are scratch; stat[k] becomes
// BS_ENOCONV where the count does not match or cannot be trusted; outcome
// (optional, kb) 0 ok, 1 count mismatch, 2 unreliable.
int bs_launch_inertia_check(zf* A, int n, int kb, const double* theta, int b, int nb,
                            double floor2, float* sigma, float* sc, int* iwork, int* stat,
                            int* outcome, cudaStream_t s, bool shift_given) {
  int* neg = iwork;
  int* expect = iwork + kb;
  int* flag = iwork + 2 * kb;
  inertia_shift_kernel<<<(kb + 127) / 128, 128, 0, s>>>(theta, b, nb, kb, floor2, sigma, expect,
                                                        flag, shift_given);
  BS_CHECK_LAUNCH("inertia_shift_kernel");
  cudaError_t e = cudaMemsetAsync(neg, 0, kb * sizeof(int), s);
  if (e != cudaSuccess) return bs_cuda_status(e, "inertia counters");
  const size_t nn = (size_t)n * n;
  inertia_diag_kernel<<<(unsigned)(((size_t)n * kb + 255) / 256), 256, 0, s>>>(A, n, kb, sc);
  BS_CHECK_LAUNCH("inertia_diag_kernel");
  inertia_scale_kernel<<<dim3((unsigned)((nn + 255) / 256), kb), 256, 0, s>>>(A, n, sigma, sc);
  BS_CHECK_LAUNCH("inertia_scale_kernel");
  const int nt = (n + NB - 1) / NB;
  ldl_diag_kernel<<<kb, 256, 0, s>>>(A, n, neg, flag);
  BS_CHECK_LAUNCH("ldl_diag_kernel");
  for (int j = 0; j + 1 < nt; ++j) {
    const int rem = nt - j - 1;
    ldl_panel_kernel<<<dim3(rem, kb), 256, 0, s>>>(A, n, j * NB);
    BS_CHECK_LAUNCH("ldl_panel_kernel");
    ldl_update_kernel<<<dim3(rem * (rem + 1) / 2, kb), 256, 0, s>>>(A, n, j * NB, neg, flag);
    BS_CHECK_LAUNCH("ldl_update_kernel");
  }
  inertia_decide_kernel<<<(kb + 127) / 128, 128, 0, s>>>(neg, expect, flag, kb, stat, outcome);
  BS_CHECK_LAUNCH("inertia_decide_kernel");
  return BS_OK;
}
