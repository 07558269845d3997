// Dense FP64 complex linear algebra of the k-independent part of the
// method: Cholesky factors of the Gram matrices Phi (isotropic blocks
// T[1/(lam+mu)], T[1/mu]) and Omega (T[rho]) (Eqs. (ep), (eo)), their
// triangular inverses, and the six k-monomial coefficient matrices of the
// reduced matrix C(k) = L^-1 H(k) Phi^-1 H(k)^* L^-dagger.
//
// With the rotated stress basis (s11 +- s22)/sqrt2, s12 the isotropic Phi
// is block diagonal, diag(T_k/2, T_m/2, T_m) (T_k = T[1/(lam+mu)],
// T_m = T[1/mu]), and H of Eq. (eh) is diagonal per plane wave with
// entries i V K_a, K_a = k + G_a.  Writing T_X^-1 = Z_X Z_X^dagger
// (Z_X = L_X^-dagger) and W_{X,i}(k) = L_R^-1 diag(K_i) Z_X = k_i F_X^0 + F_X^i
// with F_X^0 = L_R^-1 Z_X and F_X^i = L_R^-1 diag(G_i) Z_X, the blocks of C are
//   C11 = V^2 (W_k1 W_k1^+ + W_m1 W_m1^+ + W_m2 W_m2^+)
//   C22 = V^2 (W_k2 W_k2^+ + W_m2 W_m2^+ + W_m1 W_m1^+)
//   C12 = V^2 (W_k1 W_k2^+ - W_m1 W_m2^+ + W_m2 W_m1^+)
// so C(k) is a quadratic polynomial in the Cartesian k whose six matrix
// coefficients are sums of the products P_X^{ab} = F_X^a F_X^b^dagger.
#include <math.h>

#include <algorithm>

#include "bs_internal.h"

namespace {

constexpr int NB = 32;   // block size of the blocked factorisations

// ---------------------------------------------------------------- Cholesky
// Blocked right-looking Cholesky, panels of NB columns.  The factor of a
// diagonal block is computed and stored by exactly one CTA, in a launch
// whose other CTAs do not read that block: the first block by
// chol_diag_kernel, block j + 1 by the CTA of chol_update_kernel(j) that
// owns it (it holds the block's last update).  chol_panel_kernel(j) then
// reads the stored factor of block j, never a block being rewritten.

// In-place Cholesky of the jb x jb lower triangle in shared memory; a
// pivot that is not positive sets *info and is replaced by 1.
__device__ void chol_block_smem(zd (*L)[NB + 1], int jb, int* info) {
  const int tid = threadIdx.x;
  for (int c = 0; c < jb; ++c) {
    if (tid == 0) {
      double piv = L[c][c].x;
      if (!(piv > 0.0) || !isfinite(piv)) {
        atomicOr(info, 1);
        piv = 1.0;
      }
      L[c][c] = zmake(sqrt(piv), 0.0);
    }
    __syncthreads();
    const double inv = 1.0 / L[c][c].x;
    for (int r = c + 1 + tid; r < jb; r += blockDim.x) L[r][c] = zscale(L[r][c], inv);
    __syncthreads();
    const int m = jb - c - 1;
    for (int e = tid; e < m * m; e += blockDim.x) {
      int r = c + 1 + e % m, s = c + 1 + e / m;
      if (r >= s) L[r][s] = zfnmac(L[r][c], L[s][c], L[r][s]);
    }
    __syncthreads();
  }
}

// load / store the lower triangle of the diagonal block at (j0, j0)
__device__ void diag_load(const zd* a, int n, int j0, int jb, zd (*L)[NB + 1]) {
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    int r = e % NB, c = e / NB;
    L[r][c] = (r < jb && c < jb && r >= c) ? a[(size_t)(j0 + r) + (size_t)(j0 + c) * n]
                                           : zmake(0.0, 0.0);
  }
  __syncthreads();
}
__device__ void diag_store(zd* a, int n, int j0, int jb, const zd (*L)[NB + 1]) {
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    int r = e % NB, c = e / NB;
    if (r < jb && c < jb && r >= c) a[(size_t)(j0 + r) + (size_t)(j0 + c) * n] = L[r][c];
  }
}

// the first diagonal block of each matrix
__global__ void chol_diag_kernel(zd* __restrict__ A, int n, long stride, int* __restrict__ info) {
  __shared__ zd L[NB][NB + 1];
  zd* a = A + (size_t)blockIdx.x * stride;
  const int jb = min(NB, n);
  diag_load(a, n, 0, jb, L);
  chol_block_smem(L, jb, info);
  diag_store(a, n, 0, jb, L);
}

// block row i = j + 1 + blockIdx.x of panel j0: X L_jj^dagger = A_ij with
// L_jj the stored factor of the diagonal block
__global__ void chol_panel_kernel(zd* __restrict__ A, int n, long stride, int j0) {
  __shared__ zd L[NB][NB + 1];
  __shared__ zd X[NB][NB + 1];
  zd* a = A + (size_t)blockIdx.y * stride;
  const int tid = threadIdx.x;
  const int jb = min(NB, n - j0);
  const int i0 = j0 + NB * (blockIdx.x + 1);
  if (i0 >= n) return;
  const int ib = min(NB, n - i0);
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    int r = e % NB, c = e / NB;
    L[r][c] = (r < jb && c < jb && r >= c) ? a[(size_t)(j0 + r) + (size_t)(j0 + c) * n]
                                           : zmake(0.0, 0.0);
    X[r][c] = (r < ib && c < jb) ? a[(size_t)(i0 + r) + (size_t)(j0 + c) * n] : zmake(0.0, 0.0);
  }
  __syncthreads();
  // X L^dagger = A_ij: column c of X from columns t < c
  if (tid < ib) {
    const int r = tid;
    for (int c = 0; c < jb; ++c) {
      zd x = X[r][c];
      for (int t = 0; t < c; ++t) x = zfnmac(X[r][t], L[c][t], x);
      X[r][c] = zscale(x, 1.0 / L[c][c].x);
    }
  }
  __syncthreads();
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    int r = e % NB, c = e / NB;
    if (r < ib && c < jb) a[(size_t)(i0 + r) + (size_t)(j0 + c) * n] = X[r][c];
  }
}

// (bi, bk) with bi >= bk of the l-th lower-triangular tile, row-major;
// FP32 square root (FP64 square root is a long sequence on GB300), then
// exact integer correction
__device__ __forceinline__ void tri_index(int l, int& bi, int& bk) {
  int r = (int)((sqrtf(8.0f * (float)l + 1.0f) - 1.0f) * 0.5f);
  while ((r + 1) * (r + 2) / 2 <= l) ++r;
  while (r * (r + 1) / 2 > l) --r;
  bi = r;
  bk = l - r * (r + 1) / 2;
}

// Trailing update A_ik -= L_ij L_kj^dagger for block rows i >= k > j; the
// CTA of the first trailing diagonal block then factors that block (the
// next panel's diagonal block, which no other CTA of this launch reads).
__global__ void chol_update_kernel(zd* __restrict__ A, int n, long stride, int j0,
                                   int* __restrict__ info) {
  __shared__ zd Li[NB][NB + 1];
  __shared__ zd Lk[NB][NB + 1];
  zd* a = A + (size_t)blockIdx.y * stride;
  int bi, bk;
  tri_index(blockIdx.x, bi, bk);
  const int t0 = j0 / NB + 1;
  const int i0 = (t0 + bi) * NB, k0 = (t0 + bk) * NB;
  const int jb = min(NB, n - j0);
  const int tid = threadIdx.x;
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    int r = e % NB, c = e / NB;
    bool ok = c < jb;
    Li[r][c] = (ok && i0 + r < n) ? a[(size_t)(i0 + r) + (size_t)(j0 + c) * n] : zmake(0.0, 0.0);
    Lk[r][c] = (ok && k0 + r < n) ? a[(size_t)(k0 + r) + (size_t)(j0 + c) * n] : zmake(0.0, 0.0);
  }
  __syncthreads();
  const int r = tid % NB;
  for (int cc = tid / NB; cc < NB; cc += blockDim.x / NB) {
    zd acc = zmake(0.0, 0.0);
    for (int t = 0; t < jb; ++t) acc = zfmac(Li[r][t], Lk[cc][t], acc);
    if (i0 + r < n && k0 + cc < n) {
      size_t o = (size_t)(i0 + r) + (size_t)(k0 + cc) * n;
      a[o] = zsub(a[o], acc);
    }
  }
  if (bi == 0 && bk == 0) {
    __syncthreads();   // the block's updated entries, written by this CTA
    const int nb = min(NB, n - i0);
    diag_load(a, n, i0, nb, Li);
    chol_block_smem(Li, nb, info);
    diag_store(a, n, i0, nb, Li);
  }
}

// ---------------------------------------------------------------- inverse
// X_ii = L_ii^-1 for every diagonal block; zero X above the diagonal blocks.
__global__ void trinv_diag_kernel(const zd* __restrict__ Lg, zd* __restrict__ Xg, int n,
                                  long stride) {
  __shared__ zd L[NB][NB + 1];
  __shared__ zd X[NB][NB + 1];
  const zd* l = Lg + (size_t)blockIdx.y * stride;
  zd* x = Xg + (size_t)blockIdx.y * stride;
  const int i0 = blockIdx.x * NB, ib = min(NB, n - i0), tid = threadIdx.x;
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    int r = e % NB, c = e / NB;
    L[r][c] = (r < ib && c < ib && r >= c) ? l[(size_t)(i0 + r) + (size_t)(i0 + c) * n]
                                           : zmake(0.0, 0.0);
  }
  __syncthreads();
  if (tid < ib) {
    const int c = tid;
    for (int r = 0; r < ib; ++r) {
      if (r < c) {
        X[r][c] = zmake(0.0, 0.0);
        continue;
      }
      zd s = zmake(r == c ? 1.0 : 0.0, 0.0);
      for (int t = c; t < r; ++t) s = zsub(s, zmul(L[r][t], X[t][c]));
      X[r][c] = zscale(s, 1.0 / L[r][r].x);
    }
  }
  __syncthreads();
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    int r = e % NB, c = e / NB;
    if (r < ib && c < ib) x[(size_t)(i0 + r) + (size_t)(i0 + c) * n] = X[r][c];
  }
  // zero the part of block row i to the right of the diagonal block
  const int cols = n - (i0 + ib);
  for (int e = tid; e < ib * cols; e += blockDim.x) {
    int r = e % ib, c = i0 + ib + e / ib;
    x[(size_t)(i0 + r) + (size_t)c * n] = zmake(0.0, 0.0);
  }
}

// X_ij = -X_ii sum_{k=j}^{i-1} L_ik X_kj for block diagonal i - j = d.
__global__ void trinv_off_kernel(const zd* __restrict__ Lg, zd* __restrict__ Xg, int n,
                                 long stride, int d) {
  __shared__ zd As[NB][NB + 1];
  __shared__ zd Bs[NB][NB + 1];
  const zd* l = Lg + (size_t)blockIdx.y * stride;
  zd* x = Xg + (size_t)blockIdx.y * stride;
  const int bi = d + blockIdx.x, bj = blockIdx.x;
  const int i0 = bi * NB, j0 = bj * NB;
  const int ib = min(NB, n - i0);
  const int tid = threadIdx.x, r = tid % NB, c0 = tid / NB, cs = blockDim.x / NB;
  zd acc[NB / 8];
#pragma unroll
  for (int u = 0; u < NB / 8; ++u) acc[u] = zmake(0.0, 0.0);
  for (int bk = bj; bk < bi; ++bk) {
    const int k0 = bk * NB;
    __syncthreads();
    for (int e = tid; e < NB * NB; e += blockDim.x) {
      int rr = e % NB, cc = e / NB;
      As[rr][cc] = (rr < ib) ? l[(size_t)(i0 + rr) + (size_t)(k0 + cc) * n] : zmake(0.0, 0.0);
      Bs[rr][cc] = (j0 + cc < n) ? x[(size_t)(k0 + rr) + (size_t)(j0 + cc) * n] : zmake(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < NB / 8; ++u) {
      int c = c0 + u * cs;
      for (int t = 0; t < NB; ++t) acc[u] = zfma(As[r][t], Bs[t][c], acc[u]);
    }
  }
  __syncthreads();
  // As <- X_ii, Bs <- S
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    int rr = e % NB, cc = e / NB;
    As[rr][cc] = (rr < ib && cc < ib) ? x[(size_t)(i0 + rr) + (size_t)(i0 + cc) * n]
                                      : zmake(0.0, 0.0);
  }
#pragma unroll
  for (int u = 0; u < NB / 8; ++u) Bs[r][c0 + u * cs] = acc[u];
  __syncthreads();
#pragma unroll
  for (int u = 0; u < NB / 8; ++u) {
    int c = c0 + u * cs;
    zd s = zmake(0.0, 0.0);
    for (int t = 0; t < NB; ++t) s = zfma(As[r][t], Bs[t][c], s);
    if (r < ib && j0 + c < n) x[(size_t)(i0 + r) + (size_t)(j0 + c) * n] = zmake(-s.x, -s.y);
  }
}

// ---------------------------------------------------------------- GEMM
// C = alpha * opA(A) * diag(sc) * opB(B), column-major; 32 x 32 tile per CTA.
template <bool CA, bool CB>
__global__ void zgemm_kernel(int m, int nn, int k, zd alpha, const zd* __restrict__ A, int lda,
                             long sA, const zd* __restrict__ B, int ldb, long sB,
                             const double* __restrict__ sc, long sS, zd* __restrict__ C, int ldc,
                             long sC, int tri) {
  constexpr int BM = 32, BN = 32, BK = 16;
  __shared__ zd As[BK][BM + 1];
  __shared__ zd Bs[BN][BK + 1];
  const int b = blockIdx.z;
  A += (size_t)b * sA;
  B += (size_t)b * sB;
  C += (size_t)b * sC;
  if (sc) sc += (size_t)b * sS;
  const int r0 = blockIdx.x * BM, c0 = blockIdx.y * BN;
  const int tid = threadIdx.x, tx = tid % 32, ty = tid / 32;
  int kend = k, kbeg = 0;
  if (tri & 1) kend = min(kend, r0 + BM);
  if (tri & 2) kend = min(kend, c0 + BN);
  if (tri & 4) kbeg = r0 / BK * BK;      // opA upper triangular: row r needs k >= r only
  zd acc[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) acc[i] = zmake(0.0, 0.0);
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    for (int e = tid; e < BM * BK; e += 256) {
      int r, kk;
      if (!CA) { r = e % BM; kk = e / BM; } else { kk = e % BK; r = e / BK; }
      int gr = r0 + r, gk = k0 + kk;
      zd v = zmake(0.0, 0.0);
      if (gr < m && gk < k) v = CA ? zconj(A[(size_t)gk + (size_t)gr * lda]) : A[(size_t)gr + (size_t)gk * lda];
      As[kk][r] = v;
    }
    for (int e = tid; e < BN * BK; e += 256) {
      int c, kk;
      if (!CB) { kk = e % BK; c = e / BK; } else { c = e % BN; kk = e / BN; }
      int gc = c0 + c, gk = k0 + kk;
      zd v = zmake(0.0, 0.0);
      if (gc < nn && gk < k) {
        v = CB ? zconj(B[(size_t)gc + (size_t)gk * ldb]) : B[(size_t)gk + (size_t)gc * ldb];
        if (sc) v = zscale(v, sc[gk]);
      }
      Bs[c][kk] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      zd a = As[kk][tx];
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[i] = zfma(a, Bs[ty + 8 * i][kk], acc[i]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gr = r0 + tx, gc = c0 + ty + 8 * i;
    if (gr < m && gc < nn) C[(size_t)gr + (size_t)gc * ldc] = zmul(alpha, acc[i]);
  }
}

// ---------------------------------------------------------------- monomials
// P_X^{ab} for a <= b is stored at Pp[(X*6 + pidx(a,b)) * N*N]
__device__ __forceinline__ int pidx(int a, int b) {
  // (0,0)=0 (0,1)=1 (0,2)=2 (1,1)=3 (1,2)=4 (2,2)=5
  return a == 0 ? b : (a == 1 ? 2 + b : 5);
}
__device__ __forceinline__ zd getP(const zd* __restrict__ Pp, int N, int X, int a, int b, int i,
                                   int j) {
  size_t NN = (size_t)N * N;
  if (a <= b) return Pp[(size_t)(X * 6 + pidx(a, b)) * NN + i + (size_t)j * N];
  return zconj(Pp[(size_t)(X * 6 + pidx(b, a)) * NN + j + (size_t)i * N]);
}

__global__ void monomial_kernel(const zd* __restrict__ Pp, int N, double V2, zd* __restrict__ Cm) {
  const int n = 2 * N;
  size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)n * n) return;
  const int r0 = (int)(e % n), c0 = (int)(e / n);
  // the upper triangle is the conjugate of the lower one (C(k) is Hermitian)
  const bool up = r0 < c0;
  const int r = up ? c0 : r0, c = up ? r0 : c0;
  const int I = r / N, J = c / N, i = r % N, j = c % N;
  const int K = 0, Mu = 1;
  zd m[6];
  const zd z = zmake(0.0, 0.0);
#define PP(X, a, b) getP(Pp, N, X, a, b, i, j)
  if (I == 0 && J == 0) {
    m[0] = zadd(zadd(PP(K, 1, 1), PP(Mu, 1, 1)), PP(Mu, 2, 2));
    m[1] = zadd(zadd(PP(K, 0, 1), PP(K, 1, 0)), zadd(PP(Mu, 0, 1), PP(Mu, 1, 0)));
    m[2] = zadd(PP(Mu, 0, 2), PP(Mu, 2, 0));
    m[3] = zadd(PP(K, 0, 0), PP(Mu, 0, 0));
    m[4] = z;
    m[5] = PP(Mu, 0, 0);
  } else if (I == 1 && J == 1) {
    m[0] = zadd(zadd(PP(K, 2, 2), PP(Mu, 2, 2)), PP(Mu, 1, 1));
    m[1] = zadd(PP(Mu, 0, 1), PP(Mu, 1, 0));
    m[2] = zadd(zadd(PP(K, 0, 2), PP(K, 2, 0)), zadd(PP(Mu, 0, 2), PP(Mu, 2, 0)));
    m[3] = PP(Mu, 0, 0);
    m[4] = z;
    m[5] = zadd(PP(K, 0, 0), PP(Mu, 0, 0));
  } else {   // I == 1, J == 0: C21 = C12^dagger
    m[0] = zadd(zsub(PP(K, 2, 1), PP(Mu, 2, 1)), PP(Mu, 1, 2));
    m[1] = zadd(zsub(PP(K, 2, 0), PP(Mu, 2, 0)), PP(Mu, 0, 2));
    m[2] = zadd(zsub(PP(K, 0, 1), PP(Mu, 0, 1)), PP(Mu, 1, 0));
    m[3] = z;
    m[4] = PP(K, 0, 0);
    m[5] = z;
  }
#undef PP
  const size_t nn = (size_t)n * n;
#pragma unroll
  for (int t = 0; t < 6; ++t) Cm[t * nn + e] = zscale(up ? zconj(m[t]) : m[t], V2);
}

}  // namespace

int bs_launch_cholesky(zd* A, int n, int batch, long stride, int* info, cudaStream_t s) {
  const int nt = (n + NB - 1) / NB;
  chol_diag_kernel<<<batch, 256, 0, s>>>(A, n, stride, info);
  BS_CHECK_LAUNCH("chol_diag_kernel");
  for (int j = 0; j + 1 < nt; ++j) {
    const int rem = nt - j - 1;
    chol_panel_kernel<<<dim3(rem, batch), 256, 0, s>>>(A, n, stride, j * NB);
    BS_CHECK_LAUNCH("chol_panel_kernel");
    chol_update_kernel<<<dim3(rem * (rem + 1) / 2, batch), 256, 0, s>>>(A, n, stride, j * NB,
                                                                        info);
    BS_CHECK_LAUNCH("chol_update_kernel");
  }
  return BS_OK;
}

namespace {
// zero X strictly above the diagonal
__global__ void zero_upper_kernel(zd* __restrict__ Xg, int n, long stride) {
  zd* x = Xg + (size_t)blockIdx.y * stride;
  const size_t nn = (size_t)n * n;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < nn;
       e += (size_t)gridDim.x * blockDim.x)
    if (e % n < e / n) x[e] = zmake(0.0, 0.0);
}
}  // namespace

// X = L^-1 by doubling: with the NB x NB diagonal blocks inverted, each pair
// of adjacent inverted diagonal blocks of size sz (sz = NB, 2 NB, 4 NB, ...)
// gets the off-diagonal block of the inverse of [L11 0; L21 L22],
//   X21 = -X22 L21 X11,
// as two products: T^dagger = X11^dagger L21^dagger (kept in the pair's block
// above the diagonal, which X does not use until the end), then
// X21 = -X22 (T^dagger)^dagger.  The pairs of one size are a batch of
// products whose operands lie 2 sz (n + 1) apart; a ragged last pair is its
// own launch.  Every product has full 32 x 32 output tiles over a long inner
// dimension: the work no longer waits on one CTA per block diagonal.
static int trinv_doubling(const zd* L, zd* X, int n, int batch, long stride, cudaStream_t s) {
  const zd one = zmake(1.0, 0.0), mone = zmake(-1.0, 0.0);
  for (int sz = NB; sz < n; sz *= 2) {
    const int nfull = n / (2 * sz);
    const int rem = n - nfull * 2 * sz;
    const int s2r = rem > sz ? rem - sz : 0;
    const long ps = 2L * sz * ((long)n + 1);
    for (int b = 0; b < batch; ++b) {
      const zd* Lb = L + (size_t)b * stride;
      zd* Xb = X + (size_t)b * stride;
      auto pair = [&](int i0, int s2, int np) -> int {
        const zd* X11 = Xb + i0 + (size_t)i0 * n;
        const zd* L21 = Lb + (i0 + sz) + (size_t)i0 * n;
        zd* Tp = Xb + i0 + (size_t)(i0 + sz) * n;
        zd* X21 = Xb + (i0 + sz) + (size_t)i0 * n;
        const zd* X22 = Xb + (i0 + sz) + (size_t)(i0 + sz) * n;
        TRY_LAUNCH(bs_launch_zgemm(true, true, sz, s2, sz, one, X11, n, ps, L21, n, ps, nullptr, 0,
                                   Tp, n, ps, np, 4, s));
        TRY_LAUNCH(bs_launch_zgemm(false, true, s2, sz, s2, mone, X22, n, ps, Tp, n, ps, nullptr,
                                   0, X21, n, ps, np, 1, s));
        return BS_OK;
      };
      if (nfull > 0) TRY_LAUNCH(pair(0, sz, nfull));
      if (s2r > 0) TRY_LAUNCH(pair(nfull * 2 * sz, s2r, 1));
    }
  }
  const size_t nn = (size_t)n * n;
  const unsigned g = (unsigned)std::min<size_t>((nn + 255) / 256, 4096);
  zero_upper_kernel<<<dim3(g, batch), 256, 0, s>>>(X, n, stride);
  BS_CHECK_LAUNCH("zero_upper_kernel");
  return BS_OK;
}

int bs_launch_trinv(const zd* L, zd* X, int n, int batch, long stride, cudaStream_t s) {
  const int nt = (n + NB - 1) / NB;
  trinv_diag_kernel<<<dim3(nt, batch), 256, 0, s>>>(L, X, n, stride);
  BS_CHECK_LAUNCH("trinv_diag_kernel");
  // a few large factors (a cell's own): doubling; a batch of many small ones
  // (a ragged batch's cells) keeps the SMs busy diagonal by diagonal
  if (batch <= 4 && nt >= 16) return trinv_doubling(L, X, n, batch, stride, s);
  for (int d = 1; d < nt; ++d) {
    trinv_off_kernel<<<dim3(nt - d, batch), 256, 0, s>>>(L, X, n, stride, d);
    BS_CHECK_LAUNCH("trinv_off_kernel");
  }
  return BS_OK;
}

int bs_launch_zgemm(bool conjA, bool conjB, int m, int nn, int k, zd alpha, const zd* A, int lda,
                    long sA, const zd* B, int ldb, long sB, const double* sc, long sS, zd* C,
                    int ldc, long sC, int batch, int tri, cudaStream_t s) {
  dim3 grid((m + 31) / 32, (nn + 31) / 32, batch);
  if (!conjA && !conjB)
    zgemm_kernel<false, false><<<grid, 256, 0, s>>>(m, nn, k, alpha, A, lda, sA, B, ldb, sB, sc, sS, C, ldc, sC, tri);
  else if (!conjA && conjB)
    zgemm_kernel<false, true><<<grid, 256, 0, s>>>(m, nn, k, alpha, A, lda, sA, B, ldb, sB, sc, sS, C, ldc, sC, tri);
  else if (conjA && !conjB)
    zgemm_kernel<true, false><<<grid, 256, 0, s>>>(m, nn, k, alpha, A, lda, sA, B, ldb, sB, sc, sS, C, ldc, sC, tri);
  else
    zgemm_kernel<true, true><<<grid, 256, 0, s>>>(m, nn, k, alpha, A, lda, sA, B, ldb, sB, sc, sS, C, ldc, sC, tri);
  BS_CHECK_LAUNCH("zgemm_kernel");
  return BS_OK;
}

int bs_launch_monomials(bs_cell* c, cudaStream_t s) {
  const int N = c->N;
  const size_t NN = (size_t)N * N;
  const zd* LinvR = c->d_Linv + 2 * NN;
  int* err = c->d_info + 1;
  // F_X^a = L_R^-1 diag(s_a) L_X^-dagger for X in {kappa, mu} (batch of 2), a = 0, 1, 2,
  // as exact-slice tensor-core contractions (FP64 accuracy)
  // On a mesh, H = i I1 diag(K) with I1 = int conj(f_a) f_b under the centroid
  // rule (V I on a pixel grid), so L_R^-1 I1 takes the place of V L_R^-1
  // (I1 is Hermitian: L_R^-1 I1 = L_R^-1 I1^dagger).
  cudaError_t e = cudaSuccess;
  if (c->mesh) {
    TRY_LAUNCH(bs_launch_zgemm_tc(LinvR, 0, nullptr, c->d_I1, 0, c->d_LinvR2, (long)NN, N, 1,
                                  c->d_mA, c->d_mB, c->d_mD, c->d_meA, c->d_meB, err, s));
  } else {
    e = cudaMemcpyAsync(c->d_LinvR2, LinvR, NN * sizeof(zd), cudaMemcpyDeviceToDevice, s);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_LinvR2 + NN, c->d_LinvR2, NN * sizeof(zd), cudaMemcpyDeviceToDevice,
                        s);
  if (e != cudaSuccess) return bs_cuda_status(e, "monomials copy");
  for (int a = 0; a < 3; ++a) {
    const double* sc = a == 0 ? nullptr : c->d_G + (size_t)(a - 1) * N;
    TRY_LAUNCH(bs_launch_zgemm_tc(c->d_LinvR2, (long)NN, sc, c->d_Linv, (long)NN,
                                  c->d_F + (size_t)a * NN, (long)(3 * NN), N, 2, c->d_mA, c->d_mB,
                                  c->d_mD, c->d_meA, c->d_meB, err, s));
  }
  // P_X^{ab} = F_X^a F_X^b^dagger, a <= b
  const int pa[6] = {0, 0, 0, 1, 1, 2}, pb[6] = {0, 1, 2, 1, 2, 2};
  for (int t = 0; t < 6; ++t) {
    TRY_LAUNCH(bs_launch_zgemm_tc(c->d_F + (size_t)pa[t] * NN, (long)(3 * NN), nullptr,
                                  c->d_F + (size_t)pb[t] * NN, (long)(3 * NN),
                                  c->d_Pp + (size_t)t * NN, (long)(6 * NN), N, 2, c->d_mA, c->d_mB,
                                  c->d_mD, c->d_meA, c->d_meB, err, s));
  }
  const size_t tot = (size_t)c->n * c->n;
  const double V2 = c->mesh ? 1.0 : c->V * c->V;
  monomial_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(c->d_Pp, N, V2, c->d_Cm);
  BS_CHECK_LAUNCH("monomial_kernel");
  return BS_OK;
}
