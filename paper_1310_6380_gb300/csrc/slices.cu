// Digit-plane packing and FP64 recombination around the tcgen05 exact-slice
// contraction (tc_gemm.cu), for the contractions that use it:
//
//  * assembly, first separable stage of the form factors:
//      Y_f[p][d] = sum_q g_f[p][q] E[d][q],  E[d][q] = exp(-i pi dd (2q+1)/P),
//    A rows (f, p) = digits of g_f (per-row scale), B rows (d, re|im) =
//    digits of E; K = P.
//  * mixed path, Rayleigh-Ritz product Y = C X (C Hermitian n x n, X n x b):
//      Re Y = [Cr | Ci] [Xr; -Xi],  Im Y = [Cr | Ci] [Xi; Xr],
//    A rows r = digits of row r of [Cr | Ci] (row r of C is the conjugate of
//    column r, so it is read contiguously), B rows (i, part) = digits of
//    the two stacked columns; K = 2n.
//  * complex N x N products C = A diag(sc) B^dagger (the k-monomials):
//    A rows r of [Ar sc | Ai sc], B rows (c, part) of [Br | Bi], [-Bi | Br];
//    K = 2N.
//
// Digits: u = x 2^-e in (-1, 1) (e from frexp of the row maximum), then
// t_0 = rint(64 u), r_0 = 64 u - t_0, t_s = rint(128 r_{s-1}), ...: every
// |t_s| <= 64 and x = 2^e sum_s t_s 2^(-6 - 7s) + O(2^(e - 7 - 7S)).
//
// Layout: the S digits of a row sit side by side along K, each block Kp
// wide (Kp = K rounded up to 64, zero digits in the padding): A rows
// [A_0 | ... | A_{S-1}], B rows in reverse [B_{S-1} | ... | B_0].  The
// tensor cores then form each digit order u = s + t directly as one
// contraction (bs_launch_slice_orders): A columns [0, (u+1) Kp) against B
// columns [(S-1-u) Kp, S Kp), split into slabs of at most 4032 terms so
// that the FP32 sum of the digit products (each at most 2^12) stays exact
// (shorter slabs when the product is too small to fill the SMs otherwise).
// The recombination adds the slabs of each order as exact 32-bit integers
// and combines the S orders in FP64 with exactly constructed powers of two.
#include <cuda_bf16.h>
#include <math.h>
#include <stddef.h>

#include "bs_internal.h"

namespace {

// 2^e exactly (-1022 <= e <= 1023)
__device__ __forceinline__ double pow2(int e) {
  return __longlong_as_double((long long)(1023 + e) << 52);
}

// The slabs of one digit order u are summed as exact 32-bit integers (each
// slab sum is an integer below 2^24 in magnitude and there are at most
// BS_SLAB_MAX slabs); the order sums are combined as sum_u 2^(-12 - 7u) o_u
// in FP64, in increasing u (the slab table lists the orders in that order).
// Plane q of the output is Dm + q * plane; (re, im) are the two entries read.
__device__ __forceinline__ void order_sums(const float* __restrict__ Dm, size_t plane, size_t re,
                                           size_t im, const SliceSlabs& sl, double* xr,
                                           double* xi) {
  double vr = 0.0, vi = 0.0;
  int ar = 0, ai = 0, u = sl.order[0];
  for (int q = 0; q < sl.nq; ++q) {
    if (sl.order[q] != u) {
      vr = fma(pow2(-12 - 7 * u), (double)ar, vr);
      vi = fma(pow2(-12 - 7 * u), (double)ai, vi);
      ar = ai = 0;
      u = sl.order[q];
    }
    const float* dq = Dm + (size_t)q * plane;
    ar += __float2int_rn(dq[re]);
    ai += __float2int_rn(dq[im]);
  }
  *xr = fma(pow2(-12 - 7 * u), (double)ar, vr);
  *xi = fma(pow2(-12 - 7 * u), (double)ai, vi);
}

__device__ __forceinline__ uint16_t bf16_bits(double t) {
  return __bfloat16_as_ushort(__float2bfloat16_rn((float)t));
}
__device__ __forceinline__ uint16_t bf16_bits(long long t) {   // exact for |t| <= 256
  return __bfloat16_as_ushort(__int2bfloat16_rn((int)t));
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// block-wide max of |x| over a row; blockDim.x == 128
__device__ double row_max(double v, double* sh) {
  v = warp_max(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  const double m = fmax(fmax(sh[0], sh[1]), fmax(sh[2], sh[3]));
  __syncthreads();
  return m;
}

__device__ __forceinline__ int row_exp(double m) {
  int e = 0;
  if (m > 0.0) frexp(m, &e);
  return e;
}

// Digits by integer arithmetic on the FP64 bit pattern (FP64 arithmetic is
// slow on GB300): X = round(x 2^(48-e)) as a signed 64-bit integer
// (|X| <= 2^48), then t_0 = floor((X + 2^41) / 2^42), remainder r, and
// t_s = floor((r + 2^(41-7s)) / 2^(42-7s)) for s >= 1, each in [-64, 64].
// Digit s goes to out[s * plane] (plane < 0 for the reversed B layout).
__device__ __forceinline__ void put_digits(double x, int e, int S, uint16_t* out,
                                           ptrdiff_t plane) {
  const long long bits = __double_as_longlong(x);
  const int E = (int)((bits >> 52) & 0x7FF);
  long long X = 0;
  if (E != 0) {
    const long long m = (bits & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
    const int sh = 1075 - E - 48 + e;   // X = m 2^-sh
    if (sh <= 0) X = m << (-sh);        // not reached: |x| <= 2^e keeps sh >= 4
    else if (sh < 63) X = (m + (1LL << (sh - 1))) >> sh;
    if (bits < 0) X = -X;
  }
  long long r = X;
  for (int s = 0; s < S; ++s) {
    const int sh = 42 - 7 * s;
    long long t;
    if (sh > 0) t = (r + (1LL << (sh - 1))) >> sh;
    else t = r;
    r -= t << (sh > 0 ? sh : 0);
    out[(ptrdiff_t)s * plane] = bf16_bits(t);
  }
}

// ---- assembly operands
// A rows (f, p): grid (P, nf), block 128
__global__ void pack_fields_kernel(const uint16_t* __restrict__ phase,
                                   const double* __restrict__ tab, int nphase, int P, int S,
                                   int Kp, uint16_t* __restrict__ A, int* __restrict__ eA) {
  __shared__ double sh[4];
  const int p = blockIdx.x, f = blockIdx.y;
  double m = 0.0;
  for (int q = threadIdx.x; q < P; q += 128)
    m = fmax(m, fabs(tab[f * nphase + phase[(size_t)p * P + q]]));
  const int e = row_exp(row_max(m, sh));
  uint16_t* base = A + ((size_t)f * P + p) * S * Kp;
  for (int q = threadIdx.x; q < Kp; q += 128) {
    const double g = q < P ? tab[f * nphase + phase[(size_t)p * P + q]] : 0.0;
    put_digits(g, e, S, base + q, Kp);
  }
  if (threadIdx.x == 0) eA[f * P + p] = e;
}

// B rows (d, c), digits reversed: grid (2D), block 128; E from the exponential table
__global__ void pack_exp_kernel(const zd* __restrict__ E, int P, int D, int S, int Kp,
                                uint16_t* __restrict__ B, int* __restrict__ eB) {
  __shared__ double sh[4];
  const int row = blockIdx.x, d = row >> 1, c = row & 1;
  double m = 0.0;
  for (int q = threadIdx.x; q < P; q += 128) {
    const zd v = E[(size_t)d * P + q];
    m = fmax(m, fabs(c ? v.y : v.x));
  }
  const int e = row_exp(row_max(m, sh));
  uint16_t* base = B + (size_t)row * S * Kp + (size_t)(S - 1) * Kp;
  for (int q = threadIdx.x; q < Kp; q += 128) {
    double x = 0.0;
    if (q < P) {
      const zd v = E[(size_t)d * P + q];
      x = c ? v.y : v.x;
    }
    put_digits(x, e, S, base + q, -(ptrdiff_t)Kp);
  }
  if (threadIdx.x == 0) eB[row] = e;
}

// Y[f][p][d] = 2^(eA + eB) sum_u 2^(-12-7u) (slabs of order u)[(d, c)][(f, p)]
__global__ void recombine_fields_kernel(const float* __restrict__ Dm, const SliceSlabs sl,
                                        const int* __restrict__ eA, const int* __restrict__ eB,
                                        int P, int D, int nf, zd* __restrict__ Y) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)nf * P * D) return;
  const int d = (int)(i % D), p = (int)((i / D) % P), f = (int)(i / ((size_t)P * D));
  const size_t M = (size_t)nf * P, Nn = 2 * (size_t)D, m = (size_t)f * P + p;
  double xr, xi;
  order_sums(Dm, Nn * M, (2 * (size_t)d) * M + m, (2 * (size_t)d + 1) * M + m, sl, &xr, &xi);
  const int ea = eA[f * P + p];
  Y[i] = zmake(ldexp(xr, ea + eB[2 * d]), ldexp(xi, ea + eB[2 * d + 1]));
}

// ---- Rayleigh-Ritz product operands
// A rows r of [Cr | Ci] for each k: grid (n, kb), block 128
__global__ void pack_cmat_kernel(const zd* __restrict__ C, int n, int S, int Kp,
                                 uint16_t* __restrict__ A, int* __restrict__ eA) {
  __shared__ double sh[4];
  const int r = blockIdx.x, k = blockIdx.y;
  const zd* col = C + (size_t)k * n * n + (size_t)r * n;   // column r = conj(row r)
  double m = 0.0;
  for (int c = threadIdx.x; c < n; c += 128) {
    const zd v = col[c];
    m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
  }
  const int e = row_exp(row_max(m, sh));
  uint16_t* base = A + ((size_t)k * n + r) * S * Kp;
  for (int c = threadIdx.x; c < Kp; c += 128) {
    double x = 0.0;
    if (c < n) x = col[c].x;                   // Re C[r][c] = Re C[c][r]
    else if (c < 2 * n) x = -col[c - n].y;     // Im C[r][c] = -Im C[c][r]
    put_digits(x, e, S, base + c, Kp);
  }
  if (threadIdx.x == 0) eA[(size_t)k * n + r] = e;
}

// B rows (i, part), digits reversed: part 0 = [Xr; -Xi], part 1 = [Xi; Xr];
// grid (b, kb), block 128
__global__ void pack_xmat_kernel(const zd* __restrict__ X, int n, int b, int S, int Kp,
                                 uint16_t* __restrict__ B, int* __restrict__ eB) {
  __shared__ double sh[4];
  const int i = blockIdx.x, k = blockIdx.y;
  const zd* x = X + (size_t)k * n * b + (size_t)i * n;
  double m = 0.0;
  for (int r = threadIdx.x; r < n; r += 128) m = fmax(m, fmax(fabs(x[r].x), fabs(x[r].y)));
  const int e = row_exp(row_max(m, sh));
  uint16_t* base0 = B + ((size_t)k * 2 * b + 2 * i) * S * Kp + (size_t)(S - 1) * Kp;
  uint16_t* base1 = base0 + (size_t)S * Kp;
  for (int c = threadIdx.x; c < Kp; c += 128) {
    double v0 = 0.0, v1 = 0.0;
    if (c < n) {
      v0 = x[c].x;
      v1 = x[c].y;
    } else if (c < 2 * n) {
      v0 = -x[c - n].y;
      v1 = x[c - n].x;
    }
    put_digits(v0, e, S, base0 + c, -(ptrdiff_t)Kp);
    put_digits(v1, e, S, base1 + c, -(ptrdiff_t)Kp);
  }
  if (threadIdx.x == 0) eB[(size_t)k * b + i] = e;
}

// Y[k][r + i n] = 2^(eA + eB) sum_u 2^(-12-7u) (slabs of order u)[(i, part)][r]
__global__ void recombine_cx_kernel(const float* __restrict__ Dm, const SliceSlabs sl,
                                    const int* __restrict__ eA, const int* __restrict__ eB, int n,
                                    int b, zd* __restrict__ Y) {
  const int k = blockIdx.y;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * b) return;
  const int r = idx % n, i = idx / n;
  const size_t M = (size_t)n, Nn = 2 * (size_t)b;
  const float* dk = Dm + (size_t)k * sl.nq * Nn * M;
  double xr, xi;
  order_sums(dk, Nn * M, (2 * (size_t)i) * M + r, (2 * (size_t)i + 1) * M + r, sl, &xr, &xi);
  const int ex = eA[(size_t)k * n + r] + eB[(size_t)k * b + i];
  Y[(size_t)k * n * b + idx] = zmake(ldexp(xr, ex), ldexp(xi, ex));
}

}  // namespace

int bs_launch_fields_tc(bs_cell* c, cudaStream_t s) {
  const int P = c->P, D = c->D, S = BS_SLICES_ASM, Kp = (P + 63) / 64 * 64, nf = c->nf;
  SliceSlabs sl;
  if (!bs_slice_slabs(S, Kp, nf * P, 2 * D, 1, &sl)) {
    bs_set_error("form factors: P = %d gives too many digit slabs", P);
    return BS_EINVAL;
  }
  pack_fields_kernel<<<dim3(P, nf), 128, 0, s>>>(c->d_phase, c->d_table, c->nphase, P, S, Kp,
                                                 c->d_sliceA, c->d_expA);
  BS_CHECK_LAUNCH("pack_fields_kernel");
  pack_exp_kernel<<<2 * D, 128, 0, s>>>(c->d_E, P, D, S, Kp, c->d_sliceB, c->d_expB);
  BS_CHECK_LAUNCH("pack_exp_kernel");
  bs_phase_begin(c, PH_ASM_TC, s);
  TRY_LAUNCH(bs_launch_slice_orders(c->d_sliceA, c->d_sliceB, c->d_sliceD, nf * P, 2 * D, S, Kp, 1,
                                    c->d_info + 1, s));
  bs_phase_end(c, PH_ASM_TC, s);
  const size_t tot = (size_t)nf * P * D;
  recombine_fields_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
      c->d_sliceD, sl, c->d_expA, c->d_expB, P, D, nf, c->d_Y);
  BS_CHECK_LAUNCH("recombine_fields_kernel");
  return BS_OK;
}

size_t bs_fields_tc_elems(int P, int D, int nf, size_t* nA, size_t* nB, size_t* nD) {
  const int S = BS_SLICES_ASM, Kp = (P + 63) / 64 * 64;
  *nA = (size_t)nf * P * S * Kp;
  *nB = (size_t)2 * D * S * Kp;
  *nD = bs_slice_planes(S, Kp, nf * P, 2 * D, 1) * nf * P * 2 * D;
  return *nA + *nB;
}

int bs_launch_cx_tc(const zd* C, const zd* X, int n, int b, int kb, uint16_t* sA, uint16_t* sB,
                    float* sD, int* eA, int* eB, zd* Y, int* err, cudaStream_t s) {
  const int S = BS_SLICES_RR, Kp = (2 * n + 63) / 64 * 64;
  SliceSlabs sl;
  if (!bs_slice_slabs(S, Kp, n, 2 * b, kb, &sl)) {
    bs_set_error("C X product: n = %d gives too many digit slabs", n);
    return BS_EINVAL;
  }
  pack_cmat_kernel<<<dim3(n, kb), 128, 0, s>>>(C, n, S, Kp, sA, eA);
  BS_CHECK_LAUNCH("pack_cmat_kernel");
  pack_xmat_kernel<<<dim3(b, kb), 128, 0, s>>>(X, n, b, S, Kp, sB, eB);
  BS_CHECK_LAUNCH("pack_xmat_kernel");
  TRY_LAUNCH(bs_launch_slice_orders(sA, sB, sD, n, 2 * b, S, Kp, kb, err, s));
  recombine_cx_kernel<<<dim3((n * b + 255) / 256, kb), 256, 0, s>>>(sD, sl, eA, eB,
                                                                               n, b, Y);
  BS_CHECK_LAUNCH("recombine_cx_kernel");
  return BS_OK;
}

void bs_cx_tc_elems(int n, int b, int kb, size_t* nA, size_t* nB, size_t* nD) {
  const int S = BS_SLICES_RR, Kp = (2 * n + 63) / 64 * 64;
  *nA = (size_t)kb * n * S * Kp;
  *nB = (size_t)kb * 2 * b * S * Kp;
  *nD = bs_slice_planes(S, Kp, n, 2 * b, kb) * n * 2 * b;
}

// ---- complex N x N products C = A diag(sc) B^dagger (column-major, FP64)
//   Re C = [Ar sc | Ai sc] [Br | Bi]^T,  Im C = [Ar sc | Ai sc] [-Bi | Br]^T
// A rows r; B rows (c, part), digits reversed; K = 2N.
namespace {

__global__ void pack_zrows_kernel(const zd* __restrict__ A, long sA, const double* __restrict__ sc,
                                  int N, int S, int Kp, int parts, int reversed,
                                  uint16_t* __restrict__ out, int* __restrict__ ex) {
  // one CTA (128 threads) per row: the digit planes are written along K
  __shared__ double sh[4];
  const int r = blockIdx.x, z = blockIdx.y;
  const zd* a = A + (size_t)z * sA;
  double m = 0.0;
  for (int k = threadIdx.x; k < N; k += 128) {
    zd v = a[r + (size_t)k * N];
    if (sc) v = zscale(v, sc[k]);
    m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
  }
  const int e = row_exp(row_max(m, sh));
  const size_t rows = (size_t)parts * N, rowlen = (size_t)S * Kp;
  uint16_t* base = out + ((size_t)z * rows + (size_t)r * parts) * rowlen +
                   (reversed ? (size_t)(S - 1) * Kp : 0);
  const ptrdiff_t plane = reversed ? -(ptrdiff_t)Kp : (ptrdiff_t)Kp;
  for (int k = threadIdx.x; k < Kp; k += 128) {
    double v0 = 0.0, v1 = 0.0;
    if (k < 2 * N) {
      const int kk = k < N ? k : k - N;
      zd v = a[r + (size_t)kk * N];
      if (sc) v = zscale(v, sc[kk]);
      if (k < N) {          // part 0: [re | im], part 1: [-im | re]
        v0 = v.x;
        v1 = -v.y;
      } else {
        v0 = v.y;
        v1 = v.x;
      }
    }
    put_digits(v0, e, S, base + k, plane);
    if (parts == 2) put_digits(v1, e, S, base + rowlen + k, plane);
  }
  if (threadIdx.x == 0) ex[(size_t)z * N + r] = e;
}

__global__ void recombine_z_kernel(const float* __restrict__ Dm, const SliceSlabs sl,
                                   const int* __restrict__ eA, const int* __restrict__ eB, int N,
                                   zd* __restrict__ C, long sC) {
  const int z = blockIdx.y;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N * N) return;
  const int r = idx % N, c = idx / N;
  const size_t M = (size_t)N, Nn = 2 * (size_t)N;
  const float* dz = Dm + (size_t)z * sl.nq * Nn * M;
  double xr, xi;
  order_sums(dz, Nn * M, (2 * (size_t)c) * M + r, (2 * (size_t)c + 1) * M + r, sl, &xr, &xi);
  const int ex = eA[(size_t)z * N + r] + eB[(size_t)z * N + c];
  C[(size_t)z * sC + idx] = zmake(ldexp(xr, ex), ldexp(xi, ex));
}

}  // namespace

void bs_zgemm_tc_elems(int N, int batch, size_t* nA, size_t* nB, size_t* nD) {
  const int S = BS_SLICES_ASM, Kp = (2 * N + 63) / 64 * 64;
  *nA = (size_t)batch * N * S * Kp;
  *nB = (size_t)batch * 2 * N * S * Kp;
  *nD = bs_slice_planes(S, Kp, N, 2 * N, batch) * N * 2 * N;
}

int bs_launch_zgemm_tc(const zd* A, long sA, const double* sc, const zd* B, long sB, zd* C, long sC,
                       int N, int batch, uint16_t* wA, uint16_t* wB, float* wD, int* eA, int* eB,
                       int* err, cudaStream_t s) {
  const int S = BS_SLICES_ASM, Kp = (2 * N + 63) / 64 * 64;
  SliceSlabs sl;
  if (2 * N > 4096 || !bs_slice_slabs(S, Kp, N, 2 * N, batch, &sl)) {
    bs_set_error("complex product: 2N = %d exceeds the exact-slice limit 4096", 2 * N);
    return BS_EINVAL;
  }
  const dim3 g(N, batch);
  pack_zrows_kernel<<<g, 128, 0, s>>>(A, sA, sc, N, S, Kp, 1, 0, wA, eA);
  BS_CHECK_LAUNCH("pack_zrows_kernel A");
  pack_zrows_kernel<<<g, 128, 0, s>>>(B, sB, nullptr, N, S, Kp, 2, 1, wB, eB);
  BS_CHECK_LAUNCH("pack_zrows_kernel B");
  TRY_LAUNCH(bs_launch_slice_orders(wA, wB, wD, N, 2 * N, S, Kp, batch, err, s));
  recombine_z_kernel<<<dim3((N * N + 255) / 256, batch), 256, 0, s>>>(
      wD, sl, eA, eB, N, C, sC);
  BS_CHECK_LAUNCH("recombine_z_kernel");
  return BS_OK;
}
