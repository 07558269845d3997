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

// BF16 bits of a small integer (|t| <= 256, exact): t is added to the bit
// pattern of 1.5 2^23, whose unit in the last place is 1, and 1.5 2^23 is
// subtracted again, so the conversion runs on the FP32 pipe instead of the
// conversion unit; the BF16 value is the top half of the FP32 one
__device__ __forceinline__ uint16_t bf16_bits(long long t) {
  const float f = __int_as_float(0x4B400000 + (int)t) - 12582912.0f;
  return (uint16_t)(__float_as_uint(f) >> 16);
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
// slow on GB300): with B = 6 + 7 (S - 1) bits (48 for seven digits, 55 for
// eight, enough for the whole FP64 mantissa of every x within a factor 4
// of the row scale), X = round(x 2^(B-e)) as a signed 64-bit integer
// (|X| <= 2^B), then t_0 = floor((X + 2^(B-7)) / 2^(B-6)), remainder r, and
// t_s = floor((r + 2^(B-7-7s)) / 2^(B-6-7s)) for s >= 1 (the last digit is
// the remainder itself), each in [-64, 64].  Digit s goes to
// out[s * plane] (plane < 0 for the reversed B layout).
__device__ __forceinline__ void put_digits(double x, int e, int S, uint16_t* out,
                                           ptrdiff_t plane) {
  const int B = 6 + 7 * (S - 1);
  const long long bits = __double_as_longlong(x);
  const int E = (int)((bits >> 52) & 0x7FF);
  long long X = 0;
  if (E != 0) {
    const long long m = (bits & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
    const int sh = 1075 - E - B + e;    // X = m 2^-sh; |x| <= 2^e keeps sh >= 52 - B
    if (sh <= 0) X = m << (-sh);
    else if (sh < 63) X = (m + (1LL << (sh - 1))) >> sh;
    if (bits < 0) X = -X;
  }
  long long r = X;
  for (int s = 0; s < S; ++s) {
    const int sh = B - 6 - 7 * s;
    long long t;
    if (sh > 0) t = (r + (1LL << (sh - 1))) >> sh;
    else t = r;
    r -= t << (sh > 0 ? sh : 0);
    out[(ptrdiff_t)s * plane] = bf16_bits(t);
  }
}

// The eight-digit split of the band reduction, in 32-bit integer arithmetic:
// X = round(x 2^(55-e)) (as in put_digits, |X| <= 2^55) is cut into
// X = Xh 2^28 + Xl with 0 <= Xl < 2^28; the four low digits are balanced
// radix-128 digits of Xl from the bottom, d = ((v + 64) mod 128) - 64 in
// [-64, 63], whose final carry (0 or 1) joins Xh, and three more come from
// Xh the same way; the top digit is what remains (|t_0| <= 64).  The digits
// represent X exactly, so every digit product stays an integer of at most
// 2^12, as for put_digits.
template <int S>
__device__ __forceinline__ void put_digits_t(double x, int e, uint16_t* out, ptrdiff_t plane) {
  static_assert(S == 8, "the 32-bit split is written for eight digits");
  constexpr int B = 6 + 7 * (S - 1);
  const long long bits = __double_as_longlong(x);
  const int E = (int)((bits >> 52) & 0x7FF);
  long long X = 0;
  if (E != 0) {
    const long long m = (bits & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
    const int sh = 1075 - E - B + e;
    if (sh <= 0) X = m << (-sh);
    else if (sh < 63) X = (m + (1LL << (sh - 1))) >> sh;
    if (bits < 0) X = -X;
  }
  int u = (int)(X >> 28);
  int v = (int)(X & 0xFFFFFFF);
#pragma unroll
  for (int sd = S - 1; sd >= 4; --sd) {
    const int d = ((v + 64) & 127) - 64;
    v = (v - d) >> 7;
    out[(ptrdiff_t)sd * plane] = bf16_bits(d);
  }
  u += v;
#pragma unroll
  for (int sd = 3; sd >= 1; --sd) {
    const int d = ((u + 64) & 127) - 64;
    u = (u - d) >> 7;
    out[(ptrdiff_t)sd * plane] = bf16_bits(d);
  }
  out[0] = bf16_bits(u);
}

// Row scale by integer arithmetic: for non-negative doubles the bit
// patterns order as the values do, so the largest |x| is the largest of
// (bits & ~sign) as 64-bit integers, and frexp's exponent of it is the
// exponent field less 1022 (0 for a zero row, as row_exp gives).
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFULL;
}
__device__ __forceinline__ unsigned long long warp_umax(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}
// block-wide: blockDim.x == 32 * nw, sh holds nw entries
__device__ int row_exp_bits(unsigned long long v, unsigned long long* sh, int nw) {
  v = warp_umax(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  unsigned long long m = 0;
  for (int w = 0; w < nw; ++w) m = sh[w] > m ? sh[w] : m;
  __syncthreads();
  const int E = (int)(m >> 52);
  return m == 0 ? 0 : E - 1022;
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

// ---- complex products C = A diag(sc) B^dagger (column-major, FP64): A is
// M x K, B is Nc x K, C is M x Nc
//   Re C = [Ar sc | Ai sc] [Br | Bi]^T,  Im C = [Ar sc | Ai sc] [-Bi | Br]^T
// A rows r; B rows (c, part), digits reversed; the contraction runs over 2K.
namespace {

__global__ void pack_zrows_kernel(const zd* __restrict__ A, int ld, long sA,
                                  const double* __restrict__ sc, int R, int K, int S, int Kp,
                                  int parts, int reversed, uint16_t* __restrict__ out,
                                  int* __restrict__ ex) {
  // one CTA (128 threads) per row r < R of the operand: the digit planes are
  // written along K
  __shared__ double sh[4];
  const int r = blockIdx.x, z = blockIdx.y;
  const zd* a = A + (size_t)z * sA;
  double m = 0.0;
  for (int k = threadIdx.x; k < K; k += 128) {
    zd v = a[r + (size_t)k * ld];
    if (sc) v = zscale(v, sc[k]);
    m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
  }
  const int e = row_exp(row_max(m, sh));
  const size_t rows = (size_t)parts * R, rowlen = (size_t)S * Kp;
  uint16_t* base = out + ((size_t)z * rows + (size_t)r * parts) * rowlen +
                   (reversed ? (size_t)(S - 1) * Kp : 0);
  const ptrdiff_t plane = reversed ? -(ptrdiff_t)Kp : (ptrdiff_t)Kp;
  for (int k = threadIdx.x; k < Kp; k += 128) {
    double v0 = 0.0, v1 = 0.0;
    if (k < 2 * K) {
      const int kk = k < K ? k : k - K;
      zd v = a[r + (size_t)kk * ld];
      if (sc) v = zscale(v, sc[kk]);
      if (k < K) {          // part 0: [re | im], part 1: [-im | re]
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
  if (threadIdx.x == 0) ex[(size_t)z * R + r] = e;
}

__global__ void recombine_z_kernel(const float* __restrict__ Dm, const SliceSlabs sl,
                                   const int* __restrict__ eA, const int* __restrict__ eB, int M,
                                   int Nc, zd* __restrict__ C, int ldc, long sC) {
  const int z = blockIdx.y;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * Nc) return;
  const int r = idx % M, c = idx / M;
  const size_t Mz = (size_t)M, Nn = 2 * (size_t)Nc;
  const float* dz = Dm + (size_t)z * sl.nq * Nn * Mz;
  double xr, xi;
  order_sums(dz, Nn * Mz, (2 * (size_t)c) * Mz + r, (2 * (size_t)c + 1) * Mz + r, sl, &xr, &xi);
  const int ex = eA[(size_t)z * M + r] + eB[(size_t)z * Nc + c];
  C[(size_t)z * sC + r + (size_t)c * ldc] = zmake(ldexp(xr, ex), ldexp(xi, ex));
}

}  // namespace

bool bs_zgemm_tc_fits(int K) { return K >= 1 && 2 * K <= 4096; }

void bs_zgemm_tc_rect_elems(int M, int Nc, int K, int batch, size_t* nA, size_t* nB,
                            size_t* nD) {
  const int S = BS_SLICES_ASM, Kp = (2 * K + 63) / 64 * 64;
  *nA = (size_t)batch * M * S * Kp;
  *nB = (size_t)batch * 2 * Nc * S * Kp;
  *nD = bs_slice_planes(S, Kp, M, 2 * Nc, batch) * M * 2 * Nc;
}

void bs_zgemm_tc_elems(int N, int batch, size_t* nA, size_t* nB, size_t* nD) {
  bs_zgemm_tc_rect_elems(N, N, N, batch, nA, nB, nD);
}

int bs_launch_zgemm_tc_rect(const zd* A, int lda, long sA, const double* sc, const zd* B, int ldb,
                            long sB, zd* C, int ldc, long sC, int M, int Nc, int K, int batch,
                            uint16_t* wA, uint16_t* wB, float* wD, int* eA, int* eB, int* err,
                            cudaStream_t s) {
  const int S = BS_SLICES_ASM, Kp = (2 * K + 63) / 64 * 64;
  SliceSlabs sl;
  if (!bs_zgemm_tc_fits(K) || M < 1 || Nc < 1 || lda < M || ldb < Nc || ldc < M ||
      !bs_slice_slabs(S, Kp, M, 2 * Nc, batch, &sl)) {
    bs_set_error("complex product: 2K = %d exceeds the exact-slice limit 4096", 2 * K);
    return BS_EINVAL;
  }
  pack_zrows_kernel<<<dim3(M, batch), 128, 0, s>>>(A, lda, sA, sc, M, K, S, Kp, 1, 0, wA, eA);
  BS_CHECK_LAUNCH("pack_zrows_kernel A");
  pack_zrows_kernel<<<dim3(Nc, batch), 128, 0, s>>>(B, ldb, sB, nullptr, Nc, K, S, Kp, 2, 1, wB,
                                                    eB);
  BS_CHECK_LAUNCH("pack_zrows_kernel B");
  TRY_LAUNCH(bs_launch_slice_orders(wA, wB, wD, M, 2 * Nc, S, Kp, batch, err, s));
  recombine_z_kernel<<<dim3((unsigned)(((size_t)M * Nc + 255) / 256), batch), 256, 0, s>>>(
      wD, sl, eA, eB, M, Nc, C, ldc, sC);
  BS_CHECK_LAUNCH("recombine_z_kernel");
  return BS_OK;
}

int bs_launch_zgemm_tc(const zd* A, long sA, const double* sc, const zd* B, long sB, zd* C, long sC,
                       int N, int batch, uint16_t* wA, uint16_t* wB, float* wD, int* eA, int* eB,
                       int* err, cudaStream_t s) {
  return bs_launch_zgemm_tc_rect(A, N, sA, sc, B, N, sB, C, N, sC, N, N, N, batch, wA, wB, wD, eA,
                                 eB, err, s);
}

// ---- the two contractions of a dense-to-band reduction step
// (band.cu): X = A22 V with A22 the Hermitian trailing block of A (full
// storage, m x m at offset o, leading dimension n), and the two-sided
// update A22 -= V W^dagger + W V^dagger.
namespace {

// A rows r of [Re A22[r, :] | Im A22[r, :]], read as the conjugate of
// column r (eight digits); grid (m, kb), block 128
__global__ void pack_trail_kernel(const zd* __restrict__ A, int n, int o, int m, int Kp,
                                  uint16_t* __restrict__ out, int* __restrict__ ex) {
  constexpr int S = 8;
  __shared__ unsigned long long sh[4];
  const int r = blockIdx.x, k = blockIdx.y, t = threadIdx.x;
  const zd* col = A + (size_t)k * n * n + (size_t)(o + r) * n + o;
  unsigned long long mx = 0;
  for (int c = t; c < m; c += 128) {
    const zd v = col[c];
    const unsigned long long a = abs_bits(v.x), b = abs_bits(v.y);
    mx = a > mx ? a : mx;
    mx = b > mx ? b : mx;
  }
  const int e = row_exp_bits(mx, sh, 4);
  uint16_t* base = out + ((size_t)k * m + r) * S * Kp;
  for (int c = t; c < m; c += 128) {
    const zd v = col[c];
    put_digits_t<S>(v.x, e, base + c, Kp);
    // Im A22[r, c] = -Im A22[c, r]: a sign flip of the bit pattern
    put_digits_t<S>(__longlong_as_double(__double_as_longlong(v.y) ^ (1LL << 63)), e,
                    base + m + c, Kp);
  }
  for (int c = 2 * m + t; c < Kp; c += 128)
#pragma unroll
    for (int sd = 0; sd < S; ++sd) base[(size_t)sd * Kp + c] = 0;
  if (t == 0) ex[(size_t)k * m + r] = e;
}

// B rows (i, part) of the m x nb block V (leading dimension ldv, batch
// stride sv), digits reversed: part 0 = [Vr; -Vi], part 1 = [Vi; Vr];
// grid (nb, kb), block 128
__global__ void pack_panel_kernel(const zd* __restrict__ V, int ldv, long sv, int m, int nb,
                                  int S, int Kp, uint16_t* __restrict__ out,
                                  int* __restrict__ ex) {
  __shared__ double sh[4];
  const int i = blockIdx.x, k = blockIdx.y;
  const zd* x = V + (size_t)k * sv + (size_t)i * ldv;
  double mx = 0.0;
  for (int r = threadIdx.x; r < m; r += 128) mx = fmax(mx, fmax(fabs(x[r].x), fabs(x[r].y)));
  const int e = row_exp(row_max(mx, sh));
  uint16_t* base0 = out + ((size_t)k * 2 * nb + 2 * i) * S * Kp + (size_t)(S - 1) * Kp;
  uint16_t* base1 = base0 + (size_t)S * Kp;
  for (int c = threadIdx.x; c < Kp; c += 128) {
    double v0 = 0.0, v1 = 0.0;
    if (c < m) {
      v0 = x[c].x;
      v1 = x[c].y;
    } else if (c < 2 * m) {
      v0 = -x[c - m].y;
      v1 = x[c - m].x;
    }
    put_digits(v0, e, S, base0 + c, -(ptrdiff_t)Kp);
    put_digits(v1, e, S, base1 + c, -(ptrdiff_t)Kp);
  }
  if (threadIdx.x == 0) ex[(size_t)k * nb + i] = e;
}

// X[k][r + i ldx] = 2^(eA + eB) sum_u 2^(-12-7u) (slabs of order u)[(i, part)][r]
__global__ void recombine_panel_kernel(const float* __restrict__ Dm, const SliceSlabs sl,
                                       const int* __restrict__ eA, const int* __restrict__ eB,
                                       int m, int nb, zd* __restrict__ X, int ldx, long sx) {
  const int k = blockIdx.y;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * nb) return;
  const int r = idx % m, i = idx / m;
  const size_t M = (size_t)m, Nn = 2 * (size_t)nb;
  const float* dk = Dm + (size_t)k * sl.nq * Nn * M;
  double xr, xi;
  order_sums(dk, Nn * M, (2 * (size_t)i) * M + r, (2 * (size_t)i + 1) * M + r, sl, &xr, &xi);
  const int e = eA[(size_t)k * m + r] + eB[(size_t)k * nb + i];
  X[(size_t)k * sx + (size_t)i * ldx + r] = zmake(ldexp(xr, e), ldexp(xi, e));
}

// Operands of the rank-2nb update V W^dagger + W V^dagger = X Y^dagger with
// X = [V D, W D^-1], Y = [W D^-1, V D] (m x 2nb), D = diag(2^d_i) a
// power-of-two balance of column i of V (entries at most 1) against
// column i of W (of the size of the matrix norm), d_i half the difference
// of their largest exponents (ecol: kb x [V | W] x nb exponent fields), so
// that one row scale serves both halves of a row without starving V of
// digits:
// A rows r = [Re X[r, :] | Im X[r, :]], B rows (c, 0) = [Re Y[c, :] | Im Y[c, :]],
// (c, 1) = [-Im Y[c, :] | Re Y[c, :]], K = 4 nb <= 64 (one 64-column block).
// Row r of X and of Y hold the same numbers, so one exponent serves both,
// and entries (r, c) and (c, r) of the product come from the same digits.
// The scaling only shifts the digit exponents (no rounding); grid (m, kb),
// block 64
__global__ void pack_rank2_kernel(const zd* __restrict__ V, const zd* __restrict__ W, int ld,
                                  long sv, const int* __restrict__ ecol, int m, int nb, int S,
                                  uint16_t* __restrict__ oa, uint16_t* __restrict__ ob,
                                  int* __restrict__ ex) {
  __shared__ double sh[2];
  const int r = blockIdx.x, k = blockIdx.y, t = threadIdx.x;
  const zd* vk = V + (size_t)k * sv;
  const zd* wk = W + (size_t)k * sv;
  const int w2 = 2 * nb;
  // column t of A: t < 2nb -> Re X[r, t], t < 4nb -> Im X[r, t - 2nb]
  double a = 0.0, y0 = 0.0, y1 = 0.0;
  int shx = 0, shy = 0;   // exponents of the balance of the X and Y entries
  if (t < 2 * w2) {
    const int c = t < w2 ? t : t - w2;
    const int ci = c < nb ? c : c - nb;
    const int ev = ecol[(size_t)k * 2 * nb + ci], ew = ecol[(size_t)k * 2 * nb + nb + ci];
    const int d = (ev > 0 && ew > 0) ? (ew - ev) / 2 : 0;
    shx = c < nb ? d : -d;
    shy = -shx;
    const zd xv = c < nb ? vk[(size_t)c * ld + r] : wk[(size_t)(c - nb) * ld + r];
    const zd yv = c < nb ? wk[(size_t)c * ld + r] : vk[(size_t)(c - nb) * ld + r];
    if (t < w2) {
      a = xv.x;
      y0 = yv.x;
      y1 = -yv.y;
    } else {
      a = xv.y;
      y0 = yv.y;
      y1 = yv.x;
    }
  }
  double mx = warp_max(fabs(a) * pow2(shx));
  if ((t & 31) == 0) sh[t >> 5] = mx;
  __syncthreads();
  mx = fmax(sh[0], sh[1]);
  const int e = row_exp(mx);
  const size_t rowlen = (size_t)S * 64;
  put_digits_t<8>(a, e - shx, oa + ((size_t)k * m + r) * rowlen + t, 64);
  uint16_t* b0 = ob + ((size_t)k * 2 * m + 2 * (size_t)r) * rowlen + (size_t)(S - 1) * 64 + t;
  put_digits_t<8>(y0, e - shy, b0, -64);
  put_digits_t<8>(y1, e - shy, b0 + rowlen, -64);
  if (t == 0) ex[(size_t)k * m + r] = e;
}

}  // namespace

void bs_band_tc_elems(int n, int nb, int kb, int S, size_t* nA, size_t* nB, size_t* nD,
                      size_t* nE) {
  const int m = n - nb > 1 ? n - nb : 1, Kp = (2 * m + 63) / 64 * 64;
  const size_t aA = (size_t)kb * m * S * Kp, aB = (size_t)kb * 2 * nb * S * Kp;
  const size_t hA = (size_t)kb * m * S * 64, hB = (size_t)kb * 2 * m * S * 64;
  *nA = aA > hA ? aA : hA;
  *nB = aB > hB ? aB : hB;
  // the largest trailing block needs the most planes; smaller ones may cut
  // their slabs finer, so take the maximum over the sizes a reduction visits
  size_t d = 0;
  for (int mm = m; mm > 1; mm -= nb) {
    const int kp = (2 * mm + 63) / 64 * 64;
    const size_t pa = bs_slice_planes(S, kp, mm, 2 * nb, kb) * mm * 2 * nb;
    d = d > pa ? d : pa;
  }
  *nD = d;
  *nE = (size_t)kb * (m + 2 * nb);
}

// the digit planes of the trailing block (rows and columns from o on)
int bs_launch_band_pack_trail(const zd* A, int n, int o, int m, int kb, uint16_t* wA, int* eA,
                              cudaStream_t s) {
  const int Kp = (2 * m + 63) / 64 * 64;
  pack_trail_kernel<<<dim3(m, kb), 128, 0, s>>>(A, n, o, m, Kp, wA, eA);
  BS_CHECK_LAUNCH("pack_trail_kernel");
  return BS_OK;
}

// X = A22 V from the trailing block's digit planes (bs_launch_band_pack_trail)
int bs_launch_band_av(int m, const zd* V, int ldv, long sv, int nb, int kb, int S, uint16_t* wA,
                      uint16_t* wB, float* wD, int* eA, int* eB, zd* X, int ldx, long sx,
                      int* err, cudaStream_t s) {
  const int Kp = (2 * m + 63) / 64 * 64;
  SliceSlabs sl;
  if (S != 8 || !bs_slice_slabs(S, Kp, m, 2 * nb, kb, &sl)) {
    bs_set_error("band reduction: m = %d gives too many digit slabs", m);
    return BS_EINVAL;
  }
  pack_panel_kernel<<<dim3(nb, kb), 128, 0, s>>>(V, ldv, sv, m, nb, S, Kp, wB, eB);
  BS_CHECK_LAUNCH("pack_panel_kernel");
  TRY_LAUNCH(bs_launch_slice_orders(wA, wB, wD, m, 2 * nb, S, Kp, kb, err, s));
  recombine_panel_kernel<<<dim3((m * nb + 255) / 256, kb), 256, 0, s>>>(wD, sl, eA, eB, m, nb, X,
                                                                       ldx, sx);
  BS_CHECK_LAUNCH("recombine_panel_kernel");
  return BS_OK;
}

// the digit planes of the rank-2nb update's operands [V D, W D^-1], [W D^-1, V D]
int bs_launch_band_pack_rank2(const zd* V, const zd* W, int ld, long sv, const int* dsc, int m,
                              int nb, int kb, int S, uint16_t* wA, uint16_t* wB, int* ex,
                              cudaStream_t s) {
  if (S != 8 || 4 * nb > 64) {
    bs_set_error("band reduction: needs 8 digits and band width <= 16 (nb = %d)", nb);
    return BS_EINVAL;
  }
  pack_rank2_kernel<<<dim3(m, kb), 64, 0, s>>>(V, W, ld, sv, dsc, m, nb, S, wA, wB, ex);
  BS_CHECK_LAUNCH("pack_rank2_kernel");
  return BS_OK;
}
