// Two-stage reduction of batched Hermitian matrices to real tridiagonal
// form, for the FP64 eigensolve of Eq. (eigenvalueproblem) once the pencil
// is in standard form C(k) u = lambda u.
//
// The one-stage Householder reduction (tridiag.cu) spends half of its
// (16/3) n^3 flops in a matrix-vector product per column, so it stays on
// the FP64 pipe, which GB300 runs at 2 FMA per clock per SM.  Here the
// O(n^3) work becomes matrix-matrix products for the tensor cores:
//
//  stage 1, dense -> band of half-width nb (nb = 8): for the panel of
//    columns j .. j+nb-1, a Householder QR of its m x nb block below the
//    band, P = Q R with Q = I - V T V^dagger (compact WY, T upper
//    triangular), puts R in the band; the trailing block is updated as
//    Q^dagger A22 Q = A22 - V W^dagger - W V^dagger with
//      Y = A22 V T,  Z = V^dagger Y,  W = Y - (1/2) V T^dagger Z.
//    A22 V and the rank-2nb update run as exact-slice digit-plane
//    contractions on tcgen05 (slices.cu), the QR and W in FP64;
//  stage 2, band -> tridiagonal by bulge chasing: sweep s annihilates
//    column s below its subdiagonal with a reflector of length nb, applies
//    it on both sides of the next diagonal block, and chases the bulge it
//    makes one block further down with a new reflector per block.  One CTA
//    per matrix, eight lanes per sweep in flight: sweep s + 1 starts three
//    blocks behind sweep s, so the blocks that the sweeps touch in one step
//    are disjoint, and a block-wide barrier separates the steps.
//
// The unitary similarity keeps the eigenvalues; the tridiagonal is returned
// as (d, |e|) for the Sturm multisection (bisect.cu).
#include <algorithm>
#include <atomic>

#include "bs_internal.h"

namespace {

constexpr int QR_NT = 256;   // threads of the W kernels
constexpr int PQ_NT = 256;   // threads of the panel QR (512 measured 9 % slower)
constexpr int LAG = 3;       // blocks between consecutive sweeps

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------- symmetrise
// Upper triangle <- conjugate of the lower one, real diagonal; the builders
// write the lower triangle only.  32 x 32 tiles through shared memory.
__global__ void symmetrize_kernel(zd* __restrict__ A, int n) {
  __shared__ zd tile[32][33];
  const int bi = blockIdx.x, bj = blockIdx.y;
  if (bi < bj) return;
  zd* a = A + (size_t)blockIdx.z * n * n;
  const int x = threadIdx.x;
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int r = bi * 32 + x, c = bj * 32 + y;   // lower tile element (r, c)
    if (r < n && c < n) tile[y][x] = a[r + (size_t)c * n];
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int r = bj * 32 + x, c = bi * 32 + y;   // upper element (r, c) = conj(A[c, r])
    if (r < n && c < n) {
      if (r < c) {
        const zd v = tile[x][y];
        a[r + (size_t)c * n] = zconj(v);
      } else if (r == c) {
        a[r + (size_t)c * n].y = 0.0;
      }
    }
  }
}

// ---------------------------------------------------------------- panel QR
// Block-wide sum of NV complex values held by every thread of an NT-thread
// block; the result is left in out[0 .. NV).  sh: NV x (NT/32) zd.
template <int NV, int NT>
__device__ void block_zsum(zd (&v)[NV], zd* sh, zd* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    v[q].x = warp_sum_d(v[q].x);
    v[q].y = warp_sum_d(v[q].y);
  }
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[q * (NT / 32) + warp] = v[q];
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    zd t = zmake(0.0, 0.0);
    for (int w = 0; w < NT / 32; ++w) t = zadd(t, sh[threadIdx.x * (NT / 32) + w]);
    out[threadIdx.x] = t;
  }
  __syncthreads();
}

// Householder QR of the panel A[j+NB : n, j : j+NB] (m x NB) of every
// matrix of the batch, in shared memory.  Thread t owns rows t, t + PQ_NT,
// ... of the panel throughout.  Writes R (upper triangle) and zeros below
// it back into the panel, V (m x NB, unit lower trapezoidal, leading
// dimension ldv) and T (NB x NB upper triangular, column-major).
//
// One block reduction per column i: with x = P[i][i:] and v = [1; x[i+1:] s]
// (s = 1 / (x_i - beta)), every sum the step needs is a sum over the rows
// below i of quantities known before beta,
//   ||x[i+1:]||^2,  y_c = x[i+1:]^dagger P[c][i+1:] (c > i),
//   g_q = v_q[i+1:]^dagger x[i+1:] (q < i),
// and then v^dagger P[c] = P[c][i] + conj(s) y_c, v_q^dagger v = conj(v_q[i])
// + s g_q.  The reflector scalars come from two reciprocal square roots and
// one division, and the column of T of each reflector (T[0:i, i] =
// -tau_i T[0:i, 0:i] G[0:i, i], G[q][i] = v_q^dagger v_i) is formed right
// after its reduction by i threads at once.
template <int NB>
__global__ void __launch_bounds__(PQ_NT) panel_qr_kernel(zd* __restrict__ A, int n, int j,
                                                         zd* __restrict__ V, int ldv, long sv,
                                                         zd* __restrict__ T) {
  extern __shared__ zd P[];   // [NB][m]
  __shared__ zd red[NB * (PQ_NT / 32)];
  __shared__ zd dots[NB];
  __shared__ zd rowi[NB];     // row i of the panel, P[c][i]
  __shared__ zd Ts[NB * NB];  // T, column-major
  __shared__ zd beta_s[NB];
  const int k = blockIdx.x, tid = threadIdx.x;
  const int m = n - j - NB;
  zd* a = A + (size_t)k * n * n;
  for (int idx = tid; idx < NB * m; idx += PQ_NT) {
    const int i = idx / m, r = idx % m;
    P[idx] = a[(size_t)(j + i) * n + j + NB + r];
  }
  for (int idx = tid; idx < NB * NB; idx += PQ_NT) Ts[idx] = zmake(0.0, 0.0);
  __syncthreads();
  const int kk = min(NB, m - 1);   // reflectors of length >= 2
  for (int i = 0; i < kk; ++i) {
    zd* pi = P + (size_t)i * m;
    if (tid == i) {
#pragma unroll
      for (int c = 0; c < NB; ++c) rowi[c] = P[(size_t)c * m + i];
    }
    // acc[0]: ||x[i+1:]||^2; acc[q] (1 <= q <= i): g_{q-1}; acc[c] (c > i): y_c
    zd acc[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) acc[q] = zmake(0.0, 0.0);
    for (int r = tid; r < m; r += PQ_NT) {
      if (r <= i) continue;
      const zd x = pi[r];
      acc[0].x = fma(x.x, x.x, fma(x.y, x.y, acc[0].x));
#pragma unroll
      for (int q = 1; q < NB; ++q) {
        if (q <= i)
          acc[q] = zfmac(x, P[(size_t)(q - 1) * m + r], acc[q]);   // conj(v_{q-1}[r]) x[r]
        else
          acc[q] = zfmac(P[(size_t)q * m + r], x, acc[q]);         // conj(x[r]) P[q][r]
      }
    }
    block_zsum<NB, PQ_NT>(acc, red, dots);
    const zd alpha = rowi[i];
    const double a2 = fma(alpha.x, alpha.x, alpha.y * alpha.y), s2 = a2 + dots[0].x;
    double tau = 0.0;
    zd beta = zmake(0.0, 0.0), scl = zmake(0.0, 0.0);
    if (s2 > 0.0) {
      const double rn = rsqrt(s2), nu = s2 * rn;
      if (a2 > 0.0) {
        const double ra = rsqrt(a2), aa = a2 * ra;
        beta = zscale(alpha, -nu * ra);
        tau = (aa + nu) * rn;
        // 1 / (alpha - beta) = conj(alpha) / (|alpha| (|alpha| + nu))
        scl = zscale(zconj(alpha), ra / (aa + nu));
      } else {
        beta = zmake(-nu, 0.0);
        tau = 1.0;
        scl = zmake(rn, 0.0);
      }
    }
    if (tid == 0) {
      beta_s[i] = beta;
      Ts[i + i * NB] = zmake(tau, 0.0);
    }
    if (tid < i) {
      // T[tid][i] = -tau sum_{q = tid}^{i-1} T[tid][q] G[q][i]
      zd t = zmake(0.0, 0.0);
      for (int q = tid; q < i; ++q) {
        const zd g = zfma(scl, dots[q + 1], zconj(rowi[q]));
        t = zfma(Ts[tid + q * NB], g, t);
      }
      Ts[tid + i * NB] = zscale(t, -tau);
    }
    // P[c] -= tau v (v^dagger P[c]) for c > i, v stored below the diagonal
    zd tz[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c)
      tz[c] = c > i ? zscale(zfmac(dots[c], scl, rowi[c]), tau) : zmake(0.0, 0.0);
    for (int r = tid; r < m; r += PQ_NT) {
      if (r < i) continue;
      zd vr = zmake(1.0, 0.0);
      if (r > i) {
        vr = zmul(pi[r], scl);
        pi[r] = vr;
      }
#pragma unroll
      for (int c = 1; c < NB; ++c) {
        if (c <= i) continue;
        P[(size_t)c * m + r] = zfnma(vr, tz[c], P[(size_t)c * m + r]);
      }
    }
    __syncthreads();
  }
  // write back: R and zeros into the panel, V, then T
  zd* vk = V + (size_t)k * sv;
  for (int idx = tid; idx < NB * m; idx += PQ_NT) {
    const int i = idx / m, r = idx % m;
    zd out, vv;
    if (i < kk) {
      out = r < i ? P[idx] : (r == i ? beta_s[i] : zmake(0.0, 0.0));
      vv = r < i ? zmake(0.0, 0.0) : (r == i ? zmake(1.0, 0.0) : P[idx]);
    } else {
      out = P[idx];
      vv = zmake(0.0, 0.0);
    }
    a[(size_t)(j + i) * n + j + NB + r] = out;
    vk[(size_t)i * ldv + r] = vv;
  }
  zd* tk = T + (size_t)k * NB * NB;
  for (int idx = tid; idx < NB * NB; idx += PQ_NT) tk[idx] = Ts[idx];
}

// W = Y - (1/2) V (T^dagger Z) with Y = X T and Z = V^dagger Y = Z0 T,
// Z0 = V^dagger X, in two launches over WCH row chunks per matrix (the
// work is FP64 and one CTA per matrix would leave most SMs idle):
// wz_kernel forms the chunk partials of Z0 and clears the exponent maxima,
// wrow_kernel sums the partials, forms M2 = T^dagger Z0 T and the rows
// W[r, :] = X[r, :] T - (1/2) V[r, :] M2 of its chunk, and records the
// largest FP64 exponent of each column of V and of W (integer maxima of
// the exponent fields), from which pack_rank2_kernel balances V against W.
constexpr int WCH = 8;

template <int NB>
__global__ void __launch_bounds__(QR_NT) wz_kernel(const zd* __restrict__ X,
                                                   const zd* __restrict__ V, int ld, long sv,
                                                   int m, zd* __restrict__ zpart,
                                                   int* __restrict__ emax) {
  constexpr int NP = NB * NB, NG = QR_NT / NP;
  __shared__ zd Zp[NG][NP];
  const int ch = blockIdx.x, k = blockIdx.y, tid = threadIdx.x;
  const int rb = (int)((long)m * ch / WCH), re = (int)((long)m * (ch + 1) / WCH);
  const zd* xk = X + (size_t)k * sv;
  const zd* vk = V + (size_t)k * sv;
  const int p = tid % NP, g = tid / NP, a = p % NB, c = p / NB;
  zd z = zmake(0.0, 0.0);
  for (int r = rb + g; r < re; r += NG) z = zfmac(xk[(size_t)c * ld + r], vk[(size_t)a * ld + r], z);
  Zp[g][p] = z;
  __syncthreads();
  if (tid < NP) {
    zd t = zmake(0.0, 0.0);
    for (int q = 0; q < NG; ++q) t = zadd(t, Zp[q][tid]);
    zpart[((size_t)k * WCH + ch) * NP + tid] = t;   // Z0[a][c] at a + c NB
  }
  if (ch == 0 && tid < 2 * NB) emax[(size_t)k * 2 * NB + tid] = 0;
}

__device__ __forceinline__ int exp_field(double x) {
  return (int)((__double_as_longlong(x) >> 52) & 0x7FF);
}

template <int NB>
__global__ void __launch_bounds__(QR_NT) wrow_kernel(const zd* __restrict__ X,
                                                     const zd* __restrict__ V,
                                                     const zd* __restrict__ T, int ld, long sv,
                                                     int m, const zd* __restrict__ zpart,
                                                     zd* __restrict__ W, int* __restrict__ emax) {
  constexpr int NP = NB * NB;
  __shared__ zd Ts[NB][NB], Z0[NB][NB], Zt[NB][NB], M2[NB][NB];
  __shared__ int ecol[2][NB];
  const int ch = blockIdx.x, k = blockIdx.y, tid = threadIdx.x;
  const int rb = (int)((long)m * ch / WCH), re = (int)((long)m * (ch + 1) / WCH);
  for (int idx = tid; idx < NP; idx += QR_NT) {
    Ts[idx % NB][idx / NB] = T[(size_t)k * NP + idx];
    zd t = zmake(0.0, 0.0);
    for (int q = 0; q < WCH; ++q) t = zadd(t, zpart[((size_t)k * WCH + q) * NP + idx]);
    Z0[idx % NB][idx / NB] = t;
  }
  if (tid < 2 * NB) ecol[tid / NB][tid % NB] = 0;
  __syncthreads();
  if (tid < NP) {   // Zt = Z0 T
    const int a = tid % NB, c = tid / NB;
    zd t = zmake(0.0, 0.0);
    for (int q = 0; q <= c; ++q) t = zfma(Z0[a][q], Ts[q][c], t);
    Zt[a][c] = t;
  }
  __syncthreads();
  if (tid < NP) {   // M2 = T^dagger Zt
    const int a = tid % NB, c = tid / NB;
    zd t = zmake(0.0, 0.0);
    for (int d = 0; d <= a; ++d) t = zfma(zconj(Ts[d][a]), Zt[d][c], t);
    M2[a][c] = t;
  }
  __syncthreads();
  const zd* xk = X + (size_t)k * sv;
  const zd* vk = V + (size_t)k * sv;
  zd* wk = W + (size_t)k * sv;
  constexpr int RS = QR_NT / NB;
  const int c = tid % NB;
  int ev = 0, ew = 0;
  for (int r = rb + tid / NB; r < re; r += RS) {
    zd y = zmake(0.0, 0.0), t = zmake(0.0, 0.0);
    for (int q = 0; q <= c; ++q) y = zfma(xk[(size_t)q * ld + r], Ts[q][c], y);
    for (int q = 0; q < NB; ++q) t = zfma(vk[(size_t)q * ld + r], M2[q][c], t);
    y.x = fma(-0.5, t.x, y.x);
    y.y = fma(-0.5, t.y, y.y);
    wk[(size_t)c * ld + r] = y;
    const zd v = vk[(size_t)c * ld + r];
    ev = max(ev, max(exp_field(v.x), exp_field(v.y)));
    ew = max(ew, max(exp_field(y.x), exp_field(y.y)));
  }
  atomicMax(&ecol[0][c], ev);
  atomicMax(&ecol[1][c], ew);
  __syncthreads();
  if (tid < 2 * NB) atomicMax(&emax[(size_t)k * 2 * NB + tid], ecol[tid / NB][tid % NB]);
}

// ---------------------------------------------------------------- stage 2
// Band storage: column c holds A[c + d, c] for d < 2 NB (d <= NB is the
// band, the rest room for the bulges), complex, at bd[c 2NB + d].
//
// One sweep task works on an 8 x 8 block O (rows r0 .. r0+7 below the
// columns C0 .. C0+7 of the previous reflector) and the diagonal block D
// of rows r0 .. r0+7, on eight lanes, lane i holding row i of both, four
// sweeps per warp.  Row sums are lane-local; for column sums the lanes pass
// the block's entries round so that lane i forms column i's products.  The
// scalars of the reflector come from FP64 reciprocal square roots and one
// reciprocal; GB300 issues FP64 at 2 operations per clock per SM, so every
// redundant FP64 operation across lanes counts.
constexpr int CH_NB = 8;                // band half-width of the chase
constexpr int CH_WARPS = 16;            // warps per CTA
constexpr int CH_SLOTS = CH_WARPS * 4;  // sweeps in flight per matrix

__device__ __forceinline__ zd gshfl(zd v, int src) {
  return zmake(__shfl_sync(0xffffffffu, v.x, src, 8), __shfl_sync(0xffffffffu, v.y, src, 8));
}
__device__ __forceinline__ zd sel(bool c, zd a, zd b) { return c ? a : b; }

// element k of a lane's eight complex values, k differing between lanes (a
// select chain: integer work, which costs the chase nothing next to its
// FP64 issue)
__device__ __forceinline__ zd pick8(const zd (&O)[8], int k) {
  zd r = O[0];
#pragma unroll
  for (int q = 1; q < 8; ++q) r = sel(k == q, O[q], r);
  return r;
}

// z_i = sum_r conj(v_r) O[r][i] on lane i of the group (row r of O on lane
// r): in round t lane r sends O[r][(r + t) mod 8] and lane i receives
// O[(i - t) mod 8][i], so each lane forms the products of its own column
// and no FP64 additions cross lanes (8 complex multiply-adds per lane,
// against 8 products and 7 complex additions of a reduce-scatter)
__device__ __forceinline__ zd colsum8(const zd (&O)[8], zd v, int i) {
  zd z = zmake(0.0, 0.0);
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int src = (i - t) & 7;
    const zd got = gshfl(pick8(O, (i + t) & 7), src);
    z = zfmac(got, gshfl(v, src), z);
  }
  return z;
}

// 1/x from the FP32 hardware approximation r0 and the series r0 (1 + e +
// e^2), e = 1 - x r0 (below 2^-66 of it left out); exact division outside
// the FP32 normal range
__device__ __forceinline__ double rcp_d(double x) {
  const unsigned ex = ((unsigned)__double2hiint(x) >> 20) & 0x7ffu;
  if (ex - 904u <= 238u) {
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"((float)x));
    const double r0 = (double)rf;
    const double e = fma(-x, r0, 1.0);
    return fma(fma(e, e, e), r0, r0);
  }
  return 1.0 / x;
}

__device__ __forceinline__ double gsum(double v) {
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  return v;
}

__global__ void __launch_bounds__(CH_WARPS * 32, 1)
    bulge_kernel(const zd* __restrict__ A, int n, zd* __restrict__ band_g, int in_smem,
                 double* __restrict__ de) {
  constexpr int NB = CH_NB, W2 = 2 * NB;
  extern __shared__ __align__(16) unsigned char dsm[];
  const int k = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int* T0 = reinterpret_cast<int*>(dsm);   // start step of each sweep
  __shared__ int tend_s;
  zd* bd = in_smem ? reinterpret_cast<zd*>(dsm + ((size_t)n * sizeof(int) + 15) / 16 * 16)
                   : band_g + (size_t)k * n * W2;
  const zd* a = A + (size_t)k * n * n;
  for (int idx = tid; idx < n * W2; idx += CH_WARPS * 32) {
    const int c = idx / W2, d = idx % W2;
    zd v = zmake(0.0, 0.0);
    if (d <= NB && c + d < n) v = a[(size_t)c * n + c + d];
    if (d == 0) v.y = 0.0;
    bd[idx] = v;
  }
  if (tid == 0) {
    // sweep s runs on slot s mod CH_SLOTS, LAG steps after sweep s - 1
    // started and once its slot's previous sweep has finished
    int prev = -LAG, tend = 0;
    for (int s = 0; s + 1 < n; ++s) {
      const int nt = (n - 1 - s + NB - 1) / NB;
      int t0 = prev + LAG;
      if (s >= CH_SLOTS) {
        const int sp = s - CH_SLOTS, ntp = (n - 1 - sp + NB - 1) / NB;
        t0 = max(t0, T0[sp] + ntp);
      }
      T0[s] = t0;
      prev = t0;
      tend = max(tend, t0 + nt);
    }
    tend_s = tend;
  }
  __syncthreads();
  const int tend = tend_s;
  const int i = lane & 7;
  // lower-triangle entries (row, column) of the 8 x 8 diagonal block that
  // this lane updates: e = i + 8q in row-major order, 36 entries (-1: none)
  int tr[5], tc[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const int e = i + 8 * q;
    int r = 0;
    while ((r + 1) * (r + 2) / 2 <= e) ++r;
    tr[q] = e < 36 ? r : -1;
    tc[q] = e < 36 ? e - r * (r + 1) / 2 : 0;
  }
  int s = warp * 4 + (lane >> 3);   // this group's sweep
  zd vp = zmake(0.0, 0.0);          // previous reflector of the sweep (row i)
  double taup = 0.0;
  const zd zero = zmake(0.0, 0.0);
  for (int t = 0; t < tend; ++t) {
    const bool act = s + 1 < n && t >= T0[s];
    // the sweeps in flight are consecutive, so most warps have none: they
    // skip the step's FP64 work (the pipe's issue slots are per warp)
    if (!__any_sync(0xffffffffu, act)) {
      __syncthreads();
      continue;
    }
    const int kt = act ? t - T0[s] + 1 : 1;
    const int C0 = kt == 1 ? s : s + 1 + (kt - 2) * NB;
    const int Lc = kt == 1 ? 1 : NB;
    const int r0 = C0 + Lc;
    const int L = act ? min(r0 + NB - 1, n - 1) - r0 + 1 : 0;
    const double tp = kt == 1 ? 0.0 : taup;
    // O <- O H_prev (a no-op for the first task, whose O is column s)
    zd O[8];
    zd y = zero;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      O[j] = (i < L && j < Lc) ? bd[(size_t)(C0 + j) * W2 + (r0 + i - C0 - j)] : zero;
      y = zfma(O[j], gshfl(vp, j), y);
    }
    const zd ty = zscale(y, tp);
#pragma unroll
    for (int j = 0; j < 8; ++j) O[j] = zfnmac(ty, gshfl(vp, j), O[j]);
    // reflector H = I - tau v v^dagger, H x = beta e1, x = column 0 of O
    const zd x = O[0];
    const double sq = gsum((i >= 1 && i < L) ? fma(x.x, x.x, x.y * x.y) : 0.0);
    const zd al = gshfl(x, 0);
    const double a2 = fma(al.x, al.x, al.y * al.y), s2 = a2 + sq;
    double tau = 0.0;
    zd beta = zero, scl = zero;
    if (s2 > 0.0) {
      const double rn = rsqrt(s2), nu = s2 * rn;
      if (a2 > 0.0) {
        const double ra = rsqrt(a2), aa = a2 * ra;
        beta = zscale(al, -nu * ra);
        tau = (aa + nu) * rn;
        // 1 / (alpha - beta) = conj(alpha) ra / (|alpha| + nu)
        scl = zscale(zconj(al), ra * rcp_d(aa + nu));
      } else {
        beta = zmake(-nu, 0.0);
        tau = 1.0;
        scl = zmake(rn, 0.0);
      }
    }
    const zd v = i == 0 ? zmake(1.0, 0.0) : ((i < L && tau != 0.0) ? zmul(x, scl) : zero);
    // O <- H O: z_j = sum_i conj(v_i) O[i][j], O[i][j] -= tau v_i z_j
    {
      const zd zi = colsum8(O, v, i);
      const zd tv = zscale(v, tau);
#pragma unroll
      for (int j = 0; j < 8; ++j) O[j] = zfnma(tv, gshfl(zi, j), O[j]);
    }
    O[0] = i == 0 ? beta : zero;
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (i < L && j < Lc) bd[(size_t)(C0 + j) * W2 + (r0 + i - C0 - j)] = O[j];
    // D <- H D H on rows and columns r0 .. r0+L-1
    zd D[8];
    zd p = zero;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      zd dv = zero;
      if (i < L && j < L)
        dv = i >= j ? bd[(size_t)(r0 + j) * W2 + (i - j)]
                    : zconj(bd[(size_t)(r0 + i) * W2 + (j - i)]);
      D[j] = dv;
      p = zfma(dv, gshfl(v, j), p);
    }
    p = zscale(p, tau);
    const zd q = zmul(zconj(v), p);
    const double vhp = gsum(q.x);   // v^dagger p is real
    const zd w = zsub(p, zscale(v, 0.5 * tau * vhp));
    // D -= v w^dagger + w v^dagger on the 36 lower-triangle entries only,
    // five per lane (entry e = i + 8q, (tr[q], tc[q]) precomputed)
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const int rr = tr[q], cc = tc[q];
      const zd vr = gshfl(v, rr), wr = gshfl(w, rr), vc = gshfl(v, cc), wc = gshfl(w, cc);
      if (rr >= 0 && rr < L) {
        zd* dp = bd + (size_t)(r0 + cc) * W2 + (rr - cc);
        zd dv = zfnmac(vr, wc, *dp);
        dv = zfnmac(wr, vc, dv);
        if (rr == cc) dv.y = 0.0;
        *dp = dv;
      }
    }
    vp = v;
    taup = tau;
    if (act && kt == (n - 1 - s + NB - 1) / NB) s += CH_SLOTS;
    __syncthreads();
  }
  double* dk = de + (size_t)k * 2 * n;
  for (int c = tid; c < n; c += CH_WARPS * 32) {
    dk[c] = bd[(size_t)c * W2].x;
    const zd e = c + 1 < n ? bd[(size_t)c * W2 + 1] : zmake(0.0, 0.0);
    dk[n + c] = hypot(e.x, e.y);
  }
}

size_t bulge_smem(int n, bool in_smem) {
  size_t b = ((size_t)n * sizeof(int) + 15) / 16 * 16;
  if (in_smem) b += (size_t)n * 2 * CH_NB * sizeof(zd);
  return b;
}

int max_optin_smem() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 48 * 1024;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 48 * 1024;
  return v;
}

// the largest dynamic shared memory a kernel can take on this device: the
// opt-in limit per block less the kernel's static shared memory
int dyn_smem_limit(const void* fn) {
  cudaFuncAttributes fa;
  int st = 0;
  if (cudaFuncGetAttributes(&fa, fn) == cudaSuccess) st = (int)fa.sharedSizeBytes;
  else cudaGetLastError();
  return max_optin_smem() - st;
}

}  // namespace

// ---------------------------------------------------------------- host side
bool bs_band_supported(int n) {
  // the panel QR keeps an m x NB panel in shared memory
  return n >= 2 && (size_t)BS_BAND_NB * n * sizeof(zd) <=
                    (size_t)dyn_smem_limit((const void*)panel_qr_kernel<BS_BAND_NB>);
}

static void band_events_free(BandWs* w) {
  for (int i = 0; i < BS_BAND_GROUPS * 2 * w->evcap; ++i) cudaEventDestroy(w->ev[i]);
  delete[] w->ev;
  w->ev = nullptr;
  w->evcap = 0;
}

void bs_band_ws_free(BandWs* w) {
  band_events_free(w);
  if (w->fork) cudaEventDestroy(w->fork);
  for (int h = 0; h < BS_BAND_PARTS; ++h) {
    if (w->join[h]) cudaEventDestroy(w->join[h]);
    if (w->sp[h]) cudaStreamDestroy(w->sp[h]);
    if (w->sb[h]) cudaStreamDestroy(w->sb[h]);
    if (w->epr[h]) cudaEventDestroy(w->epr[h]);
    if (w->eru[h]) cudaEventDestroy(w->eru[h]);
  }
  void* p[] = {w->V, w->X, w->W, w->T, w->wA, w->wB, w->wD, w->eA, w->eB, w->band, w->dsc,
               w->zpart};
  for (void* q : p) cudaFree(q);
  *w = BandWs();
}

// The batch runs in BAND_PARTS parts on as many streams (the caller's and
// the workspace's own): the panel QR and W formation of one part are
// FP64-bound on one CTA per matrix, and run beside the tensor-core and
// memory-bound products of the others.  The digit planes and sums have one
// region per part.
constexpr int BAND_PARTS = BS_BAND_PARTS;
static void parts(int kb, int* k) {
  const int np = kb < BAND_PARTS ? kb : BAND_PARTS;
  for (int h = 0; h < BAND_PARTS; ++h) k[h] = h < np ? kb / np + (h < kb % np ? 1 : 0) : 0;
}

int bs_band_ws_alloc(BandWs* w, int n, int kb, int S) {
  if (w->n == n && w->kb >= kb && w->S == S) return BS_OK;
  bs_band_ws_free(w);
  const int NB = BS_BAND_NB;
  const int m = std::max(n - NB, 1);
  int kp[BAND_PARTS];
  parts(kb, kp);
  size_t nA = 0, nB = 0, nD = 0, nE = 0;
  bs_band_tc_elems(n, NB, kp[0], S, &nA, &nB, &nD, &nE);   // part 0 is the largest
  w->hA = nA;
  w->hB = nB;
  w->hD = nD;
  w->hE = nE;
  const size_t pv = (size_t)kb * m * NB;
  struct Item { void** p; size_t bytes; const char* what; } items[] = {
      {(void**)&w->V, pv * sizeof(zd), "band reflectors"},
      {(void**)&w->X, pv * sizeof(zd), "band A22 V"},
      {(void**)&w->W, pv * sizeof(zd), "band W"},
      {(void**)&w->T, (size_t)kb * NB * NB * sizeof(zd), "band T"},
      {(void**)&w->wA, BAND_PARTS * nA * sizeof(uint16_t), "band digit planes A"},
      {(void**)&w->wB, BAND_PARTS * nB * sizeof(uint16_t), "band digit planes B"},
      {(void**)&w->wD, BAND_PARTS * nD * sizeof(float), "band digit-order sums"},
      {(void**)&w->eA, BAND_PARTS * nE * sizeof(int), "band exponents A"},
      {(void**)&w->eB, BAND_PARTS * nE * sizeof(int), "band exponents B"},
      {(void**)&w->band, (size_t)kb * n * 2 * NB * sizeof(zd), "band storage"},
      {(void**)&w->dsc, (size_t)kb * 2 * NB * sizeof(int), "band column exponents"},
      {(void**)&w->zpart, (size_t)kb * WCH * NB * NB * sizeof(zd), "band Z0 partials"},
  };
  for (auto& it : items) {
    cudaError_t e = cudaMalloc(it.p, it.bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      bs_band_ws_free(w);
      bs_set_error("out of device memory (%s, %zu bytes)", it.what, it.bytes);
      return BS_ENOMEM;
    }
  }
  // the chain of panel steps (QR, digit planes, A22 V, W, the next panel's
  // columns) goes first whenever an SM frees up; the bulk of the trailing
  // update fills the rest
  int prio_lo = 0, prio_hi = 0;
  cudaError_t e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w->fork, cudaEventDisableTiming);
  for (int h = 0; e == cudaSuccess && h < BAND_PARTS; ++h) {
    e = cudaStreamCreateWithPriority(&w->sp[h], cudaStreamNonBlocking, prio_hi);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w->join[h], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&w->sb[h], cudaStreamNonBlocking, prio_lo);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w->epr[h], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w->eru[h], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    bs_band_ws_free(w);
    return bs_cuda_status(e, "band reduction stream");
  }
  w->n = n;
  w->kb = kb;
  w->S = S;
  return BS_OK;
}

int bs_launch_eig_band(zd* A, int n, int kb, BandWs& w, double* de, int* err, cudaStream_t s,
                       const BandBisect* bis) {
  constexpr int NB = BS_BAND_NB;
  if (w.n != n || w.kb < kb || !bs_band_supported(n)) {
    bs_set_error("band reduction: workspace for n = %d, %d matrices not set up", n, kb);
    return BS_EINVAL;
  }
  const int nt = (n + 31) / 32;
  symmetrize_kernel<<<dim3(nt, nt, kb), dim3(32, 8), 0, s>>>(A, n);
  BS_CHECK_LAUNCH("symmetrize_kernel");
  const int ld = std::max(n - NB, 1);
  const long sv = (long)ld * NB;
  {
    // the shared-memory opt-ins are per-device attributes of the kernels,
    // set once per device to the device's limit (not during a capture)
    static std::atomic<bool> attr[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    if (!attr[dev].load(std::memory_order_acquire)) {
      cudaError_t e = cudaFuncSetAttribute(panel_qr_kernel<NB>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           dyn_smem_limit((const void*)panel_qr_kernel<NB>));
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(bulge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 dyn_smem_limit((const void*)bulge_kernel));
      if (e != cudaSuccess) return bs_cuda_status(e, "band reduction smem");
      attr[dev].store(true, std::memory_order_release);
    }
  }
  // timing: event pairs per kernel group and step, on the first part's stream
  const int steps = n - NB > 1 ? (n - NB - 2) / NB + 1 : 0;
  if (w.prof && w.evcap < steps + 1) {
    band_events_free(&w);
    const int cap = steps + 1;
    w.ev = new cudaEvent_t[BS_BAND_GROUPS * 2 * cap];
    for (int i = 0; i < BS_BAND_GROUPS * 2 * cap; ++i) {
      cudaError_t e = cudaEventCreate(&w.ev[i]);
      if (e != cudaSuccess) {
        for (int q = 0; q < i; ++q) cudaEventDestroy(w.ev[q]);
        delete[] w.ev;
        w.ev = nullptr;
        return bs_cuda_status(e, "band reduction events");
      }
    }
    w.evcap = cap;
  }
  int hk[BAND_PARTS], off[BAND_PARTS];
  cudaStream_t hs[BAND_PARTS];
  parts(kb, hk);
  for (int h = 0; h < BAND_PARTS; ++h) {
    off[h] = h == 0 ? 0 : off[h - 1] + hk[h - 1];
    hs[h] = w.sp[h];
  }
  w.nsteps = steps;
  w.timed = hk[0];
  {
    cudaError_t e = cudaEventRecord(w.fork, s);
    for (int h = 0; e == cudaSuccess && h < BAND_PARTS; ++h)
      if (hk[h] > 0) e = cudaStreamWaitEvent(hs[h], w.fork, 0);
    if (e != cudaSuccess) return bs_cuda_status(e, "band reduction fork");
  }
  auto mark = [&](int h, int grp, int step, int end, cudaStream_t st) {
    if (w.prof && h == 0) cudaEventRecord(w.ev[(grp * w.evcap + step) * 2 + end], st);
  };
  // Per part, with look-ahead: after step j's operands of the rank-2
  // update are packed, the update of the next panel's columns (the first
  // column tile) runs first and the next panel's QR follows at once on the
  // part's stream A, while the rest of the update runs on its stream B.
  // Events: epr (rank-2 operands packed), eru (the rest of the update done).
  // The panel QR reads and writes only the panel's columns, which stream B
  // does not touch; the next step's digit planes of A22 (stream A) wait for
  // the rest of the update, which also still reads this step's digit buffers.
  int step = 0;
  for (int j = 0; n - j - NB > 1; j += NB, ++step) {
    const int m = n - j - NB;
    const bool next = n - (j + NB) - NB > 1;
    for (int h = 0; h < BAND_PARTS; ++h) {
      const int kh = hk[h];
      if (kh == 0) continue;
      const cudaStream_t st = hs[h], sb = w.sb[h];
      zd* Ah = A + (size_t)off[h] * n * n;
      zd* Vh = w.V + (size_t)off[h] * sv;
      zd* Xh = w.X + (size_t)off[h] * sv;
      zd* Wh = w.W + (size_t)off[h] * sv;
      zd* Th = w.T + (size_t)off[h] * NB * NB;
      int* dh = w.dsc + (size_t)off[h] * 2 * NB;
      zd* zh = w.zpart + (size_t)off[h] * WCH * NB * NB;
      uint16_t* wAh = w.wA + h * w.hA;
      uint16_t* wBh = w.wB + h * w.hB;
      float* wDh = w.wD + h * w.hD;
      int* eAh = w.eA + h * w.hE;
      int* eBh = w.eB + h * w.hE;
      if (step == 0) {
        mark(h, 0, step, 0, st);
        panel_qr_kernel<NB><<<kh, PQ_NT, (size_t)NB * m * sizeof(zd), st>>>(Ah, n, j, Vh, ld, sv,
                                                                            Th);
        BS_CHECK_LAUNCH("panel_qr_kernel");
        mark(h, 0, step, 1, st);
      } else {
        cudaError_t e = cudaStreamWaitEvent(st, w.eru[h], 0);
        if (e != cudaSuccess) return bs_cuda_status(e, "band reduction wait");
      }
      mark(h, 1, step, 0, st);
      TRY_LAUNCH(bs_launch_band_pack_trail(Ah, n, j + NB, m, kh, wAh, eAh, st));
      TRY_LAUNCH(bs_launch_band_av(m, Vh, ld, sv, NB, kh, w.S, wAh, wBh, wDh, eAh, eBh, Xh, ld, sv,
                                   err, st));
      mark(h, 1, step, 1, st);
      mark(h, 2, step, 0, st);
      wz_kernel<NB><<<dim3(WCH, kh), QR_NT, 0, st>>>(Xh, Vh, ld, sv, m, zh, dh);
      BS_CHECK_LAUNCH("wz_kernel");
      wrow_kernel<NB><<<dim3(WCH, kh), QR_NT, 0, st>>>(Xh, Vh, Th, ld, sv, m, zh, Wh, dh);
      BS_CHECK_LAUNCH("wrow_kernel");
      mark(h, 2, step, 1, st);
      TRY_LAUNCH(bs_launch_band_pack_rank2(Vh, Wh, ld, sv, dh, m, NB, kh, w.S, wAh, wBh, eAh, st));
      if (!next) {
        mark(h, 3, step, 0, st);
        TRY_LAUNCH(bs_launch_rank2_update(wAh, wBh, eAh, m, kh, Ah, n, j + NB, 0, 0, err, st));
        mark(h, 3, step, 1, st);
        continue;
      }
      cudaError_t e = cudaEventRecord(w.epr[h], st);
      if (e != cudaSuccess) return bs_cuda_status(e, "band reduction events");
      // the next panel's columns (first column tile), then its QR
      TRY_LAUNCH(bs_launch_rank2_update(wAh, wBh, eAh, m, kh, Ah, n, j + NB, 0, 1, err, st));
      const int m2 = m - NB;
      mark(h, 0, step + 1, 0, st);
      panel_qr_kernel<NB><<<kh, PQ_NT, (size_t)NB * m2 * sizeof(zd), st>>>(Ah, n, j + NB, Vh,
                                                                           ld, sv, Th);
      BS_CHECK_LAUNCH("panel_qr_kernel");
      mark(h, 0, step + 1, 1, st);
      // stream B: the rest of the update
      e = cudaStreamWaitEvent(sb, w.epr[h], 0);
      if (e != cudaSuccess) return bs_cuda_status(e, "band reduction wait");
      mark(h, 3, step, 0, sb);
      TRY_LAUNCH(bs_launch_rank2_update(wAh, wBh, eAh, m, kh, Ah, n, j + NB, 1, 0, err, sb));
      mark(h, 3, step, 1, sb);
      e = cudaEventRecord(w.eru[h], sb);
      if (e != cudaSuccess) return bs_cuda_status(e, "band reduction events");
    }
  }
  static_assert(NB == CH_NB, "the bulge chase is written for a band half-width of 8");
  const bool in_smem = bulge_smem(n, true) <= (size_t)dyn_smem_limit((const void*)bulge_kernel);
  const size_t smem = bulge_smem(n, in_smem);
  for (int h = 0; h < BAND_PARTS; ++h) {
    if (hk[h] == 0) continue;
    mark(h, 4, 0, 0, hs[h]);
    bulge_kernel<<<hk[h], CH_WARPS * 32, smem, hs[h]>>>(
        A + (size_t)off[h] * n * n, n, w.band + (size_t)off[h] * n * 2 * NB, in_smem ? 1 : 0,
        de + (size_t)off[h] * 2 * n);
    BS_CHECK_LAUNCH("bulge_kernel");
    mark(h, 4, 0, 1, hs[h]);
    // the part's eigenvalues right behind its bulge chase, beside the
    // other parts' chases
    if (bis)
      TRY_LAUNCH(bs_launch_bisect(de + (size_t)off[h] * 2 * n, n, hk[h], bis->nbands,
                                  bis->omega + (size_t)off[h] * bis->nbands,
                                  bis->stat ? bis->stat + off[h] : nullptr, hs[h]));
  }
  for (int h = 0; h < BAND_PARTS; ++h) {
    if (hk[h] == 0) continue;
    cudaError_t e = cudaEventRecord(w.join[h], hs[h]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, w.join[h], 0);
    if (e != cudaSuccess) return bs_cuda_status(e, "band reduction join");
  }
  return BS_OK;
}

int bs_band_times(BandWs& w, double ms[BS_BAND_GROUPS]) {
  for (int g = 0; g < BS_BAND_GROUPS; ++g) ms[g] = 0.0;
  if (!w.prof || !w.ev) return BS_OK;
  cudaError_t e = cudaEventSynchronize(w.ev[(4 * w.evcap) * 2 + 1]);
  if (e != cudaSuccess) return bs_cuda_status(e, "band reduction times");
  for (int g = 0; g < BS_BAND_GROUPS; ++g) {
    const int ns = g == 4 ? 1 : w.nsteps;
    for (int st = 0; st < ns; ++st) {
      float t = 0.f;
      e = cudaEventElapsedTime(&t, w.ev[(g * w.evcap + st) * 2], w.ev[(g * w.evcap + st) * 2 + 1]);
      if (e != cudaSuccess) return bs_cuda_status(e, "band reduction times");
      ms[g] += t;
    }
  }
  return BS_OK;
}
