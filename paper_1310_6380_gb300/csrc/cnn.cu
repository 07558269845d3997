// Learned warm start for the block LOBPCG path: a small convolutional
// network that maps a cell's material maps and a wavevector to a starting
// subspace (the low-order plane-wave displacement coefficients of nvec
// vectors), with its own forward and backward kernels and Adam, in FP32.
//
// Architecture (fixed; the parameter layout follows this list):
//   input  3 x 64 x 64: standardised log(lam + 2 mu), log mu, log rho per pixel
//   conv 3x3 (circular padding: the cell is periodic) 3 -> 16, ReLU, 2x2 mean pool -> 32x32
//   conv 16 -> 32, ReLU, pool -> 16x16;  conv 32 -> 32, ReLU, pool -> 8x8
//   conv 32 -> 32, ReLU, pool -> 4x4  => 512 features per cell
//   per (cell, k): [features | 7 wavevector features] -> dense 519 -> 512, ReLU
//                  -> dense 512 -> 512, ReLU -> dense 512 -> nvec * L * 2
//   (L = 2 (2Mp+1)^2 complex coefficients per vector, interleaved re, im).
// The convolutional trunk runs once per cell; the head once per (cell, k).
//
// Loss (basis-invariant): with U the predicted L x nvec block and V the L x nb
// low-order part of the true eigenvectors,
//   loss = (||V||^2 - tr(B^H G^-1 B)) / ||V||^2,  G = U^H U + eps I,  B = U^H V,
// the part of V outside span(U); its gradient is dloss/dU* = -(V - U F) F^H
// / ||V||^2 with F = G^-1 B (so d/dRe U = 2 Re, d/dIm U = 2 Im of that).
#include <math.h>

#include <algorithm>
#include <vector>

#include "bs_internal.h"

namespace {

constexpr int IMG = 64;
constexpr int KF = 7;          // wavevector features
constexpr int FEAT = 512;      // trunk output
constexpr int HID = 512;
constexpr float LOSS_EPS = 1e-4f;
constexpr int NCONV = 4;
const int CIN[NCONV] = {3, 16, 32, 32};
const int COUT[NCONV] = {16, 32, 32, 32};
const int SIDE[NCONV] = {64, 32, 16, 8};   // input side of conv l (output side equal, then pooled)

// ------------------------------------------------------------ convolution (3x3, circular)
// out[b][co][y][x] = relu(bias[co] + sum_ci,dy,dx w[co][ci][dy][dx] in[b][ci][y+dy-1][x+dx-1])
constexpr int CO_T = 8;   // output channels per thread
__global__ void conv_fwd_kernel(const float* __restrict__ in, const float* __restrict__ w,
                                const float* __restrict__ bias, int cin, int cout, int S,
                                float* __restrict__ out) {
  extern __shared__ float wsh[];   // CO_T x cin x 9
  const int b = blockIdx.z, co0 = blockIdx.y * CO_T;
  const int npix = S * S, p = blockIdx.x * blockDim.x + threadIdx.x;
  for (int e = threadIdx.x; e < CO_T * cin * 9; e += blockDim.x) {
    const int co = co0 + e / (cin * 9);
    wsh[e] = co < cout ? w[(size_t)co * cin * 9 + e % (cin * 9)] : 0.f;
  }
  __syncthreads();
  if (p >= npix) return;
  const int y = p / S, x = p % S;
  float acc[CO_T];
#pragma unroll
  for (int t = 0; t < CO_T; ++t) acc[t] = co0 + t < cout ? bias[co0 + t] : 0.f;
  const float* ib = in + (size_t)b * cin * npix;
  for (int ci = 0; ci < cin; ++ci) {
    const float* ic = ib + (size_t)ci * npix;
    float v[9];
#pragma unroll
    for (int d = 0; d < 9; ++d) {
      const int yy = (y + d / 3 - 1 + S) % S, xx = (x + d % 3 - 1 + S) % S;
      v[d] = ic[yy * S + xx];
    }
#pragma unroll
    for (int t = 0; t < CO_T; ++t) {
      const float* wt = wsh + (t * cin + ci) * 9;
#pragma unroll
      for (int d = 0; d < 9; ++d) acc[t] = fmaf(wt[d], v[d], acc[t]);
    }
  }
#pragma unroll
  for (int t = 0; t < CO_T; ++t)
    if (co0 + t < cout) out[((size_t)b * cout + co0 + t) * npix + p] = fmaxf(acc[t], 0.f);
}

// gin[b][ci][y][x] = sum_co,dy,dx w[co][ci][dy][dx] g[b][co][y-dy+1][x-dx+1]
constexpr int CI_T = 8;
__global__ void conv_bwd_data_kernel(const float* __restrict__ g, const float* __restrict__ w,
                                     int cin, int cout, int S, float* __restrict__ gin) {
  extern __shared__ float wsh[];   // CI_T x cout x 9, [t][co][d]
  const int b = blockIdx.z, ci0 = blockIdx.y * CI_T;
  const int npix = S * S, p = blockIdx.x * blockDim.x + threadIdx.x;
  for (int e = threadIdx.x; e < CI_T * cout * 9; e += blockDim.x) {
    const int t = e / (cout * 9), co = (e / 9) % cout, d = e % 9;
    wsh[e] = ci0 + t < cin ? w[((size_t)co * cin + ci0 + t) * 9 + d] : 0.f;
  }
  __syncthreads();
  if (p >= npix) return;
  const int y = p / S, x = p % S;
  float acc[CI_T];
#pragma unroll
  for (int t = 0; t < CI_T; ++t) acc[t] = 0.f;
  const float* gb = g + (size_t)b * cout * npix;
  for (int co = 0; co < cout; ++co) {
    const float* gc = gb + (size_t)co * npix;
    float v[9];
#pragma unroll
    for (int d = 0; d < 9; ++d) {
      const int yy = (y - d / 3 + 1 + S) % S, xx = (x - d % 3 + 1 + S) % S;
      v[d] = gc[yy * S + xx];
    }
#pragma unroll
    for (int t = 0; t < CI_T; ++t) {
      const float* wt = wsh + (t * cout + co) * 9;
#pragma unroll
      for (int d = 0; d < 9; ++d) acc[t] = fmaf(wt[d], v[d], acc[t]);
    }
  }
#pragma unroll
  for (int t = 0; t < CI_T; ++t)
    if (ci0 + t < cin) gin[((size_t)b * cin + ci0 + t) * npix + p] = acc[t];
}

// partial weight gradients: part[split][co][ci][9] (+ bias partial at part[split][co][cin][0])
// over the samples b with b % nsplit == split
__global__ void conv_bwd_weight_kernel(const float* __restrict__ g, const float* __restrict__ in,
                                       int B, int cin, int cout, int S, int nsplit,
                                       float* __restrict__ part) {
  const int co = blockIdx.x / (cin + 1), ci = blockIdx.x % (cin + 1), split = blockIdx.y;
  const int npix = S * S;
  float acc[9];
#pragma unroll
  for (int d = 0; d < 9; ++d) acc[d] = 0.f;
  for (int b = split; b < B; b += nsplit) {
    const float* gc = g + ((size_t)b * cout + co) * npix;
    if (ci == cin) {   // bias
      for (int p = threadIdx.x; p < npix; p += blockDim.x) acc[0] += gc[p];
      continue;
    }
    const float* ic = in + ((size_t)b * cin + ci) * npix;
    for (int p = threadIdx.x; p < npix; p += blockDim.x) {
      const float gv = gc[p];
      if (gv == 0.f) continue;
      const int y = p / S, x = p % S;
#pragma unroll
      for (int d = 0; d < 9; ++d) {
        const int yy = (y + d / 3 - 1 + S) % S, xx = (x + d % 3 - 1 + S) % S;
        acc[d] = fmaf(gv, ic[yy * S + xx], acc[d]);
      }
    }
  }
  __shared__ float red[9][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int d = 0; d < 9; ++d) {
    float v = acc[d];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[d][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < 9) {
    float sum = 0.f;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) sum += red[threadIdx.x][q];
    part[(((size_t)split * cout + co) * (cin + 1) + ci) * 9 + threadIdx.x] = sum;
  }
}

// sum the partials over splits into gw (cout x cin x 9) and gb (cout)
__global__ void conv_wgrad_reduce_kernel(const float* __restrict__ part, int cin, int cout,
                                         int nsplit, float* __restrict__ gw,
                                         float* __restrict__ gb) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int per = (cin + 1) * 9;
  if (e >= cout * per) return;
  float s = 0.f;
  for (int q = 0; q < nsplit; ++q) s += part[(size_t)q * cout * per + e];
  const int co = e / per, ci = (e / 9) % (cin + 1), d = e % 9;
  if (ci < cin) gw[((size_t)co * cin + ci) * 9 + d] = s;
  else if (d == 0) gb[co] = s;
}

// 2x2 mean pooling and its adjoint (the latter also applies the ReLU mask of
// the pooled layer's input: zero gradient where that activation is zero)
__global__ void pool_fwd_kernel(const float* __restrict__ in, int S, size_t planes,
                                float* __restrict__ out) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int h = S / 2;
  if (e >= planes * h * h) return;
  const size_t pl = e / (h * h);
  const int y = (int)(e % (h * h)) / h, x = (int)(e % h);
  const float* ip = in + pl * S * S;
  out[e] = 0.25f * (ip[(2 * y) * S + 2 * x] + ip[(2 * y) * S + 2 * x + 1] +
                    ip[(2 * y + 1) * S + 2 * x] + ip[(2 * y + 1) * S + 2 * x + 1]);
}
__global__ void pool_bwd_kernel(const float* __restrict__ gout, const float* __restrict__ act,
                                int S, size_t planes, float* __restrict__ gin) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= planes * S * S) return;
  const size_t pl = e / (S * S);
  const int y = (int)(e % (S * S)) / S, x = (int)(e % S), h = S / 2;
  gin[e] = act[e] > 0.f ? 0.25f * gout[pl * h * h + (y / 2) * h + x / 2] : 0.f;
}

// ------------------------------------------------------------ dense layers
// C[m][n] = sum_k A(m,k) B(k,n) (+ bias[n], ReLU): A(m,k) = TA ? A[k*lda+m] : A[m*lda+k],
// B(k,n) = TB ? B[n*ldb+k] : B[k*ldb+n]; 64 x 64 tiles, 4 x 4 per thread
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) sgemm_kernel(int M, int N, int K, const float* __restrict__ A,
                                                    int lda, const float* __restrict__ Bm, int ldb,
                                                    const float* __restrict__ bias, bool relu,
                                                    float* __restrict__ C, int ldc) {
  __shared__ float As[16][64 + 4];
  __shared__ float Bs[16][64 + 4];
  const int tid = threadIdx.x, tm = tid / 16, tn = tid % 16;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = tid; e < 16 * 64; e += 256) {
      const int kk = e / 64, mm = e % 64;
      const int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < M && k < K) ? (TA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k]) : 0.f;
      const int n = n0 + mm;
      Bs[kk][mm] = (n < N && k < K) ? (TB ? Bm[(size_t)n * ldb + k] : Bm[(size_t)k * ldb + n]) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][tm * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tn * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + tm * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tn * 4 + j;
      if (n >= N) continue;
      float v = acc[i][j] + (bias ? bias[n] : 0.f);
      if (relu) v = fmaxf(v, 0.f);
      C[(size_t)m * ldc + n] = v;
    }
  }
}

// column sums: out[n] = sum_m A[m*ld + n]
__global__ void colsum_kernel(const float* __restrict__ A, int M, int N, int ld,
                              float* __restrict__ out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int m = 0; m < M; ++m) s += A[(size_t)m * ld + n];
  out[n] = s;
}

// g[i] *= (act[i] > 0)
__global__ void relu_mask_kernel(float* __restrict__ g, const float* __restrict__ act, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !(act[i] > 0.f)) g[i] = 0.f;
}

// head input: h0[s] = [feat[s / kper] | kf[s]]
__global__ void head_input_kernel(const float* __restrict__ feat, const float* __restrict__ kf,
                                  int ns, int kper, float* __restrict__ h0) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int w = FEAT + KF;
  if (e >= ns * w) return;
  const int s = e / w, j = e % w;
  h0[e] = j < FEAT ? feat[(size_t)(s / kper) * FEAT + j] : kf[(size_t)s * KF + (j - FEAT)];
}

// gfeat[c] = sum over the kper samples of cell c of gh0[s][0..FEAT)
__global__ void feat_grad_kernel(const float* __restrict__ gh0, int nc, int kper,
                                 float* __restrict__ gfeat) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nc * FEAT) return;
  const int c = e / FEAT, j = e % FEAT;
  float s = 0.f;
  for (int t = 0; t < kper; ++t) s += gh0[(size_t)(c * kper + t) * (FEAT + KF) + j];
  gfeat[e] = s;
}

// ------------------------------------------------------------ inputs
// x[c] = standardised log(lam + 2 mu), log mu, log rho of every pixel of cell c
// (phase maps P x P with P = 64, tables lam | mu | rho at table + toff[c]);
// kf[s] = (Q1, Q2, cos 2 pi Q1, sin 2 pi Q1, cos 2 pi Q2, sin 2 pi Q2, hex)
__global__ void encode_kernel(const uint16_t* __restrict__ phase, const double* __restrict__ table,
                              const long* __restrict__ toff, const int* __restrict__ nph, int nc,
                              float* __restrict__ x) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t npix = (size_t)IMG * IMG;
  if (e >= nc * npix) return;
  const int c = (int)(e / npix);
  const int p = phase[e], np = nph[c];
  const double* t = table + toff[c];
  const double lam = t[p], mu = t[np + p], rho = t[2 * np + p];
  float* xc = x + (size_t)c * 3 * npix + e % npix;
  xc[0] = (float)((log(lam + 2.0 * mu) - 3.5) / 1.0);
  xc[npix] = (float)((log(mu) - 2.2) / 1.2);
  xc[2 * npix] = (float)((log(rho) - 1.0) / 0.6);
}
__global__ void kfeat_kernel(const double* __restrict__ Q, const int* __restrict__ hex, int ns,
                             int kper, float* __restrict__ kf) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ns) return;
  const double q1 = Q[2 * s], q2 = Q[2 * s + 1];
  float* o = kf + (size_t)s * KF;
  o[0] = (float)q1;
  o[1] = (float)q2;
  o[2] = (float)cospi(2.0 * q1);
  o[3] = (float)sinpi(2.0 * q1);
  o[4] = (float)cospi(2.0 * q2);
  o[5] = (float)sinpi(2.0 * q2);
  o[6] = hex[s / kper] ? 1.f : 0.f;
}

// ------------------------------------------------------------ subspace loss
// one CTA per sample: U (L x nv, from out), V (L x nb, from tgt), loss[s], gout[s]
constexpr int LMAX = 2 * 49;   // Mp <= 3
constexpr int NVMAX = 16;
__global__ void __launch_bounds__(128) loss_kernel(const float* __restrict__ out,
                                                   const float* __restrict__ tgt, int L, int nv,
                                                   int nb, float scale, float* __restrict__ loss,
                                                   float* __restrict__ gout) {
  __shared__ float2 U[LMAX][NVMAX + 1], V[LMAX][NVMAX + 1], R[LMAX][NVMAX + 1];
  __shared__ float2 G[NVMAX][NVMAX + 1], Bm[NVMAX][NVMAX + 1], F[NVMAX][NVMAX + 1];
  __shared__ float vn2, cap;
  __shared__ int bad;
  const int s = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const float* o = out + (size_t)s * nv * L * 2;
  const float* t = tgt + (size_t)s * nb * L * 2;
  for (int e = tid; e < nv * L; e += nt) {
    const int v = e / L, i = e % L;
    U[i][v] = make_float2(o[2 * e], o[2 * e + 1]);
  }
  for (int e = tid; e < nb * L; e += nt) {
    const int v = e / L, i = e % L;
    V[i][v] = make_float2(t[2 * e], t[2 * e + 1]);
  }
  if (tid == 0) bad = 0;
  __syncthreads();
  // G = U^H U + eps I, B = U^H V
  for (int e = tid; e < nv * (nv + nb); e += nt) {
    const int a = e / (nv + nb), c = e % (nv + nb);
    float2 acc = make_float2(0.f, 0.f);
    for (int i = 0; i < L; ++i) {
      const float2 u = U[i][a], w = c < nv ? U[i][c] : V[i][c - nv];
      acc.x += u.x * w.x + u.y * w.y;
      acc.y += u.x * w.y - u.y * w.x;
    }
    if (c < nv) {
      if (a == c) acc.x += LOSS_EPS;
      G[a][c] = acc;
    } else {
      Bm[a][c - nv] = acc;
    }
  }
  __syncthreads();
  // Cholesky G = C C^H (lower, in place) and F = G^-1 B (thread 0; nv <= 16)
  if (tid == 0) {
    for (int c = 0; c < nv; ++c) {
      float p = G[c][c].x;
      for (int k = 0; k < c; ++k) p -= G[c][k].x * G[c][k].x + G[c][k].y * G[c][k].y;
      if (!(p > 0.f)) {
        bad = 1;
        p = 1.f;
      }
      const float d = sqrtf(p);
      G[c][c] = make_float2(d, 0.f);
      for (int r = c + 1; r < nv; ++r) {
        float2 v = G[r][c];
        for (int k = 0; k < c; ++k) {   // v -= G[r][k] conj(G[c][k])
          const float2 a = G[r][k], b = G[c][k];
          v.x -= a.x * b.x + a.y * b.y;
          v.y -= a.y * b.x - a.x * b.y;
        }
        G[r][c] = make_float2(v.x / d, v.y / d);
      }
    }
    for (int j = 0; j < nb; ++j) {
      float2 y[NVMAX];
      for (int r = 0; r < nv; ++r) {   // forward: C y = B
        float2 v = Bm[r][j];
        for (int k = 0; k < r; ++k) {
          const float2 a = G[r][k];
          v.x -= a.x * y[k].x - a.y * y[k].y;
          v.y -= a.x * y[k].y + a.y * y[k].x;
        }
        y[r] = make_float2(v.x / G[r][r].x, v.y / G[r][r].x);
      }
      for (int r = nv - 1; r >= 0; --r) {   // backward: C^H f = y
        float2 v = y[r];
        for (int k = r + 1; k < nv; ++k) {   // v -= conj(G[k][r]) f_k
          const float2 a = G[k][r], f = F[k][j];
          v.x -= a.x * f.x + a.y * f.y;
          v.y -= a.x * f.y - a.y * f.x;
        }
        F[r][j] = make_float2(v.x / G[r][r].x, v.y / G[r][r].x);
      }
    }
  }
  __syncthreads();
  // R = V - U F, ||V||^2, captured part tr(B^H F)
  for (int e = tid; e < L * nb; e += nt) {
    const int i = e / nb, j = e % nb;
    float2 v = V[i][j];
    for (int a = 0; a < nv; ++a) {
      const float2 u = U[i][a], f = F[a][j];
      v.x -= u.x * f.x - u.y * f.y;
      v.y -= u.x * f.y + u.y * f.x;
    }
    R[i][j] = v;
  }
  if (tid == 0) {
    float sv = 0.f, sc = 0.f;
    for (int i = 0; i < L; ++i)
      for (int j = 0; j < nb; ++j) sv += V[i][j].x * V[i][j].x + V[i][j].y * V[i][j].y;
    for (int a = 0; a < nv; ++a)
      for (int j = 0; j < nb; ++j) sc += Bm[a][j].x * F[a][j].x + Bm[a][j].y * F[a][j].y;
    vn2 = fmaxf(sv, 1e-30f);
    cap = sc;
    loss[s] = bad ? 1.f : (sv - sc) / vn2;
  }
  __syncthreads();
  // d loss / d(Re, Im) U = 2 (Re, Im) of -(R F^H) / ||V||^2, times scale
  const float f2 = bad ? 0.f : -2.f * scale / vn2;
  float* g = gout + (size_t)s * nv * L * 2;
  for (int e = tid; e < nv * L; e += nt) {
    const int a = e / L, i = e % L;
    float2 acc = make_float2(0.f, 0.f);
    for (int j = 0; j < nb; ++j) {   // R[i][j] conj(F[a][j])
      const float2 r = R[i][j], f = F[a][j];
      acc.x += r.x * f.x + r.y * f.y;
      acc.y += r.y * f.x - r.x * f.y;
    }
    g[2 * e] = f2 * acc.x;
    g[2 * e + 1] = f2 * acc.y;
  }
}

// ------------------------------------------------------------ Adam
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, size_t n, float lr, float b1, float b2,
                            float c1, float c2, float eps) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace

// ------------------------------------------------------------------ the network object
struct bs_cnn {
  int nvec, Mp, L, OUT;
  int cmax, smax;          // capacity: cells and samples per call
  size_t nparam;
  size_t off_w[NCONV], off_b[NCONV], off_dw[3], off_db[3];
  float* d_p;              // parameters
  float* d_g;              // gradients
  float* d_m;              // Adam moments
  float* d_v;
  long step;
  // activations (capacity cmax cells, smax samples)
  float* x;                // cmax x 3 x 64 x 64
  float* z[NCONV];         // conv outputs (post-ReLU), before pooling
  float* pl[NCONV];        // pooled outputs (pl[3] = features)
  float* kf;               // smax x KF
  float* h0;               // smax x (FEAT + KF)
  float* h1;
  float* h2;
  float* out;              // smax x OUT
  // backward scratch
  float* gout;
  float* gh0;
  float* gh1;
  float* gh2;
  float* gpl;              // max pooled plane gradients
  float* gz;               // max conv-output gradients
  float* gtmp;
  float* wpart;            // conv weight-gradient partials
  float* loss;             // smax
  // encode inputs
  uint16_t* phase;
  double* table;
  long* toff;
  int* nph;
  int* hex;
  double* Q;
  float* tgt;
  size_t table_cap;
};

namespace {

constexpr int WSPLIT = 32;

template <typename T>
int calloc_dev(T** p, size_t n, const char* what) {
  *p = nullptr;
  if (!n) return BS_OK;
  cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    bs_set_error("cudaMalloc(%s) failed: %s", what, cudaGetErrorString(e));
    return BS_ENOMEM;
  }
  return BS_OK;
}

#define TRYC(x)            \
  do {                     \
    int r__ = (x);         \
    if (r__) return r__;   \
  } while (0)

int conv_forward(bs_cnn* m, int nc, cudaStream_t s) {
  const float* in = m->x;
  for (int l = 0; l < NCONV; ++l) {
    const int S = SIDE[l], ci = CIN[l], co = COUT[l];
    dim3 grid((S * S + 255) / 256, (co + CO_T - 1) / CO_T, nc);
    conv_fwd_kernel<<<grid, 256, CO_T * ci * 9 * sizeof(float), s>>>(
        in, m->d_p + m->off_w[l], m->d_p + m->off_b[l], ci, co, S, m->z[l]);
    BS_CHECK_LAUNCH("conv_fwd_kernel");
    const size_t planes = (size_t)nc * co, tot = planes * (S / 2) * (S / 2);
    pool_fwd_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(m->z[l], S, planes, m->pl[l]);
    BS_CHECK_LAUNCH("pool_fwd_kernel");
    in = m->pl[l];
  }
  return BS_OK;
}

int sgemm(bool ta, bool tb, int M, int N, int K, const float* A, int lda, const float* B, int ldb,
          const float* bias, bool relu, float* C, int ldc, cudaStream_t s) {
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  if (!ta && !tb) sgemm_kernel<false, false><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, bias, relu, C, ldc);
  else if (!ta && tb) sgemm_kernel<false, true><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, bias, relu, C, ldc);
  else if (ta && !tb) sgemm_kernel<true, false><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, bias, relu, C, ldc);
  else sgemm_kernel<true, true><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, bias, relu, C, ldc);
  BS_CHECK_LAUNCH("sgemm_kernel");
  return BS_OK;
}

int head_forward(bs_cnn* m, int nc, int kper, cudaStream_t s) {
  const int ns = nc * kper, W0 = FEAT + KF;
  head_input_kernel<<<(ns * W0 + 255) / 256, 256, 0, s>>>(m->pl[NCONV - 1], m->kf, ns, kper, m->h0);
  BS_CHECK_LAUNCH("head_input_kernel");
  TRYC(sgemm(false, true, ns, HID, W0, m->h0, W0, m->d_p + m->off_dw[0], W0, m->d_p + m->off_db[0],
             true, m->h1, HID, s));
  TRYC(sgemm(false, true, ns, HID, HID, m->h1, HID, m->d_p + m->off_dw[1], HID,
             m->d_p + m->off_db[1], true, m->h2, HID, s));
  TRYC(sgemm(false, true, ns, m->OUT, HID, m->h2, HID, m->d_p + m->off_dw[2], HID,
             m->d_p + m->off_db[2], false, m->out, m->OUT, s));
  return BS_OK;
}

// gradients of everything from m->gout (ns x OUT) into m->d_g
int backward(bs_cnn* m, int nc, int kper, cudaStream_t s) {
  const int ns = nc * kper, W0 = FEAT + KF;
  // dense 3
  TRYC(sgemm(true, false, m->OUT, HID, ns, m->gout, m->OUT, m->h2, HID, nullptr, false,
             m->d_g + m->off_dw[2], HID, s));
  colsum_kernel<<<(m->OUT + 255) / 256, 256, 0, s>>>(m->gout, ns, m->OUT, m->OUT, m->d_g + m->off_db[2]);
  BS_CHECK_LAUNCH("colsum_kernel");
  TRYC(sgemm(false, false, ns, HID, m->OUT, m->gout, m->OUT, m->d_p + m->off_dw[2], HID, nullptr,
             false, m->gh2, HID, s));
  relu_mask_kernel<<<(unsigned)(((size_t)ns * HID + 255) / 256), 256, 0, s>>>(m->gh2, m->h2, (size_t)ns * HID);
  BS_CHECK_LAUNCH("relu_mask_kernel");
  // dense 2
  TRYC(sgemm(true, false, HID, HID, ns, m->gh2, HID, m->h1, HID, nullptr, false,
             m->d_g + m->off_dw[1], HID, s));
  colsum_kernel<<<(HID + 255) / 256, 256, 0, s>>>(m->gh2, ns, HID, HID, m->d_g + m->off_db[1]);
  BS_CHECK_LAUNCH("colsum_kernel");
  TRYC(sgemm(false, false, ns, HID, HID, m->gh2, HID, m->d_p + m->off_dw[1], HID, nullptr, false,
             m->gh1, HID, s));
  relu_mask_kernel<<<(unsigned)(((size_t)ns * HID + 255) / 256), 256, 0, s>>>(m->gh1, m->h1, (size_t)ns * HID);
  BS_CHECK_LAUNCH("relu_mask_kernel");
  // dense 1
  TRYC(sgemm(true, false, HID, W0, ns, m->gh1, HID, m->h0, W0, nullptr, false,
             m->d_g + m->off_dw[0], W0, s));
  colsum_kernel<<<(HID + 255) / 256, 256, 0, s>>>(m->gh1, ns, HID, HID, m->d_g + m->off_db[0]);
  BS_CHECK_LAUNCH("colsum_kernel");
  TRYC(sgemm(false, false, ns, W0, HID, m->gh1, HID, m->d_p + m->off_dw[0], W0, nullptr, false,
             m->gh0, W0, s));
  // features: sum over the samples of each cell
  feat_grad_kernel<<<(nc * FEAT + 255) / 256, 256, 0, s>>>(m->gh0, nc, kper, m->gpl);
  BS_CHECK_LAUNCH("feat_grad_kernel");
  // convolution layers, last to first
  for (int l = NCONV - 1; l >= 0; --l) {
    const int S = SIDE[l], ci = CIN[l], co = COUT[l];
    const size_t planes = (size_t)nc * co;
    pool_bwd_kernel<<<(unsigned)((planes * S * S + 255) / 256), 256, 0, s>>>(m->gpl, m->z[l], S,
                                                                             planes, m->gz);
    BS_CHECK_LAUNCH("pool_bwd_kernel");
    const float* in = l == 0 ? m->x : m->pl[l - 1];
    conv_bwd_weight_kernel<<<dim3(co * (ci + 1), WSPLIT), 256, 0, s>>>(m->gz, in, nc, ci, co, S,
                                                                        WSPLIT, m->wpart);
    BS_CHECK_LAUNCH("conv_bwd_weight_kernel");
    conv_wgrad_reduce_kernel<<<(co * (ci + 1) * 9 + 255) / 256, 256, 0, s>>>(
        m->wpart, ci, co, WSPLIT, m->d_g + m->off_w[l], m->d_g + m->off_b[l]);
    BS_CHECK_LAUNCH("conv_wgrad_reduce_kernel");
    if (l > 0) {
      dim3 grid((S * S + 255) / 256, (ci + CI_T - 1) / CI_T, nc);
      conv_bwd_data_kernel<<<grid, 256, CI_T * co * 9 * sizeof(float), s>>>(
          m->gz, m->d_p + m->off_w[l], ci, co, S, m->gtmp);
      BS_CHECK_LAUNCH("conv_bwd_data_kernel");
      // gtmp is the gradient of the pooled output of layer l-1
      cudaError_t e = cudaMemcpyAsync(m->gpl, m->gtmp, (size_t)nc * ci * S * S * sizeof(float),
                                      cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) return bs_cuda_status(e, "cnn backward");
    }
  }
  return BS_OK;
}

int stage_inputs(bs_cnn* m, const uint16_t* phase, const double* table, const long* toff,
                 const int* nph, const int* hex, int nc, const double* Q, int kper,
                 cudaStream_t s) {
  const int ns = nc * kper;
  std::vector<long> to(nc);
  std::vector<int> np(nc);
  cudaError_t e = cudaMemcpy(to.data(), toff, nc * sizeof(long), cudaMemcpyDefault);
  if (e == cudaSuccess) e = cudaMemcpy(np.data(), nph, nc * sizeof(int), cudaMemcpyDefault);
  if (e != cudaSuccess) return bs_cuda_status(e, "cnn table offsets");
  long tot = 0;
  for (int c = 0; c < nc; ++c) {
    if (to[c] < 0 || np[c] < 1) {
      bs_set_error("cnn: cell %d has a negative table offset or no phase", c);
      return BS_EINVAL;
    }
    tot = std::max(tot, to[c] + 3L * np[c]);
  }
  e = cudaMemcpyAsync(m->phase, phase, (size_t)nc * IMG * IMG * 2, cudaMemcpyDefault, s);
  if ((size_t)tot > m->table_cap) {
    bs_set_error("cnn: property tables exceed the capacity (%ld > %zu doubles)", tot, m->table_cap);
    return BS_EINVAL;
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->table, table, tot * sizeof(double), cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->toff, toff, nc * sizeof(long), cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->nph, nph, nc * sizeof(int), cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->hex, hex, nc * sizeof(int), cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->Q, Q, (size_t)ns * 2 * sizeof(double), cudaMemcpyDefault, s);
  if (e != cudaSuccess) return bs_cuda_status(e, "cnn inputs");
  encode_kernel<<<(unsigned)(((size_t)nc * IMG * IMG + 255) / 256), 256, 0, s>>>(
      m->phase, m->table, m->toff, m->nph, nc, m->x);
  BS_CHECK_LAUNCH("encode_kernel");
  kfeat_kernel<<<(ns + 255) / 256, 256, 0, s>>>(m->Q, m->hex, ns, kper, m->kf);
  BS_CHECK_LAUNCH("kfeat_kernel");
  // the stack copies above must complete before the vectors go out of scope
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bs_cuda_status(e, "cnn inputs");
  return BS_OK;
}

int check_call(const bs_cnn* m, int nc, int kper) {
  if (!m || nc < 1 || kper < 1 || nc > m->cmax || nc * kper > m->smax) {
    bs_set_error("cnn: need 1 <= ncells <= %d and ncells * kper <= %d", m ? m->cmax : 0,
                 m ? m->smax : 0);
    return BS_EINVAL;
  }
  return BS_OK;
}

}  // namespace

extern "C" int bs_cnn_create(int nvec, int Mp, int max_cells, int max_samples, bs_cnn** out) {
  if (!out || nvec < 1 || nvec > NVMAX || Mp < 0 || Mp > 3 || max_cells < 1 ||
      max_samples < max_cells) {
    bs_set_error("bs_cnn_create: need 1 <= nvec <= %d, 0 <= Mp <= 3, max_samples >= max_cells >= 1",
                 NVMAX);
    return BS_EINVAL;
  }
  *out = nullptr;
  bs_cnn* m = new bs_cnn();
  m->nvec = nvec;
  m->Mp = Mp;
  m->L = 2 * (2 * Mp + 1) * (2 * Mp + 1);
  m->OUT = nvec * m->L * 2;
  m->cmax = max_cells;
  m->smax = max_samples;
  size_t o = 0;
  for (int l = 0; l < NCONV; ++l) {
    m->off_w[l] = o;
    o += (size_t)COUT[l] * CIN[l] * 9;
    m->off_b[l] = o;
    o += COUT[l];
  }
  const int din[3] = {FEAT + KF, HID, HID}, dout[3] = {HID, HID, m->OUT};
  for (int l = 0; l < 3; ++l) {
    m->off_dw[l] = o;
    o += (size_t)din[l] * dout[l];
    m->off_db[l] = o;
    o += dout[l];
  }
  m->nparam = o;
  const size_t C = max_cells, Sm = max_samples;
  int r = BS_OK;
  if (!r) r = calloc_dev(&m->d_p, o, "cnn parameters");
  if (!r) r = calloc_dev(&m->d_g, o, "cnn gradients");
  if (!r) r = calloc_dev(&m->d_m, o, "cnn moments");
  if (!r) r = calloc_dev(&m->d_v, o, "cnn moments");
  if (!r) r = calloc_dev(&m->x, C * 3 * IMG * IMG, "cnn input");
  size_t zmax = 0;
  for (int l = 0; !r && l < NCONV; ++l) {
    const size_t zs = C * COUT[l] * SIDE[l] * SIDE[l];
    zmax = std::max(zmax, zs);
    r = calloc_dev(&m->z[l], zs, "cnn activations");
    if (!r) r = calloc_dev(&m->pl[l], zs / 4, "cnn pooled");
  }
  const size_t W0 = FEAT + KF;
  if (!r) r = calloc_dev(&m->kf, Sm * KF, "cnn k features");
  if (!r) r = calloc_dev(&m->h0, Sm * W0, "cnn h0");
  if (!r) r = calloc_dev(&m->h1, Sm * HID, "cnn h1");
  if (!r) r = calloc_dev(&m->h2, Sm * HID, "cnn h2");
  if (!r) r = calloc_dev(&m->out, Sm * m->OUT, "cnn out");
  if (!r) r = calloc_dev(&m->gout, Sm * m->OUT, "cnn gout");
  if (!r) r = calloc_dev(&m->gh0, Sm * W0, "cnn gh0");
  if (!r) r = calloc_dev(&m->gh1, Sm * HID, "cnn gh1");
  if (!r) r = calloc_dev(&m->gh2, Sm * HID, "cnn gh2");
  if (!r) r = calloc_dev(&m->gpl, std::max(zmax / 4, C * FEAT), "cnn pooled gradients");
  if (!r) r = calloc_dev(&m->gz, zmax, "cnn conv gradients");
  if (!r) r = calloc_dev(&m->gtmp, zmax, "cnn scratch");
  if (!r) r = calloc_dev(&m->wpart, (size_t)WSPLIT * 32 * 33 * 9, "cnn weight partials");
  if (!r) r = calloc_dev(&m->loss, Sm, "cnn loss");
  if (!r) r = calloc_dev(&m->phase, C * IMG * IMG, "cnn phase maps");
  m->table_cap = C * 3 * 64;
  if (!r) r = calloc_dev(&m->table, m->table_cap, "cnn tables");
  if (!r) r = calloc_dev(&m->toff, C, "cnn table offsets");
  if (!r) r = calloc_dev(&m->nph, C, "cnn phase counts");
  if (!r) r = calloc_dev(&m->hex, C, "cnn lattice flags");
  if (!r) r = calloc_dev(&m->Q, Sm * 2, "cnn wavevectors");
  if (!r) r = calloc_dev(&m->tgt, Sm * 16 * m->L * 2, "cnn targets");
  if (!r && cudaMemset(m->d_m, 0, o * 4) != cudaSuccess) r = BS_ECUDA;
  if (!r && cudaMemset(m->d_v, 0, o * 4) != cudaSuccess) r = BS_ECUDA;
  if (r) {
    bs_cnn_destroy(m);
    return r;
  }
  *out = m;
  return BS_OK;
}

extern "C" int bs_cnn_destroy(bs_cnn* m) {
  if (!m) return BS_OK;
  void* ps[] = {m->d_p, m->d_g, m->d_m, m->d_v, m->x, m->kf, m->h0, m->h1, m->h2, m->out, m->gout,
                m->gh0, m->gh1, m->gh2, m->gpl, m->gz, m->gtmp, m->wpart, m->loss, m->phase,
                m->table, m->toff, m->nph, m->hex, m->Q, m->tgt};
  for (void* p : ps) cudaFree(p);
  for (int l = 0; l < NCONV; ++l) {
    cudaFree(m->z[l]);
    cudaFree(m->pl[l]);
  }
  delete m;
  return BS_OK;
}

extern "C" int bs_cnn_num_params(const bs_cnn* m, long long* n) {
  if (!m || !n) {
    bs_set_error("bs_cnn_num_params: NULL argument");
    return BS_EINVAL;
  }
  *n = (long long)m->nparam;
  return BS_OK;
}

extern "C" int bs_cnn_set_params(bs_cnn* m, const float* p) {
  if (!m || !p) {
    bs_set_error("bs_cnn_set_params: NULL argument");
    return BS_EINVAL;
  }
  cudaError_t e = cudaMemcpy(m->d_p, p, m->nparam * 4, cudaMemcpyDefault);
  if (e == cudaSuccess) e = cudaMemset(m->d_m, 0, m->nparam * 4);
  if (e == cudaSuccess) e = cudaMemset(m->d_v, 0, m->nparam * 4);
  if (e != cudaSuccess) return bs_cuda_status(e, "bs_cnn_set_params");
  m->step = 0;
  return BS_OK;
}

extern "C" int bs_cnn_get_params(const bs_cnn* m, float* p, float* grad) {
  if (!m || (!p && !grad)) {
    bs_set_error("bs_cnn_get_params: NULL argument");
    return BS_EINVAL;
  }
  cudaError_t e = cudaSuccess;
  if (p) e = cudaMemcpy(p, m->d_p, m->nparam * 4, cudaMemcpyDefault);
  if (e == cudaSuccess && grad) e = cudaMemcpy(grad, m->d_g, m->nparam * 4, cudaMemcpyDefault);
  if (e != cudaSuccess) return bs_cuda_status(e, "bs_cnn_get_params");
  return BS_OK;
}

extern "C" int bs_cnn_forward(bs_cnn* m, const uint16_t* phase, const double* table,
                              const long* toff, const int* nph, const int* hex, int ncells,
                              const double* Q, int kper, float* U_out, void* stream) {
  TRYC(check_call(m, ncells, kper));
  if (!phase || !table || !toff || !nph || !hex || !Q || !U_out) {
    bs_set_error("bs_cnn_forward: NULL argument");
    return BS_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  TRYC(stage_inputs(m, phase, table, toff, nph, hex, ncells, Q, kper, s));
  TRYC(conv_forward(m, ncells, s));
  TRYC(head_forward(m, ncells, kper, s));
  cudaError_t e = cudaMemcpyAsync(U_out, m->out, (size_t)ncells * kper * m->OUT * 4,
                                  cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bs_cuda_status(e, "bs_cnn_forward");
  return BS_OK;
}

extern "C" int bs_cnn_train_step(bs_cnn* m, const uint16_t* phase, const double* table,
                                 const long* toff, const int* nph, const int* hex, int ncells,
                                 const double* Q, int kper, const float* V, int nb, float lr,
                                 float* loss_out, void* stream) {
  TRYC(check_call(m, ncells, kper));
  if (!phase || !table || !toff || !nph || !hex || !Q || !V || nb < 1 || nb > 16) {
    bs_set_error("bs_cnn_train_step: NULL argument or nb outside [1, 16]");
    return BS_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int ns = ncells * kper;
  TRYC(stage_inputs(m, phase, table, toff, nph, hex, ncells, Q, kper, s));
  cudaError_t e = cudaMemcpyAsync(m->tgt, V, (size_t)ns * nb * m->L * 2 * 4, cudaMemcpyDefault, s);
  if (e != cudaSuccess) return bs_cuda_status(e, "bs_cnn_train_step targets");
  TRYC(conv_forward(m, ncells, s));
  TRYC(head_forward(m, ncells, kper, s));
  loss_kernel<<<ns, 128, 0, s>>>(m->out, m->tgt, m->L, m->nvec, nb, 1.f / ns, m->loss, m->gout);
  BS_CHECK_LAUNCH("loss_kernel");
  TRYC(backward(m, ncells, kper, s));
  if (lr > 0.f) {
    m->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)m->step), c2 = 1.f - powf(b2, (float)m->step);
    adam_kernel<<<(unsigned)((m->nparam + 255) / 256), 256, 0, s>>>(m->d_p, m->d_g, m->d_m, m->d_v,
                                                                    m->nparam, lr, b1, b2, c1, c2,
                                                                    1e-8f);
    BS_CHECK_LAUNCH("adam_kernel");
  }
  if (loss_out) {
    e = cudaMemcpyAsync(loss_out, m->loss, ns * sizeof(float), cudaMemcpyDefault, s);
    if (e != cudaSuccess) return bs_cuda_status(e, "bs_cnn_train_step loss");
  }
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bs_cuda_status(e, "bs_cnn_train_step");
  return BS_OK;
}
