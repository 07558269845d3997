// Mixed-precision eigen path: an FP32 Householder reduction gives
// approximate eigenvectors of the reduced matrix C(k), and one FP64
// Rayleigh-Ritz projection with the FP64 C(k) turns them into eigenvalues
// accurate to FP64 working accuracy times (eps32 ||C|| / gap)^2.
//
//   C32(k) --FP32 Householder--> T (real after a diagonal unitary scaling)
//   T --FP64 bisection--> lambda_1..lambda_{b+1}
//   T --FP64 inverse iteration + MGS--> y_1..y_b
//   y --phases of beta, FP32 reflectors--> X (n x b)
//   X --FP64: C X, X^dagger X, X^dagger C X, Cholesky + Jacobi--> Ritz pairs
//   Ritz pairs --FP64 residuals R, E = R^dagger R--> Lehmann lower bounds
//
// b = nbands + guard vectors, so clusters at the edge of the wanted band
// stay inside the subspace.  Each Ritz value is an upper bound of its
// eigenvalue; Lehmann's method (certify_kernel) gives a lower bound from
// E and a bound rho on the next eigenvalue (from T's eigenvalues), and the
// difference is checked against the requested tolerance; wavevectors that
// miss it are reported with BS_ENOCONV.
#include <float.h>
#include <math.h>

#include "bs_internal.h"

namespace {

// ------------------------------------------------------------ builder
// C64 full (FP64) and C32 (FP32; lower triangle, or all of it) from the
// full monomials.
__global__ void builder_mixed_kernel(const zd* __restrict__ Cm, int n,
                                     const double* __restrict__ Q, int nk, double q1x, double q1y,
                                     double q2x, double q2y, zd* __restrict__ C64,
                                     zf* __restrict__ C32, bool full32) {
  constexpr int KB = 32;
  __shared__ double coef[KB][6];
  const size_t nn = (size_t)n * n;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = e < nn;
  const bool lower = live && (full32 || (int)(e % n) >= (int)(e / n));
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
      C64[(size_t)(k0 + b) * nn + e] = zmake(re, im);
      if (lower) C32[(size_t)(k0 + b) * nn + e] = make_float2((float)re, (float)im);
    }
  }
}

// ------------------------------------------------------------ tridiagonal eigenvectors
// 1/q: FP32 seed refined by two Newton-Raphson steps r <- r + r (1 - q r)
// (FP64 division is a long sequence on GB300); exact division outside the
// FP32 normal range.
__device__ __forceinline__ double rcp64(double q) {
  const double aq = fabs(q);
  if (aq > 1e-36 && aq < 1e36) {
    double r = (double)__frcp_rn((float)q);
    r = fma(r, fma(-q, r, 1.0), r);
    r = fma(r, fma(-q, r, 1.0), r);
    return r;
  }
  return 1.0 / q;
}

__device__ __forceinline__ double hash_unit(unsigned a, unsigned b) {
  unsigned h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u;
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  h *= 0x297A2D39u;
  h ^= h >> 15;
  return (double)h * (2.0 / 4294967296.0) - 1.0;
}

// Inverse iteration on T - sigma I (Gaussian elimination with partial
// pivoting of the tridiagonal), two solves from a pseudo-random start, then
// modified Gram-Schmidt of the block in FP64.  Thread i < b owns vector i.
// Also writes the diagonal unitary scaling D (T_complex = D T_real D^dagger).
// in_smem: the b x n block lives in shared memory while it is built and
// orthogonalised (the b (b + 1) / 2 dependent dot products of the
// Gram-Schmidt sweep then run on shared memory), and is stored at the end;
// used when there are few problems (one large CTA per SM), otherwise the
// block stays in global memory and many small CTAs share each SM.
__global__ void tri_eigvec_kernel(const double* __restrict__ de, const zd* __restrict__ beta,
                                  const double* __restrict__ lam, int n, int b, int lstride,
                                  double* __restrict__ scratch, double* __restrict__ Y,
                                  zd* __restrict__ phase, bool in_smem) {
  extern __shared__ double ysh[];
  __shared__ double red[32];
  const int k = blockIdx.x, tid = threadIdx.x;
  const double* d = de + (size_t)k * 2 * n;
  const double* e = d + n;
  double* yg = Y + (size_t)k * b * n;
  double* y = in_smem ? ysh : yg;
  if (tid < b) {
    const int i = tid;
    double* u0 = scratch + ((size_t)k * b + i) * 5 * n;
    double* u1 = u0 + n;
    double* u2 = u1 + n;
    double* ml = u2 + n;
    double* pv = ml + n;   // 1 where rows r, r+1 were interchanged
    double tnorm = 0.0;
    for (int r = 0; r < n; ++r)
      tnorm = fmax(tnorm, fabs(d[r]) + (r > 0 ? e[r - 1] : 0.0) + (r + 1 < n ? e[r] : 0.0));
    const double tiny = DBL_EPSILON * fmax(tnorm, DBL_MIN);
    const double sigma = lam[(size_t)k * lstride + i];
    // factor: u0, u1, u2 = the three diagonals of U; ml = multipliers of L
    double al = d[0] - sigma, bt = n > 1 ? e[0] : 0.0;
    for (int r = 0; r + 1 < n; ++r) {
      const double g = e[r];
      const double dn = d[r + 1] - sigma, en = r + 2 < n ? e[r + 1] : 0.0;
      if (fabs(al) >= fabs(g)) {
        const double a0 = fabs(al) < tiny ? (al < 0 ? -tiny : tiny) : al;
        const double ia = rcp64(a0);
        const double mlt = g * ia;
        u0[r] = ia; u1[r] = bt; u2[r] = 0.0; ml[r] = mlt; pv[r] = 0.0;
        al = dn - mlt * bt;
        bt = en;
      } else {
        const double mlt = al * rcp64(g);
        u0[r] = rcp64(g); u1[r] = dn; u2[r] = en; ml[r] = mlt; pv[r] = 1.0;
        al = bt - mlt * dn;
        bt = -mlt * en;
      }
    }
    u0[n - 1] = rcp64(fabs(al) < tiny ? (al < 0 ? -tiny : tiny) : al);   // u0 holds 1/pivot
    double* yi = y + (size_t)i * n;
    for (int r = 0; r < n; ++r) yi[r] = hash_unit(r, i + 977u * k);
    for (int it = 0; it < 2; ++it) {
      // forward: L^-1 with interchanges
      for (int r = 0; r + 1 < n; ++r) {
        const double mlt = ml[r];
        if (pv[r] != 0.0) {   // interchange rows r, r+1
          const double t = yi[r];
          yi[r] = yi[r + 1];
          yi[r + 1] = t - mlt * yi[r];
        } else {
          yi[r + 1] -= mlt * yi[r];
        }
      }
      // backward: U y = rhs
      double amax = 0.0;
      for (int r = n - 1; r >= 0; --r) {
        double s = yi[r];
        if (r + 1 < n) s -= u1[r] * yi[r + 1];
        if (r + 2 < n) s -= u2[r] * yi[r + 2];
        yi[r] = s * u0[r];
        amax = fmax(amax, fabs(yi[r]));
      }
      const double sc = amax > 0.0 ? 1.0 / amax : 1.0;
      for (int r = 0; r < n; ++r) yi[r] *= sc;
    }
  }
  if (tid == 0) {
    zd ph = zmake(1.0, 0.0);
    zd* pk = phase + (size_t)k * n;
    pk[0] = ph;
    for (int r = 0; r + 1 < n; ++r) {
      const zd bt = beta[(size_t)k * n + r];
      const double ab = hypot(bt.x, bt.y);
      if (ab > 0.0) ph = zmul(ph, zmake(bt.x / ab, bt.y / ab));
      pk[r + 1] = ph;
    }
  }
  __syncthreads();
  // modified Gram-Schmidt over the b vectors (block-cooperative)
  for (int i = 0; i < b; ++i) {
    double* yi = y + (size_t)i * n;
    for (int jj = 0; jj <= i; ++jj) {
      const double* yj = y + (size_t)jj * n;
      double s = 0.0;
      for (int r = tid; r < n; r += blockDim.x) s = fma(yj[r], yi[r], s);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if ((tid & 31) == 0) red[tid >> 5] = s;
      __syncthreads();
      double tot = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
      __syncthreads();
      if (jj < i) {
        for (int r = tid; r < n; r += blockDim.x) yi[r] = fma(-tot, yj[r], yi[r]);
      } else {
        const double sc = tot > 0.0 ? 1.0 / sqrt(tot) : 0.0;
        for (int r = tid; r < n; r += blockDim.x) yi[r] *= sc;
      }
      __syncthreads();
    }
  }
  if (in_smem)
    for (int q = tid; q < b * n; q += blockDim.x) yg[q] = ysh[q];
}

// ------------------------------------------------------------ back-transformation
// X = Q D y with Q = H_0 H_1 ... H_{n-2}: one warp per column, reflectors
// applied from the last to the first, in FP32 (the reflectors are FP32).
__global__ void backtransform_kernel(const zf* __restrict__ A32, const double* __restrict__ tau,
                                     const zd* __restrict__ phase, const double* __restrict__ Y,
                                     int n, int b, zf* __restrict__ X32, zd* __restrict__ X64) {
  const int k = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.y * (blockDim.x >> 5) + warp;
  if (i >= b) return;
  const zf* a = A32 + (size_t)k * n * n;
  const double* tk = tau + (size_t)k * n;
  const zd* pk = phase + (size_t)k * n;
  const double* y = Y + ((size_t)k * b + i) * n;
  zf* x = X32 + ((size_t)k * b + i) * n;
  for (int r = lane; r < n; r += 32) {
    const zd v = zscale(pk[r], y[r]);
    x[r] = make_float2((float)v.x, (float)v.y);
  }
  __syncwarp();
  for (int j = n - 2; j >= 0; --j) {
    const float t = (float)tk[j];
    if (t == 0.0f) continue;
    // s = v^dagger x over rows j+1..n-1 (v[j+1] = 1)
    float sr = 0.f, si = 0.f;
    for (int r = j + 1 + lane; r < n; r += 32) {
      const zf v = r == j + 1 ? make_float2(1.f, 0.f) : a[r + (size_t)j * n];
      const zf xv = x[r];
      sr = fmaf(v.x, xv.x, fmaf(v.y, xv.y, sr));
      si = fmaf(v.x, xv.y, fmaf(-v.y, xv.x, si));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, o);
      si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    const zf ts = make_float2(t * sr, t * si);
    for (int r = j + 1 + lane; r < n; r += 32) {
      const zf v = r == j + 1 ? make_float2(1.f, 0.f) : a[r + (size_t)j * n];
      x[r] = zsub(x[r], zmul(v, ts));
    }
    __syncwarp();
  }
  zd* xo = X64 + (size_t)k * n * b + (size_t)i * n;
  for (int r = lane; r < n; r += 32) xo[r] = zmake(x[r].x, x[r].y);
}

// ------------------------------------------------------------ small eigenproblem
// H w = theta G w for b x b Hermitian H and HPD G (b <= 32, even): Cholesky
// of G, standard form, cyclic parallel Jacobi with the round-robin pairing.
constexpr int BMAX = 32;

__global__ void small_eig_kernel(const zd* __restrict__ Gg, const zd* __restrict__ Hg, int b,
                                 double* __restrict__ theta, zd* __restrict__ Wg,
                                 int* __restrict__ stat) {
  __shared__ zd G[BMAX][BMAX + 1], A[BMAX][BMAX + 1], V[BMAX][BMAX + 1];
  __shared__ double cs_[BMAX / 2], sn_[BMAX / 2];
  __shared__ zd ph_[BMAX / 2];
  __shared__ int pp_[BMAX / 2], qq_[BMAX / 2];
  __shared__ double offn, totn;
  __shared__ int fail;
  const int k = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const zd* gk = Gg + (size_t)k * b * b;
  const zd* hk = Hg + (size_t)k * b * b;
  for (int e = tid; e < b * b; e += nt) {
    const int r = e % b, c = e / b;
    G[r][c] = gk[e];
    A[r][c] = hk[e];
  }
  if (tid == 0) fail = 0;
  __syncthreads();
  // Cholesky G = L L^dagger (lower, in place), column by column
  for (int c = 0; c < b; ++c) {
    if (tid == 0) {
      double p = G[c][c].x;
      for (int t = 0; t < c; ++t) p -= G[c][t].x * G[c][t].x + G[c][t].y * G[c][t].y;
      if (!(p > 0.0)) {
        fail = 1;
        p = 1.0;
      }
      G[c][c] = zmake(sqrt(p), 0.0);
    }
    __syncthreads();
    for (int r = c + 1 + tid; r < b; r += nt) {
      zd s = G[r][c];
      for (int t = 0; t < c; ++t) s = zfnmac(G[r][t], G[c][t], s);
      G[r][c] = zscale(s, 1.0 / G[c][c].x);
    }
    __syncthreads();
  }
  // A <- L^-1 A L^-dagger: forward substitution on columns, then on rows
  for (int c = tid; c < b; c += nt)
    for (int r = 0; r < b; ++r) {
      zd s = A[r][c];
      for (int t = 0; t < r; ++t) s = zsub(s, zmul(G[r][t], A[t][c]));
      A[r][c] = zscale(s, 1.0 / G[r][r].x);
    }
  __syncthreads();
  for (int r = tid; r < b; r += nt)
    for (int c = 0; c < b; ++c) {
      zd s = A[r][c];
      for (int t = 0; t < c; ++t) s = zsub(s, zmul(A[r][t], zconj(G[c][t])));
      A[r][c] = zscale(s, 1.0 / G[c][c].x);
    }
  __syncthreads();
  // Hermitian part: H = X^dagger (C X) is Hermitian only to the accuracy of
  // the C X product, and one-sided rotations cannot remove an anti-Hermitian
  // residue, so the sweeps would never meet the stopping test
  for (int e = tid; e < b * b; e += nt) {
    const int r = e % b, c = e / b;
    if (r < c) {
      const zd h = zscale(zadd(A[r][c], zconj(A[c][r])), 0.5);
      A[r][c] = h;
      A[c][r] = zconj(h);
    }
  }
  __syncthreads();
  for (int e = tid; e < b * b; e += nt) {
    const int r = e % b, c = e / b;
    V[r][c] = zmake(r == c ? 1.0 : 0.0, 0.0);
    if (r == c) A[r][c].y = 0.0;
  }
  __syncthreads();
  __shared__ double red[4][2];
  const int np = b / 2;
  for (int sweep = 0; sweep < 20; ++sweep) {
    double o = 0.0, t = 0.0;
    for (int e = tid; e < b * b; e += nt) {
      const int r = e % b, c = e / b;
      const double m2 = A[r][c].x * A[r][c].x + A[r][c].y * A[r][c].y;
      t += m2;
      if (r != c) o += m2;
    }
    for (int sh = 16; sh > 0; sh >>= 1) {
      o += __shfl_xor_sync(0xffffffffu, o, sh);
      t += __shfl_xor_sync(0xffffffffu, t, sh);
    }
    if ((tid & 31) == 0) {
      red[tid >> 5][0] = o;
      red[tid >> 5][1] = t;
    }
    __syncthreads();
    if (tid == 0) {
      offn = red[0][0] + red[1][0] + red[2][0] + red[3][0];
      totn = red[0][1] + red[1][1] + red[2][1] + red[3][1];
    }
    __syncthreads();
    // off-diagonal Frobenius norm below 1e-12 of the whole: the Ritz values
    // then carry errors of order (1e-12 ||H||)^2 / gap, far below FP64 noise
    if (offn <= 1e-24 * totn) break;

    for (int rd = 0; rd < b - 1; ++rd) {
      if (tid < np) {
        int p, q;
        if (tid == 0) {
          p = rd % (b - 1);
          q = b - 1;
        } else {
          p = (rd + tid) % (b - 1);
          q = (rd - tid + (b - 1)) % (b - 1);
        }
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        const zd c = A[p][q];
        const double ca = hypot(c.x, c.y);
        double cs = 1.0, sn = 0.0;
        zd ph = zmake(1.0, 0.0);
        if (ca > 0.0) {
          ph = zmake(c.x / ca, c.y / ca);
          const double zeta = (A[q][q].x - A[p][p].x) / (2.0 * ca);
          const double t = zeta >= 0.0 ? 1.0 / (zeta + sqrt(1.0 + zeta * zeta))
                                       : -1.0 / (-zeta + sqrt(1.0 + zeta * zeta));
          cs = 1.0 / sqrt(1.0 + t * t);
          sn = t * cs;
        }
        pp_[tid] = p;
        qq_[tid] = q;
        cs_[tid] = cs;
        sn_[tid] = sn;
        ph_[tid] = ph;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J with J = [[cs, sn], [-sn conj(ph), cs conj(ph)]]
      for (int e = tid; e < np * b; e += nt) {
        const int u = e / b, r = e % b, p = pp_[u], q = qq_[u];
        const double cs = cs_[u], sn = sn_[u];
        const zd cph = zconj(ph_[u]);
        const zd ap = A[r][p], aq = zmul(A[r][q], cph);
        A[r][p] = zsub(zscale(ap, cs), zscale(aq, sn));
        A[r][q] = zadd(zscale(ap, sn), zscale(aq, cs));
        const zd vp = V[r][p], vq = zmul(V[r][q], cph);
        V[r][p] = zsub(zscale(vp, cs), zscale(vq, sn));
        V[r][q] = zadd(zscale(vp, sn), zscale(vq, cs));
      }
      __syncthreads();
      // rows: A <- J^dagger A
      for (int e = tid; e < np * b; e += nt) {
        const int u = e / b, c = e % b, p = pp_[u], q = qq_[u];
        const double cs = cs_[u], sn = sn_[u];
        const zd ap = A[p][c], aq = zmul(A[q][c], ph_[u]);
        A[p][c] = zsub(zscale(ap, cs), zscale(aq, sn));
        A[q][c] = zadd(zscale(ap, sn), zscale(aq, cs));
      }
      __syncthreads();
    }
  }
  // sort ascending (selection, one thread), W = L^-dagger V
  __shared__ int ord[BMAX];
  __shared__ double ev[BMAX];
  if (tid == 0) {
    for (int r = 0; r < b; ++r) {
      ev[r] = A[r][r].x;
      ord[r] = r;
    }
    for (int r = 0; r < b; ++r)
      for (int s = r + 1; s < b; ++s)
        if (ev[ord[s]] < ev[ord[r]]) {
          const int t = ord[r];
          ord[r] = ord[s];
          ord[s] = t;
        }
  }
  __syncthreads();
  for (int c = tid; c < b; c += nt) {
    const int oc = ord[c];
    theta[(size_t)k * b + c] = ev[oc];
    // back substitution L^dagger w = v
    for (int r = b - 1; r >= 0; --r) {
      zd s = V[r][oc];
      for (int t = r + 1; t < b; ++t) s = zsub(s, zmul(zconj(G[t][r]), Wg[(size_t)k * b * b + t + (size_t)c * b]));
      Wg[(size_t)k * b * b + r + (size_t)c * b] = zscale(s, 1.0 / G[r][r].x);
    }
  }
  if (tid == 0 && fail) stat[k] = BS_ENOTPD;
}

// ------------------------------------------------------------ certificate
// Guaranteed lower bounds for the lowest eigenvalues from the Rayleigh-Ritz
// data, by Lehmann's method.  The Ritz vectors y_i = X w_i (i < m) are
// orthonormal with Ritz values theta_i and residuals r_i = C y_i - theta_i y_i
// (orthogonal to every y_j); let E = R^dagger R.  For any rho with
// theta_i < rho <= lambda_{m+1}(C), the Rayleigh-Ritz method applied to
// (C - rho)^-1 on the trial space (C - rho) span(Y) gives the Ritz values
// -1/nu_i, with nu_1 <= ... <= nu_m the eigenvalues of
//     K = D + D^-1/2 E D^-1/2,   D = diag(rho - theta_i),
// and, (C - rho)^-1 having exactly m eigenvalues 1/(lambda_j - rho) < 0,
// min-max turns them into  lambda_{m+1-i} >= rho - nu_i.  Only the distance
// of each Ritz value to rho enters: a cluster of close Ritz values inside
// the block needs no gap of its own.  Upper bounds are the Ritz values
// themselves (lambda_i <= theta_i), so theta_j - (rho - nu_{m+1-j}) bounds
// the error of theta_j.
//
// rho comes from an eigenvalue count: the Sturm count of the FP32
// tridiagonal T of the mixed path (rho from lambda_{m+1}(T)) or the FP32
// LDL^dagger count of the LOBPCG path (rho = its shift sigma, m = the
// expected count, which that check verifies).  Both counts are exact for an
// FP32 perturbation of C(k); the margin 2^-20 max_r C_rr subtracted from rho
// covers that perturbation (FP32 rounding of C and of the reduction).

constexpr int RCH = 8;   // rows of C X and X staged per step of the residual Gram

// Hermitian eigenvalues of the m x m matrix K (shared, row stride BMAX + 1)
// by cyclic Jacobi with the round-robin pairing of small_eig_kernel; m even
// (callers pad with a decoupled zero); eigenvalues left on the diagonal.
__device__ void jacobi_eigenvalues(zd (*K)[BMAX + 1], int m, double* red) {
  __shared__ double cs_[BMAX / 2], sn_[BMAX / 2];
  __shared__ zd ph_[BMAX / 2];
  __shared__ int pp_[BMAX / 2], qq_[BMAX / 2];
  __shared__ double offn, totn;
  const int tid = threadIdx.x, nt = blockDim.x, np = m / 2;
  for (int sweep = 0; sweep < 30; ++sweep) {
    double o = 0.0, t = 0.0;
    for (int e = tid; e < m * m; e += nt) {
      const int r = e % m, c = e / m;
      const double m2 = K[r][c].x * K[r][c].x + K[r][c].y * K[r][c].y;
      t += m2;
      if (r != c) o += m2;
    }
    for (int sh = 16; sh > 0; sh >>= 1) {
      o += __shfl_xor_sync(0xffffffffu, o, sh);
      t += __shfl_xor_sync(0xffffffffu, t, sh);
    }
    if ((tid & 31) == 0) {
      red[2 * (tid >> 5)] = o;
      red[2 * (tid >> 5) + 1] = t;
    }
    __syncthreads();
    if (tid == 0) {
      double so = 0.0, st = 0.0;
      for (int w = 0; w < nt / 32; ++w) {
        so += red[2 * w];
        st += red[2 * w + 1];
      }
      offn = so;
      totn = st;
    }
    __syncthreads();
    if (offn <= 1e-26 * totn) break;
    for (int rd = 0; rd < m - 1; ++rd) {
      if (tid < np) {
        int p, q;
        if (tid == 0) {
          p = rd % (m - 1);
          q = m - 1;
        } else {
          p = (rd + tid) % (m - 1);
          q = (rd - tid + (m - 1)) % (m - 1);
        }
        if (p > q) {
          const int tq = p;
          p = q;
          q = tq;
        }
        const zd c = K[p][q];
        const double ca = hypot(c.x, c.y);
        double cs = 1.0, sn = 0.0;
        zd ph = zmake(1.0, 0.0);
        if (ca > 0.0) {
          ph = zmake(c.x / ca, c.y / ca);
          const double zeta = (K[q][q].x - K[p][p].x) / (2.0 * ca);
          const double tt = zeta >= 0.0 ? 1.0 / (zeta + sqrt(1.0 + zeta * zeta))
                                        : -1.0 / (-zeta + sqrt(1.0 + zeta * zeta));
          cs = 1.0 / sqrt(1.0 + tt * tt);
          sn = tt * cs;
        }
        pp_[tid] = p;
        qq_[tid] = q;
        cs_[tid] = cs;
        sn_[tid] = sn;
        ph_[tid] = ph;
      }
      __syncthreads();
      for (int e = tid; e < np * m; e += nt) {
        const int u = e / m, r = e % m, p = pp_[u], q = qq_[u];
        const double cs = cs_[u], sn = sn_[u];
        const zd ap = K[r][p], aq = zmul(K[r][q], zconj(ph_[u]));
        K[r][p] = zsub(zscale(ap, cs), zscale(aq, sn));
        K[r][q] = zadd(zscale(ap, sn), zscale(aq, cs));
      }
      __syncthreads();
      for (int e = tid; e < np * m; e += nt) {
        const int u = e / m, c = e % m, p = pp_[u], q = qq_[u];
        const double cs = cs_[u], sn = sn_[u];
        const zd ap = K[p][c], aq = zmul(K[q][c], ph_[u]);
        K[p][c] = zsub(zscale(ap, cs), zscale(aq, sn));
        K[q][c] = zadd(zscale(ap, sn), zscale(aq, cs));
      }
      __syncthreads();
    }
  }
}

// Lehmann lower bounds of the wanted eigenvalues for one cut (m Ritz
// vectors, bound rho on lambda_{m+1}); lower[j] = max(lower[j], bound).
__device__ void lehmann_cut(const double* th, zd (*E)[BMAX + 1], zd (*K)[BMAX + 1], int m,
                            double rho, int nbands, double* lower, double* red, double* nu) {
  const int tid = threadIdx.x;
  const int me = m + (m & 1);   // even size for the round-robin sweeps
  for (int e = tid; e < me * me; e += blockDim.x) {
    const int r = e % me, c = e / me;
    zd v = zmake(0.0, 0.0);
    if (r < m && c < m) {
      const double dr = rho - th[r], dc = rho - th[c];
      v = zscale(E[r][c], 1.0 / sqrt(dr * dc));
      if (r == c) v = zmake(v.x + dr, 0.0);
    }
    K[r][c] = v;
  }
  __syncthreads();
  jacobi_eigenvalues(K, me, red);
  if (tid == 0) {
    // ascending eigenvalues of K; the padding zero (if any) is the smallest
    for (int i = 0; i < me; ++i) nu[i] = K[i][i].x;
    for (int i = 1; i < me; ++i) {
      const double v = nu[i];
      int j = i - 1;
      while (j >= 0 && nu[j] > v) {
        nu[j + 1] = nu[j];
        --j;
      }
      nu[j + 1] = v;
    }
    const int off = me - m;
    // lambda_{j+1} >= rho - nu_(m - j)  (0-based j, ascending nu of the m real ones)
    for (int j = 0; j < nbands && j < m; ++j) {
      const double lb = rho - nu[off + m - 1 - j];
      if (lb == lb) lower[j] = fmax(lower[j], lb);
    }
  }
  __syncthreads();
}

// One CTA (256 threads) per problem: the residual Gram E = R^dagger R of the
// Ritz vectors (R = C X W - X W Theta, from the FP64 C X), then the Lehmann
// bounds for up to two cuts and the status: certified when every wanted
// theta_j is within 2 tol max(theta_j, floor2) of its lower bound.
__global__ void __launch_bounds__(256) certify_kernel(
    const zd* __restrict__ C64, const zd* __restrict__ CX, const zd* __restrict__ X,
    const zd* __restrict__ W, const double* __restrict__ theta, const double* __restrict__ lamT,
    int lstride, int n, int b, int nbands, double tol, double floor2, double* __restrict__ omega,
    int* __restrict__ stat, double* __restrict__ errb, float* __restrict__ csig,
    int* __restrict__ cexp) {
  __shared__ zd Ws[BMAX][BMAX + 1];        // W, later K
  __shared__ zd Es[BMAX][BMAX + 1];        // E
  __shared__ zd CXs[RCH][BMAX + 1], Xs[RCH][BMAX + 1];
  __shared__ double th[BMAX], lower[BMAX], nu[BMAX + 1], red[16];
  __shared__ double cmax_s;
  const int k = blockIdx.x, tid = threadIdx.x;
  const zd* cx = CX + (size_t)k * n * b;
  const zd* x = X + (size_t)k * n * b;
  const zd* wk = W + (size_t)k * b * b;
  for (int e = tid; e < b * b; e += blockDim.x) Ws[e % b][e / b] = wk[e];
  if (tid < b) {
    th[tid] = theta[(size_t)k * b + tid];
    lower[tid] = -1e300;
  }
  // max_r C_rr: the scale of the FP32 perturbation margin
  double cm = 0.0;
  for (int r = tid; r < n; r += blockDim.x)
    cm = fmax(cm, C64[(size_t)k * n * n + (size_t)r * n + r].x);
  for (int o = 16; o > 0; o >>= 1) cm = fmax(cm, __shfl_xor_sync(0xffffffffu, cm, o));
  if ((tid & 31) == 0) red[tid >> 5] = cm;
  __syncthreads();
  if (tid == 0) {
    double v = 0.0;
    for (int w = 0; w < 8; ++w) v = fmax(v, red[w]);
    cmax_s = v;
  }
  // residual Gram: thread t owns entries p = t, t + 256, ... of the b x b E
  zd acc[(BMAX * BMAX + 255) / 256];
#pragma unroll
  for (int q = 0; q < (BMAX * BMAX + 255) / 256; ++q) acc[q] = zmake(0.0, 0.0);
  const int rr = tid / 32, ci = tid % 32;   // staging: row rr, column ci of the chunk
  for (int r0 = 0; r0 < n; r0 += RCH) {
    __syncthreads();
    if (ci < b) {
      const int r = r0 + rr;
      CXs[rr][ci] = r < n ? cx[(size_t)ci * n + r] : zmake(0.0, 0.0);
      Xs[rr][ci] = r < n ? x[(size_t)ci * n + r] : zmake(0.0, 0.0);
    }
    __syncthreads();
    // R[rr][ci] = sum_l (CX[rr][l] - theta_ci X[rr][l]) W[l][ci]
    zd rv = zmake(0.0, 0.0);
    if (ci < b) {
      const double t = th[ci];
      for (int l = 0; l < b; ++l)
        rv = zfma(zsub(CXs[rr][l], zscale(Xs[rr][l], t)), Ws[l][ci], rv);
    }
    __syncthreads();
    if (ci < b) CXs[rr][ci] = rv;   // the chunk of R replaces the chunk of C X
    __syncthreads();
#pragma unroll
    for (int q = 0; q < (BMAX * BMAX + 255) / 256; ++q) {
      const int p = tid + 256 * q;
      if (p < b * b) {
        const int i = p % b, j = p / b;
        zd a = acc[q];
        for (int u = 0; u < RCH; ++u) a = zfma(zconj(CXs[u][i]), CXs[u][j], a);
        acc[q] = a;
      }
    }
  }
  __syncthreads();
  // the FP64 product C X carries an error of order 2^-46 |C| |X| per term:
  // allow for it in the residual norms (a negligible widening)
  const double ecx = 0x1p-36 * cmax_s;
#pragma unroll
  for (int q = 0; q < (BMAX * BMAX + 255) / 256; ++q) {
    const int p = tid + 256 * q;
    if (p < b * b) {
      const int i = p % b, j = p / b;
      zd v = acc[q];
      if (i == j) v = zmake(v.x + ecx * ecx * n, 0.0);
      Es[i][j] = v;
    }
  }
  __syncthreads();
  const double margin = 0x1p-20 * cmax_s;
  if (lamT) {
    // cuts where T's spectrum has a gap above the m-th Ritz value, rho just
    // below lambda_{m+1}(T): the highest and the lowest such m in
    // [nbands, b] (degenerate eigenvalues rule out the cuts inside a multiplet)
    const double* lt = lamT + (size_t)k * lstride;
    int mhi = 0, mlo = 0;
    for (int m = b; m >= nbands; --m)
      if (lt[m] - margin > th[m - 1]) {
        if (!mhi) mhi = m;
        mlo = m;
      }
    if (mhi) lehmann_cut(th, Es, Ws, mhi, lt[mhi] - margin, nbands, lower, red, nu);
    if (mlo && mlo != mhi) lehmann_cut(th, Es, Ws, mlo, lt[mlo] - margin, nbands, lower, red, nu);
  } else if (csig) {
    // The count certificate checks one shift sigma per problem; choose it
    // here: the cuts i = b - 2 .. nbands - 1 with a usable gap (bs_shift_at),
    // top-down, each with its own Lehmann bounds (Ritz vectors above a cut
    // do not enter, so poorly converged guard vectors can be left out); the
    // first cut that certifies every wanted band, else the one with the
    // smallest worst ratio of error bound to tolerance.
    __shared__ double lowc[BMAX], ratio_s;
    __shared__ float best_sig;
    __shared__ int best_m;
    double best = 1e300;
    if (tid == 0) {
      best_sig = 0.f;
      best_m = -1;
    }
    for (int i = b - 2; i >= nbands - 1; --i) {
      float sig;
      if (!bs_shift_at(th, i, floor2, &sig)) continue;
      const double rho = (double)sig - margin;
      if (!(rho > th[i])) continue;
      if (tid < BMAX) lowc[tid] = -1e300;
      __syncthreads();
      lehmann_cut(th, Es, Ws, i + 1, rho, nbands, lowc, red, nu);
      if (tid == 0) {
        double r = 0.0;
        for (int j = 0; j < nbands; ++j)
          r = fmax(r, (th[j] - lowc[j]) / (tol * 2.0 * fmax(th[j], floor2)));
        ratio_s = r == r ? r : 1e300;
      }
      __syncthreads();
      const double r = ratio_s;
      if (r < best) {
        best = r;
        if (tid < nbands) lower[tid] = lowc[tid];
        if (tid == 0) {
          best_sig = sig;
          best_m = i + 1;
        }
      }
      __syncthreads();
      if (best <= 1.0) break;
    }
    if (tid == 0 && csig) {
      csig[k] = best_sig;
      cexp[k] = best_m;
    }
  }
  if (tid == 0) {
    int bad = 0;
    for (int j = 0; j < nbands; ++j) {
      const double t = th[j];
      const double err = t - lower[j];
      if (!(err <= tol * 2.0 * fmax(t, floor2)) || !isfinite(t)) bad = 1;
      omega[(size_t)k * nbands + j] = sqrt(fmax(t, 0.0));
      if (errb) errb[(size_t)k * nbands + j] = err;
    }
    if (stat[k] == 0 && bad) stat[k] = BS_ENOCONV;
  }
}

// C32 (lower triangle, FP32) from the full FP64 C, batch of kb
__global__ void c64_to_c32_kernel(const zd* __restrict__ C64, zf* __restrict__ C32, int n, int kb) {
  const size_t nn = (size_t)n * n;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nn * kb) return;
  const size_t l = e % nn;
  if ((int)(l % n) < (int)(l / n)) return;
  C32[e] = make_float2((float)C64[e].x, (float)C64[e].y);
}

__global__ void zero_int_kernel(int* p, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = 0;
}

}  // namespace

// Block size of the refinement: nbands plus up to 8 guard vectors, even
// (round-robin Jacobi), at most BMAX and at most n - 1 (T's eigenvalue
// b + 1 serves as the gap reference).  Callers ensure nbands + 2 <= n.
int bs_mixed_guard(int nbands, int n) {
  int b = (nbands + 8 + 3) / 4 * 4;
  if (b > BMAX) b = BMAX;
  if (b > n - 1) b = n - 1;
  if (b & 1) --b;
  if (b < nbands) b = nbands + (nbands & 1);
  return b;
}

int bs_launch_builder_mixed(const zd* Cm, int n, const double* Q, int nk, double q1x, double q1y,
                            double q2x, double q2y, zd* C64, zf* C32, cudaStream_t s,
                            bool full32) {
  const size_t nn = (size_t)n * n;
  builder_mixed_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(Cm, n, Q, nk, q1x, q1y, q2x,
                                                                    q2y, C64, C32, full32);
  BS_CHECK_LAUNCH("builder_mixed_kernel");
  return BS_OK;
}

int bs_launch_c64_to_c32(const zd* C64, zf* C32, int n, int kb, cudaStream_t s) {
  const size_t tot = (size_t)n * n * kb;
  c64_to_c32_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(C64, C32, n, kb);
  BS_CHECK_LAUNCH("c64_to_c32_kernel");
  return BS_OK;
}

int bs_launch_mixed_refine(const MixedWs& w, int n, int kb, int nbands, int b, double tol,
                           double floor2, double* omega, int* stat, cudaStream_t s) {
  zero_int_kernel<<<(kb + 255) / 256, 256, 0, s>>>(stat, kb);
  BS_CHECK_LAUNCH("zero_int_kernel");
  // the vector block in shared memory when it fits (n <= about 900 at b = 28)
  const size_t ysm = (size_t)b * n * sizeof(double);
  int smax = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    smax = 0;
  }
  // shared memory pays when the problems do not fill the GPU anyway (one
  // large block per SM); with many problems, many small CTAs per SM win
  const bool in_smem = ysm + 1024 <= (size_t)smax && kb <= 2 * bs_sm_count();
  if (in_smem && ysm > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(tri_eigvec_kernel,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)ysm);
    if (e != cudaSuccess) return bs_cuda_status(e, "tri_eigvec smem");
  }
  tri_eigvec_kernel<<<kb, in_smem ? 256 : 64, in_smem ? ysm : 0, s>>>(
      w.de, w.beta, w.lamT, n, b, b + 1, w.scratch, w.Y, w.phase, in_smem);
  BS_CHECK_LAUNCH("tri_eigvec_kernel");
  backtransform_kernel<<<dim3(kb, (b + 7) / 8), 256, 0, s>>>(w.C32, w.tau, w.phase, w.Y, n, b,
                                                              w.X32, w.X64);
  BS_CHECK_LAUNCH("backtransform_kernel");
  return bs_launch_rr_tail(w, n, kb, nbands, b, tol, floor2, omega, stat, s);
}

int bs_launch_rr_tail(const MixedWs& w, int n, int kb, int nbands, int b, double tol,
                      double floor2, double* omega, int* stat, cudaStream_t s) {
  const zd one = zmake(1.0, 0.0);
  const long nb = (long)n * b, bb = (long)b * b;
  // C X with FP64-level accuracy on the tensor cores (exact digit-plane contraction)
  TRY_LAUNCH(bs_launch_cx_tc(w.C64, w.X64, n, b, kb, w.cxA, w.cxB, w.cxD, w.cxeA, w.cxeB, w.CX,
                             w.err, s));
  TRY_LAUNCH(bs_launch_zgemm(true, false, b, b, n, one, w.X64, n, nb, w.X64, n, nb, nullptr, 0,
                             w.G, b, bb, kb, 0, s));
  TRY_LAUNCH(bs_launch_zgemm(true, false, b, b, n, one, w.X64, n, nb, w.CX, n, nb, nullptr, 0,
                             w.H, b, bb, kb, 0, s));
  small_eig_kernel<<<kb, 128, 0, s>>>(w.G, w.H, b, w.theta, w.W, stat);
  BS_CHECK_LAUNCH("small_eig_kernel");
  certify_kernel<<<kb, 256, 0, s>>>(w.C64, w.CX, w.X64, w.W, w.theta, w.lamT, b + 1, n, b,
                                    nbands, tol, floor2, omega, stat, w.errb, w.csig, w.cexp);
  BS_CHECK_LAUNCH("certify_kernel");
  return BS_OK;
}
