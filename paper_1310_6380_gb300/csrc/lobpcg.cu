// Block LOBPCG for the lowest eigenpairs of the reduced matrix C(k) (the
// Hermitian standard form of the Sec. IV eigenproblem), batched over k:
// an iterative alternative to the dense reduction whose cost follows the
// quality of the starting block.
//
// Each k carries an orthonormal basis S = [X | P | W] (FP32):
//   X  the current Ritz block (b columns),
//   P  the previous search directions, orthonormal and orthogonal to X,
//   W  preconditioned residuals of the unconverged columns, orthonormalised
//      against X and P (Cholesky QR, twice, dropping dependent columns).
// One iteration is three launches over all unfinished k:
//   lob_cw_kernel      C W (the O(n^2 b) product) and S^dagger (C W) by row block,
//   lob_eig_kernel     Rayleigh-Ritz on S: the m x m (m <= 3b) Hermitian
//                      eigenproblem by Householder tridiagonalisation, Sturm
//                      bisection and inverse iteration (one warp per k), the
//                      new P directions orthonormalised in the small space,
//   lob_update_kernel  X <- S Z, P <- S Y (and C X, C P likewise), residuals,
//                      convergence, the next W and the [X P] Gram block.
// Because S stays orthonormal the Rayleigh-Ritz problem is a standard one and
// P needs no tall orthogonalisation (the "basis selection" form of LOBPCG).
// Columns whose FP32 residual meets the tolerance are soft-locked (they stay
// in X but get no W or P column).  The FP32 block is finished by the FP64
// Rayleigh-Ritz tail of the mixed path, whose residual bound decides; the
// caller falls back to the dense FP64 solve where it fails.
#include <float.h>
#include <math.h>

#include "bs_internal.h"

namespace {

constexpr int LB = BS_LOB_MAX_BLOCK;   // largest block size b
constexpr int LM = 3 * LB;             // largest Rayleigh-Ritz dimension
constexpr int UT = 256;                // threads of the per-k kernels
constexpr int RC = 64;                 // rows per staging step of the tall Gram products
constexpr int PPT = (LM * LM + UT - 1) / UT;
constexpr int CWT = 128;               // rows of C W per CTA
constexpr int CWJ = 64;                // columns of C per staged chunk of W
constexpr int PPG = (LM * LB + CWT - 1) / CWT;
constexpr int ALD = LM + 1;            // leading dimension of the small matrix

__device__ __forceinline__ zf zf0() { return make_float2(0.f, 0.f); }
// acc + conj(a) b
__device__ __forceinline__ zf zfcma(zf a, zf b, zf acc) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
  return acc;
}
__device__ __forceinline__ float zabs2(zf a) { return a.x * a.x + a.y * a.y; }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// counter-based hash -> uniform in [-1, 1) (deterministic noise for the seeds)
__device__ __forceinline__ float hash_unit(unsigned a, unsigned b) {
  unsigned h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u;
  h ^= h >> 16;
  h *= 0x7FEB352Du;
  h ^= h >> 15;
  h *= 0x846CA68Bu;
  h ^= h >> 16;
  return (float)(h >> 8) * (2.0f / 16777216.0f) - 1.0f;
}

// compact basis index -> column slot (X at 0, P at b, W at 2b)
__device__ __forceinline__ int bcol(int i, int nx, int np, int b) {
  return i < nx ? i : (i < nx + np ? b + (i - nx) : 2 * b + (i - nx - np));
}

__device__ __forceinline__ size_t blk_off(int buf, int k, int kb, int b, int n) {
  return ((size_t)buf * kb + k) * (size_t)(3 * b) * n;
}

// ------------------------------------------------------------ CTA-wide tall-skinny helpers
struct SmU {
  zf* stA;     // RC x LM
  zf* stB;     // RC x LM
  zf* G;       // LM x LM, row-major [i][j]
  zf* Zs;      // LM x LB
  zf* Ys;      // LM x LB
  zf* L;       // LB x LB Cholesky factor, row-major
  float* red;  // (UT/32) x LB
  float* nrm;  // LB
  int* colA;   // LM
  int* colB;   // LM
  int* kept;   // LB
  int* ival;   // 4 scalars
};

__host__ __device__ constexpr size_t smu_bytes() {
  return sizeof(zf) * (2 * RC * LM + LM * LM + 2 * LM * LB + LB * LB) +
         sizeof(float) * ((UT / 32) * LB + LB) + sizeof(int) * (2 * LM + LB + 4);
}

__device__ SmU carve_u(void* base) {
  SmU s;
  zf* z = (zf*)base;
  s.stA = z;
  s.stB = s.stA + RC * LM;
  s.G = s.stB + RC * LM;
  s.Zs = s.G + LM * LM;
  s.Ys = s.Zs + LM * LB;
  s.L = s.Ys + LM * LB;
  float* f = (float*)(s.L + LB * LB);
  s.red = f;
  s.nrm = s.red + (UT / 32) * LB;
  int* ip = (int*)(s.nrm + LB);
  s.colA = ip;
  s.colB = s.colA + LM;
  s.kept = s.colB + LM;
  s.ival = s.kept + LB;
  return s;
}

// G[i][j] = sum_r conj(A[:, colA[i]]) B[:, colB[j]] for i < ca, j < cb (all threads)
__device__ void tall_gram(const zf* A, const int* colA, int ca, const zf* B, const int* colB,
                          int cb, int n, const SmU& sm) {
  const int tid = threadIdx.x;
  const int npair = ca * cb;
  zf acc[PPT];
#pragma unroll
  for (int t = 0; t < PPT; ++t) acc[t] = zf0();
  for (int r0 = 0; r0 < n; r0 += RC) {
    const int rc = min(RC, n - r0);
    __syncthreads();
    for (int e = tid; e < RC * ca; e += UT) {
      const int r = e % RC, i = e / RC;
      sm.stA[r * LM + i] = r < rc ? A[(size_t)colA[i] * n + r0 + r] : zf0();
    }
    for (int e = tid; e < RC * cb; e += UT) {
      const int r = e % RC, j = e / RC;
      sm.stB[r * LM + j] = r < rc ? B[(size_t)colB[j] * n + r0 + r] : zf0();
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < PPT; ++t) {
      const int p = tid + t * UT;
      if (p < npair) {
        const int i = p / cb, j = p % cb;
        zf a = acc[t];
        for (int r = 0; r < rc; ++r) a = zfcma(sm.stA[r * LM + i], sm.stB[r * LM + j], a);
        acc[t] = a;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < PPT; ++t) {
    const int p = tid + t * UT;
    if (p < npair) sm.G[(p / cb) * LM + (p % cb)] = acc[t];
  }
  __syncthreads();
}

// W[:, colB[j]] -= sum_i A[:, colA[i]] G[i][j], j < cb (all threads)
__device__ void tall_sub(zf* W, const int* colB, int cb, const zf* A, const int* colA, int ca,
                         int n, const SmU& sm) {
  for (int r = threadIdx.x; r < n; r += UT) {
    zf acc[LB];
#pragma unroll
    for (int j = 0; j < LB; ++j) acc[j] = j < cb ? W[(size_t)colB[j] * n + r] : zf0();
    for (int i = 0; i < ca; ++i) {
      const zf a = A[(size_t)colA[i] * n + r];
#pragma unroll
      for (int j = 0; j < LB; ++j) acc[j] = zfnmac(a, zconj(sm.G[i * LM + j]), acc[j]);
    }
#pragma unroll
    for (int j = 0; j < LB; ++j)
      if (j < cb) W[(size_t)colB[j] * n + r] = acc[j];
  }
  __syncthreads();
}

// squared column norms of W[:, colB[j]] into sm.nrm (all threads)
__device__ void col_norms(const zf* W, const int* colB, int cb, int n, const SmU& sm) {
  float p[LB];
#pragma unroll
  for (int j = 0; j < LB; ++j) p[j] = 0.f;
  for (int r = threadIdx.x; r < n; r += UT) {
#pragma unroll
    for (int j = 0; j < LB; ++j)
      if (j < cb) p[j] += zabs2(W[(size_t)colB[j] * n + r]);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < LB; ++j) {
    const float v = warp_sum(p[j]);
    if (lane == 0) sm.red[warp * LB + j] = v;
  }
  __syncthreads();
  if (threadIdx.x < LB) {
    float s = 0.f;
    for (int w = 0; w < UT / 32; ++w) s += sm.red[w * LB + threadIdx.x];
    sm.nrm[threadIdx.x] = s;
  }
  __syncthreads();
}

// W[:, colB[j]] /= sqrt(nrm[j]) (zero columns stay zero)
__device__ void col_normalise(zf* W, const int* colB, int cb, int n, const SmU& sm) {
  for (int r = threadIdx.x; r < n; r += UT) {
#pragma unroll
    for (int j = 0; j < LB; ++j)
      if (j < cb) {
        const float s = sm.nrm[j] > 0.f ? rsqrtf(sm.nrm[j]) : 0.f;
        const size_t o = (size_t)colB[j] * n + r;
        W[o] = zscale(W[o], s);
      }
  }
  __syncthreads();
}

// Cholesky with column dropping of the Hermitian cb x cb matrix sm.G (one
// thread): keeps column j when its pivot exceeds thr2 (absolute) or
// thr2 * G[j][j]; sm.L (rows in kept order) and sm.kept, returns the kept
// count through sm.ival[0].
__device__ void chol_drop(int cb, float thr2, bool absolute, const SmU& sm) {
  if (threadIdx.x == 0) {
    int nk = 0;
    for (int j = 0; j < cb; ++j) {
      const float gjj = sm.G[j * LM + j].x;
      zf row[LB];
      float piv = gjj;
      for (int s = 0; s < nk; ++s) {
        // L[nk][s] = (G[j][kept_s] - sum_{u<s} L[nk][u] conj(L[s][u])) / L[s][s]
        zf v = sm.G[j * LM + sm.kept[s]];
        for (int u = 0; u < s; ++u) v = zfnmac(row[u], sm.L[s * LB + u], v);
        v = zscale(v, 1.0f / sm.L[s * LB + s].x);
        row[s] = v;
        piv -= zabs2(v);
      }
      if (gjj > 0.f && piv > thr2 * (absolute ? 1.f : gjj) && isfinite(piv)) {
        for (int s = 0; s < nk; ++s) sm.L[nk * LB + s] = row[s];
        sm.L[nk * LB + nk] = make_float2(sqrtf(piv), 0.f);
        sm.kept[nk++] = j;
      }
    }
    sm.ival[0] = nk;
  }
  __syncthreads();
}

// W[:, colB[t]] <- (W[:, colB[kept[t]]] - sum_{s<t} W'[:, s] conj(L[t][s])) / L[t][t]:
// the kept columns times L^-dagger, compacted to the first nk slots
__device__ void tri_apply(zf* W, const int* colB, int cb, int nk, int n, const SmU& sm) {
  for (int r = threadIdx.x; r < n; r += UT) {
    zf v[LB];
#pragma unroll
    for (int t = 0; t < LB; ++t) v[t] = t < nk ? W[(size_t)colB[sm.kept[t]] * n + r] : zf0();
#pragma unroll
    for (int t = 0; t < LB; ++t) {
      if (t < nk) {
        zf x = v[t];
#pragma unroll
        for (int s = 0; s < t; ++s) x = zfnmac(v[s], sm.L[t * LB + s], x);
        v[t] = zscale(x, 1.0f / sm.L[t * LB + t].x);
      }
    }
#pragma unroll
    for (int t = 0; t < LB; ++t)
      if (t < nk) W[(size_t)colB[t] * n + r] = v[t];
  }
  __syncthreads();
  (void)cb;
}

// Orthonormalise the cb columns colB of S against the ca orthonormal
// columns colA (two projections) and among themselves (Cholesky QR twice,
// dropping columns whose independent part is below sqrt(thr2) of their
// norm).  Survivors are compacted to colB[0..nk); returns nk.
__device__ int orth_block(zf* S, int ca, int cb, int n, float thr2, const SmU& sm) {
  col_norms(S, sm.colB, cb, n, sm);
  col_normalise(S, sm.colB, cb, n, sm);
  if (ca > 0) {
    for (int pass = 0; pass < 2; ++pass) {
      tall_gram(S, sm.colA, ca, S, sm.colB, cb, n, sm);
      tall_sub(S, sm.colB, cb, S, sm.colA, ca, n, sm);
    }
  }
  int nk = cb;
  for (int pass = 0; pass < 2 && nk > 0; ++pass) {
    tall_gram(S, sm.colB, nk, S, sm.colB, nk, n, sm);
    // first pass: the columns were unit before the projections, so the
    // pivot threshold is absolute (relative to that unit norm)
    if (pass == 0 && threadIdx.x == 0)
      for (int j = 0; j < nk; ++j) sm.G[j * LM + j].y = 0.f;
    __syncthreads();
    chol_drop(nk, pass == 0 ? thr2 : 1e-6f, pass == 0, sm);
    const int kept = sm.ival[0];
    tri_apply(S, sm.colB, nk, kept, n, sm);
    nk = kept;
  }
  return nk;
}

// block reduction of one float per thread to thread 0's return value
__device__ float block_sum(float v, float* red) {
  v = warp_sum(v);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  float s = 0.f;
  for (int w = 0; w < UT / 32; ++w) s += red[w];
  __syncthreads();
  return s;
}

// ------------------------------------------------------------ seed
// Starting block in the W slot: the given vectors (reduced basis) first, then
// unit vectors at the smallest diagonal entries of C (cold start), each with
// 1e-3 deterministic noise; orthonormalised with dependent columns replaced
// by preconditioned noise.
__global__ void __launch_bounds__(UT) lob_seed_kernel(LobWs w, int n, int kb, int b) {
  extern __shared__ float4 dyn_u[];
  const SmU sm = carve_u(dyn_u);
  __shared__ float s_val[UT / 32];
  __shared__ int s_idx[UT / 32];
  __shared__ int pick[LB];
  const int k = blockIdx.x, tid = threadIdx.x;
  const zf* C = w.C32 + (size_t)k * n * n;
  zf* S = w.S + blk_off(0, k, kb, b, n);
  // preconditioner shift: 1e-3 of the mean diagonal entry
  float dsum = 0.f;
  for (int r = tid; r < n; r += UT) dsum += C[(size_t)r * n + r].x;
  const float dshift = 1e-3f * block_sum(dsum, sm.red) / n;
  const int nv = w.X0 ? min(w.nvec, b) : 0;
  // cold columns: the b - nv smallest diagonal entries, by repeated block argmin
  for (int t = 0; t < b - nv; ++t) {
    float bv = FLT_MAX;
    int bi = 0x7fffffff;
    for (int r = tid; r < n; r += UT) {
      bool used = false;
      for (int u = 0; u < t; ++u) used |= pick[u] == r;
      const float dv = C[(size_t)r * n + r].x;
      if (!used && (dv < bv || (dv == bv && r < bi))) {
        bv = dv;
        bi = r;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov < bv || (ov == bv && oi < bi)) {
        bv = ov;
        bi = oi;
      }
    }
    if ((tid & 31) == 0) {
      s_val[tid >> 5] = bv;
      s_idx[tid >> 5] = bi;
    }
    __syncthreads();
    if (tid == 0) {
      float v = s_val[0];
      int i = s_idx[0];
      for (int q = 1; q < UT / 32; ++q)
        if (s_val[q] < v || (s_val[q] == v && s_idx[q] < i)) {
          v = s_val[q];
          i = s_idx[q];
        }
      pick[t] = i;
    }
    __syncthreads();
  }
  const zf* x0 = w.X0 ? w.X0 + (size_t)k * w.nvec * n : nullptr;
  for (int r = tid; r < n; r += UT) {
    for (int j = 0; j < b; ++j) {
      zf v;
      if (j < nv) {
        v = x0[(size_t)j * n + r];
      } else {
        v = make_float2(r == pick[j - nv] ? 1.f : 0.f, 0.f);
        v.x += 1e-3f * hash_unit(r, 2 * j);
        v.y += 1e-3f * hash_unit(r, 2 * j + 1);
      }
      S[(size_t)(2 * b + j) * n + r] = v;
    }
  }
  if (tid < LB) sm.colB[tid] = 2 * b + tid;
  __syncthreads();
  int nk = orth_block(S, 0, b, n, 1e-6f, sm);
  // refill dropped columns with preconditioned noise (at most three rounds)
  for (int round = 0; round < 3 && nk < b; ++round) {
    const int need = b - nk;
    for (int r = tid; r < n; r += UT) {
      const float pr = 1.f / (C[(size_t)r * n + r].x + dshift);
      for (int j = 0; j < need; ++j) {
        const unsigned salt = 1000u + 64u * round + j;
        S[(size_t)(2 * b + nk + j) * n + r] =
            make_float2(pr * hash_unit(r, 2 * salt), pr * hash_unit(r, 2 * salt + 1));
      }
    }
    if (tid < LB) {
      sm.colA[tid] = 2 * b + tid;           // the kept columns
      sm.colB[tid] = 2 * b + nk + tid;      // the new ones
    }
    __syncthreads();
    nk += orth_block(S, nk, need, n, 1e-6f, sm);
    __syncthreads();
  }
  if (tid == 0) {
    LobState st;
    st.done = nk < b ? 1 : 0;
    st.it = 0;
    st.nx = 0;
    st.np = 0;
    st.nw = nk;
    st.cur = 0;
    st.npn = 0;
    st.nact = b;
    st.amask = b >= 32 ? 0xffffffffu : ((1u << b) - 1u);
    st.dshift = dshift;
    st.rmax = 0.f;
    st.rbest = FLT_MAX;
    st.itbest = 0;
    st.seedfail = nk < b ? 1 : 0;
    for (int j = 0; j < LB; ++j) st.theta[j] = 0.f;
    w.st[k] = st;
    if (st.done) atomicAdd(w.ndone, 1);
  }
}

// ------------------------------------------------------------ C W
// CW = C W for the nw columns of W (rows of this CTA), then the partial
// Gram S_rows^dagger CW_rows over all m basis columns, summed by lob_eig_kernel.
__global__ void __launch_bounds__(CWT) lob_cw_kernel(LobWs w, int n, int kb, int b) {
  __shared__ __align__(16) zf Wst[CWJ * LB];
  __shared__ __align__(16) zf Sst[32 * LM];
  __shared__ __align__(16) zf CWst[32 * LB];
  __shared__ int colS[LM];
  const int k = blockIdx.y, rb = blockIdx.x, tid = threadIdx.x;
  const LobState* stp = w.st + k;
  if (stp->done) return;
  const int nx = stp->nx, np = stp->np, nw = stp->nw, cur = stp->cur;
  const int m = nx + np + nw;
  const zf* C = w.C32 + (size_t)k * n * n;
  const zf* S = w.S + blk_off(cur, k, kb, b, n);
  zf* CS = w.CS + blk_off(cur, k, kb, b, n);
  const zf* Wb = S + (size_t)2 * b * n;
  const int r = rb * CWT + tid;
  zf acc[LB];
#pragma unroll
  for (int c = 0; c < LB; ++c) acc[c] = zf0();
  for (int j0 = 0; j0 < n; j0 += CWJ) {
    const int jc = min(CWJ, n - j0);
    __syncthreads();
    for (int e = tid; e < CWJ * LB; e += CWT) {
      const int c = e & (LB - 1), jj = e / LB;
      Wst[jj * LB + c] = (jj < jc && c < nw) ? Wb[(size_t)c * n + j0 + jj] : zf0();
    }
    __syncthreads();
    if (r < n) {
      const zf* cp = C + (size_t)j0 * n + r;
#pragma unroll 4
      for (int jj = 0; jj < jc; ++jj) {
        const zf cv = cp[(size_t)jj * n];
        const float4* wr = reinterpret_cast<const float4*>(Wst + jj * LB);
#pragma unroll
        for (int c2 = 0; c2 < LB / 2; ++c2) {
          const float4 w4 = wr[c2];
          acc[2 * c2] = zfma(cv, make_float2(w4.x, w4.y), acc[2 * c2]);
          acc[2 * c2 + 1] = zfma(cv, make_float2(w4.z, w4.w), acc[2 * c2 + 1]);
        }
      }
    }
  }
  if (r < n) {
#pragma unroll
    for (int c = 0; c < LB; ++c)
      if (c < nw) CS[(size_t)(2 * b + c) * n + r] = acc[c];
  }
  for (int i = tid; i < m; i += CWT) colS[i] = bcol(i, nx, np, b);
  zf g[PPG];
#pragma unroll
  for (int t = 0; t < PPG; ++t) g[t] = zf0();
  const int npair = m * nw;
  for (int sub = 0; sub < CWT / 32; ++sub) {
    const int rr0 = rb * CWT + sub * 32;
    if (rr0 >= n) break;
    __syncthreads();
    if (tid >= sub * 32 && tid < sub * 32 + 32) {
#pragma unroll
      for (int c = 0; c < LB; ++c) CWst[(tid - sub * 32) * LB + c] = r < n ? acc[c] : zf0();
    }
    for (int e = tid; e < 32 * m; e += CWT) {
      const int rr = e % 32, i = e / 32;
      Sst[rr * LM + i] = rr0 + rr < n ? S[(size_t)colS[i] * n + rr0 + rr] : zf0();
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < PPG; ++t) {
      const int p = tid + t * CWT;
      if (p < npair) {
        const int i = p / nw, c = p % nw;
        zf a = g[t];
        for (int rr = 0; rr < 32; ++rr) a = zfcma(Sst[rr * LM + i], CWst[rr * LB + c], a);
        g[t] = a;
      }
    }
  }
  const int nrb = (n + CWT - 1) / CWT;
  zf* part = w.part + ((size_t)k * nrb + rb) * LB * LM;
#pragma unroll
  for (int t = 0; t < PPG; ++t) {
    const int p = tid + t * CWT;
    if (p < npair) part[(size_t)(p % nw) * LM + p / nw] = g[t];
  }
}

// ------------------------------------------------------------ small Rayleigh-Ritz problem
struct SmE {
  zf* A;       // LM x ALD, row-major
  zf* Zs;      // LM x LB eigenvectors (complex)
  float* U;    // LM x LB tridiagonal eigenvectors, [i][c]
  float* lu;   // 5 x LM x LB factors of T - theta I, [arr][i][c]
  float* d;    // LM
  float* e;    // LM
  float* e2;   // LM
  zf* tau;     // LM
  zf* wv;      // LM
  float* th;   // LB
  int* act;    // LB
  int* iv;     // 4 scalars
  zf* Ys;      // LM x LB (aliases lu)
  zf* Gs;      // LB x LB (aliases lu after Ys)
  zf* L;       // LB x LB (aliases lu after Gs)
  int* kept;   // LB
};

__host__ __device__ constexpr size_t sme_bytes() {
  return sizeof(zf) * (LM * ALD + LM * LB + 2 * LM) +
         sizeof(float) * (LM * LB + 5 * LM * LB + 3 * LM + LB) + sizeof(int) * (2 * LB + 4);
}

__device__ SmE carve_e(void* base) {
  SmE s;
  zf* z = (zf*)base;
  s.A = z;
  s.Zs = s.A + LM * ALD;
  s.tau = s.Zs + LM * LB;
  s.wv = s.tau + LM;
  float* f = (float*)(s.wv + LM);
  s.U = f;
  s.lu = s.U + LM * LB;
  s.d = s.lu + 5 * LM * LB;
  s.e = s.d + LM;
  s.e2 = s.e + LM;
  s.th = s.e2 + LM;
  int* ip = (int*)(s.th + LB);
  s.act = ip;
  s.kept = s.act + LB;
  s.iv = s.kept + LB;
  // aliases inside lu (5 * LM * LB floats = 2.5 * LM * LB complex)
  s.Ys = (zf*)s.lu;
  s.Gs = s.Ys + LM * LB;
  s.L = s.Gs + LB * LB;
  return s;
}

__device__ __forceinline__ float lu_get(const SmE& s, int arr, int i, int c) {
  return s.lu[(arr * LM + i) * LB + c];
}
__device__ __forceinline__ void lu_set(const SmE& s, int arr, int i, int c, float v) {
  s.lu[(arr * LM + i) * LB + c] = v;
}

__global__ void __launch_bounds__(32) lob_eig_kernel(LobWs w, int n, int kb, int b) {
  extern __shared__ float4 dyn_e[];
  const SmE s = carve_e(dyn_e);
  const int k = blockIdx.x, lane = threadIdx.x;
  LobState* stp = w.st + k;
  if (stp->done) return;
  const int nx = stp->nx, np = stp->np, nw = stp->nw;
  const int mp = nx + np, m = mp + nw;
  const unsigned amask = stp->amask;
  const int q = b;   // wanted Ritz pairs (m >= b)
  const int nrb = (n + CWT - 1) / CWT;
  const zf* axp = w.Axp + (size_t)k * LM * LM;
  const zf* pt = w.part + (size_t)k * nrb * LB * LM;
  // assemble A = S^dagger C S
  for (int e = lane; e < m * m; e += 32) {
    const int i = e % m, j = e / m;
    zf v = zf0();
    if (i < mp && j < mp) {
      v = axp[(size_t)j * LM + i];
    } else if (j >= mp) {
      for (int rb = 0; rb < nrb; ++rb) v = zadd(v, pt[((size_t)rb * LB + (j - mp)) * LM + i]);
    } else {
      for (int rb = 0; rb < nrb; ++rb) v = zadd(v, pt[((size_t)rb * LB + (i - mp)) * LM + j]);
      v = zconj(v);
    }
    s.A[i * ALD + j] = v;
  }
  __syncwarp();
  for (int e = lane; e < m * m; e += 32) {
    const int i = e % m, j = e / m;
    if (i < j) {
      const zf h = zscale(zadd(s.A[i * ALD + j], zconj(s.A[j * ALD + i])), 0.5f);
      s.A[i * ALD + j] = h;
      s.A[j * ALD + i] = zconj(h);
    } else if (i == j) {
      s.A[i * ALD + i].y = 0.f;
    }
  }
  __syncwarp();
  // Householder tridiagonalisation (lower): T = Q^dagger A Q, Q = H_0 ... H_{m-2},
  // H_j = I - tau_j v_j v_j^dagger with v_j[j+1] = 1 and v_j below in A[.][j]
  const zf one = make_float2(1.f, 0.f);
  for (int j = 0; j < m - 1; ++j) {
    const int r0 = j + 1;
    float xn2 = 0.f;
    for (int r = r0 + 1 + lane; r < m; r += 32) xn2 += zabs2(s.A[r * ALD + j]);
    xn2 = __shfl_sync(0xffffffffu, warp_sum(xn2), 0);
    const zf alpha = s.A[r0 * ALD + j];
    zf tau = zf0();
    float beta = alpha.x;
    if (xn2 > 0.f || alpha.y != 0.f) {
      const float anorm = sqrtf(zabs2(alpha) + xn2);
      beta = alpha.x >= 0.f ? -anorm : anorm;
      tau = make_float2((beta - alpha.x) / beta, -alpha.y / beta);
      const zf den = make_float2(alpha.x - beta, alpha.y);
      const float dd = zabs2(den);
      const zf sc = make_float2(den.x / dd, -den.y / dd);
      for (int r = r0 + 1 + lane; r < m; r += 32) s.A[r * ALD + j] = zmul(s.A[r * ALD + j], sc);
    }
    __syncwarp();
    if (lane == 0) {
      s.e[j] = beta;
      s.tau[j] = tau;
    }
    if (tau.x != 0.f || tau.y != 0.f) {
      for (int r = r0 + lane; r < m; r += 32) {
        zf acc = s.A[r * ALD + r0];
        for (int c = r0 + 1; c < m; ++c) acc = zfma(s.A[r * ALD + c], s.A[c * ALD + j], acc);
        s.wv[r] = zmul(tau, acc);
      }
      __syncwarp();
      float dx = 0.f, dy = 0.f;
      for (int r = r0 + lane; r < m; r += 32) {
        const zf vr = r == r0 ? one : s.A[r * ALD + j];
        const zf yr = s.wv[r];
        dx += vr.x * yr.x + vr.y * yr.y;
        dy += vr.x * yr.y - vr.y * yr.x;
      }
      dx = __shfl_sync(0xffffffffu, warp_sum(dx), 0);
      dy = __shfl_sync(0xffffffffu, warp_sum(dy), 0);
      const float hk = 0.5f * (tau.x * dx + tau.y * dy);   // Re(conj(tau) v^H y) / 2
      for (int r = r0 + lane; r < m; r += 32) {
        const zf vr = r == r0 ? one : s.A[r * ALD + j];
        s.wv[r] = zsub(s.wv[r], zscale(vr, hk));
      }
      __syncwarp();
      for (int r = r0 + lane; r < m; r += 32) {
        const zf vr = r == r0 ? one : s.A[r * ALD + j];
        const zf wr = s.wv[r];
        for (int c = r0; c < m; ++c) {
          const zf vc = c == r0 ? one : s.A[c * ALD + j];
          const zf wc = s.wv[c];
          zf a = s.A[r * ALD + c];
          a = zfnmac(vr, wc, a);
          a = zfnmac(wr, vc, a);
          s.A[r * ALD + c] = a;
        }
      }
    }
    __syncwarp();
    if (lane == 0) s.d[j] = s.A[j * ALD + j].x;
    __syncwarp();
  }
  if (lane == 0) {
    s.d[m - 1] = s.A[(m - 1) * ALD + (m - 1)].x;
    s.e[m - 1] = 0.f;
  }
  __syncwarp();
  for (int i = lane; i < m; i += 32) s.e2[i] = s.e[i] * s.e[i];
  __syncwarp();
  // Gershgorin interval and scales
  float gl = FLT_MAX, gu = -FLT_MAX, emax2 = 0.f;
  for (int i = 0; i < m; ++i) {
    const float rad = fabsf(s.e[i]) + (i > 0 ? fabsf(s.e[i - 1]) : 0.f);
    gl = fminf(gl, s.d[i] - rad);
    gu = fmaxf(gu, s.d[i] + rad);
    emax2 = fmaxf(emax2, s.e2[i]);
  }
  const float tnorm = fmaxf(fabsf(gl), fabsf(gu));
  const float pivmin = FLT_MIN * fmaxf(1.f, emax2);
  const float tinyp = FLT_EPSILON * fmaxf(tnorm, FLT_MIN);
  // Sturm multisection: lanes c and c + 16 find eigenvalue c (ascending),
  // each step the pair counts at the two interior third points.  The wanted
  // eigenvalues lie in [0, theta_top] of the previous block (the basis
  // contains that block, so the Ritz values can only decrease, and A is
  // positive semidefinite); that bracket is used when one count confirms it.
  {
    auto sturm = [&](float x) {
      int cnt = 0;
      float qv = s.d[0] - x;
      if (fabsf(qv) < pivmin) qv = -pivmin;
      cnt += qv < 0.f;
      for (int i = 1; i < m; ++i) {
        qv = s.d[i] - x - __fdividef(s.e2[i - 1], qv);
        if (fabsf(qv) < pivmin) qv = -pivmin;
        cnt += qv < 0.f;
      }
      return cnt;
    };
    const int c = lane & (LB - 1), h = lane / LB;
    float lo = gl - FLT_EPSILON * tnorm, hi = gu + FLT_EPSILON * tnorm;
    if (nx > 0) {
      const float top = stp->theta[q - 1];
      const float hb = top + 1e-3f * fabsf(top) + 16.f * FLT_EPSILON * tnorm;
      if (hb < hi && sturm(hb) >= q) {
        hi = hb;
        lo = fmaxf(lo, -16.f * FLT_EPSILON * tnorm);
      }
      // The basis contains the previous Ritz block, so Ritz value c can only
      // have decreased, and between iterations it moves little: try the
      // bracket [theta_c - 1e-3 |theta_c|, theta_c] (slightly widened), kept
      // when the pair's two counts confirm it (about a third of the
      // trisection steps of the full bracket)
      const float t = stp->theta[c];
      const float slack = 16.f * FLT_EPSILON * tnorm;
      const float l1 = fmaxf(lo, t - 1e-3f * fabsf(t) - slack);
      const float h1 = fminf(hi, t + 1e-6f * fabsf(t) + slack);
      const int mine = sturm(h ? h1 : l1);
      const int other = __shfl_xor_sync((1u << c) | (1u << (c + LB)), mine, LB);
      const int clo = h ? other : mine, chi = h ? mine : other;
      if (l1 < h1 && clo <= c && chi > c) {
        lo = l1;
        hi = h1;
      }
    }
    for (int it = 0; it < 48; ++it) {
      // 1e-6 relative: the FP64 Rayleigh-Ritz stage recomputes the values
      if (hi - lo <= 1e-6f * fmaxf(fabsf(lo), fabsf(hi)) + pivmin) break;
      const float x1 = lo + (hi - lo) * (1.f / 3.f), x2 = lo + (hi - lo) * (2.f / 3.f);
      const int mine = sturm(h ? x2 : x1);
      // the two lanes of a pair run the same number of steps (identical
      // brackets), so the pair alone synchronises here
      const int other = __shfl_xor_sync((1u << c) | (1u << (c + LB)), mine, LB);
      const int c1 = h ? other : mine, c2 = h ? mine : other;
      if (c1 > c) hi = x1;
      else if (c2 > c) {
        lo = x1;
        hi = x2;
      } else {
        lo = x2;
      }
    }
    if (h == 0 && c < q) s.th[c] = 0.5f * (lo + hi);
  }
  __syncwarp();
  // inverse iteration on T - theta I (tridiagonal LU with partial pivoting);
  // lane c owns vector c, vectors are orthogonalised in ascending order
  if (lane < q) {
    const float lam = s.th[lane];
    float cd = s.d[0] - lam, cs = m > 1 ? s.e[0] : 0.f;
    for (int i = 0; i < m - 1; ++i) {
      const float sub = s.e[i], nd = s.d[i + 1] - lam, ns = i + 1 < m - 1 ? s.e[i + 1] : 0.f;
      if (fabsf(cd) >= fabsf(sub)) {
        const float piv = fabsf(cd) < tinyp ? (cd < 0.f ? -tinyp : tinyp) : cd;
        const float l = sub / piv;
        lu_set(s, 0, i, lane, piv);
        lu_set(s, 1, i, lane, cs);
        lu_set(s, 2, i, lane, 0.f);
        lu_set(s, 3, i, lane, l);
        lu_set(s, 4, i, lane, 0.f);
        cd = nd - l * cs;
        cs = ns;
      } else {
        const float l = cd / sub;
        lu_set(s, 0, i, lane, sub);
        lu_set(s, 1, i, lane, nd);
        lu_set(s, 2, i, lane, ns);
        lu_set(s, 3, i, lane, l);
        lu_set(s, 4, i, lane, 1.f);
        cd = cs - l * nd;
        cs = -l * ns;
      }
    }
    lu_set(s, 0, m - 1, lane, fabsf(cd) < tinyp ? (cd < 0.f ? -tinyp : tinyp) : cd);
    for (int i = 0; i < m; ++i) s.U[i * LB + lane] = hash_unit(i, 7919u + lane);
  }
  for (int pass = 0; pass < 2; ++pass) {
    if (lane < q) {
      float* u = s.U + lane;
      for (int i = 0; i < m - 1; ++i) {
        const float l = lu_get(s, 3, i, lane);
        if (lu_get(s, 4, i, lane) != 0.f) {
          const float t = u[i * LB];
          u[i * LB] = u[(i + 1) * LB];
          u[(i + 1) * LB] = t - l * u[i * LB];
        } else {
          u[(i + 1) * LB] -= l * u[i * LB];
        }
      }
      u[(m - 1) * LB] /= lu_get(s, 0, m - 1, lane);
      if (m >= 2)
        u[(m - 2) * LB] =
            (u[(m - 2) * LB] - lu_get(s, 1, m - 2, lane) * u[(m - 1) * LB]) / lu_get(s, 0, m - 2, lane);
      for (int i = m - 3; i >= 0; --i)
        u[i * LB] = (u[i * LB] - lu_get(s, 1, i, lane) * u[(i + 1) * LB] -
                     lu_get(s, 2, i, lane) * u[(i + 2) * LB]) /
                    lu_get(s, 0, i, lane);
      float nn = 0.f;
      for (int i = 0; i < m; ++i) nn += u[i * LB] * u[i * LB];
      if (!(nn > 0.f) || !isfinite(nn)) {
        for (int i = 0; i < m; ++i) u[i * LB] = i == lane ? 1.f : 0.f;
        nn = 1.f;
      }
      const float sc = rsqrtf(nn);
      for (int i = 0; i < m; ++i) u[i * LB] *= sc;
    }
    __syncwarp();
    // modified Gram-Schmidt in ascending order
    for (int j = 0; j < q - 1; ++j) {
      if (lane > j && lane < q) {
        float dt = 0.f;
        for (int i = 0; i < m; ++i) dt += s.U[i * LB + j] * s.U[i * LB + lane];
        for (int i = 0; i < m; ++i) s.U[i * LB + lane] -= dt * s.U[i * LB + j];
      }
      __syncwarp();
      if (lane == j + 1) {
        float nn = 0.f;
        for (int i = 0; i < m; ++i) nn += s.U[i * LB + lane] * s.U[i * LB + lane];
        const float sc = nn > 0.f ? rsqrtf(nn) : 0.f;
        for (int i = 0; i < m; ++i) s.U[i * LB + lane] *= sc;
      }
      __syncwarp();
    }
  }
  // back-transform z = Q u: H_{m-2} first, H_0 last; lanes (c, half) share a column
  for (int e = lane; e < m * LB; e += 32) {
    const int i = e / LB, c = e % LB;
    s.Zs[i * LB + c] = make_float2(c < q ? s.U[i * LB + c] : 0.f, 0.f);
  }
  __syncwarp();
  {
    const int c = lane & (LB - 1), h = lane / LB;
    for (int j = m - 2; j >= 0; --j) {
      const zf tj = s.tau[j];
      if (tj.x == 0.f && tj.y == 0.f) continue;
      zf sdot = zf0();
      for (int r = j + 1 + h; r < m; r += 2) {
        const zf vr = r == j + 1 ? one : s.A[r * ALD + j];
        sdot = zfcma(vr, s.Zs[r * LB + c], sdot);
      }
      sdot.x += __shfl_xor_sync(0xffffffffu, sdot.x, LB);
      sdot.y += __shfl_xor_sync(0xffffffffu, sdot.y, LB);
      const zf f = zmul(tj, sdot);
      for (int r = j + 1 + h; r < m; r += 2) {
        const zf vr = r == j + 1 ? one : s.A[r * ALD + j];
        s.Zs[r * LB + c] = zsub(s.Zs[r * LB + c], zmul(vr, f));
      }
      __syncwarp();
    }
  }
  __syncwarp();
  zf* Zg = w.Z + (size_t)k * LB * LM;
  for (int e = lane; e < q * m; e += 32) {
    const int c = e / m, i = e % m;
    Zg[(size_t)c * LM + i] = s.Zs[i * LB + c];
  }
  if (lane < q) stp->theta[lane] = s.th[lane];
  // P directions: the W and P parts of the active Ritz vectors, orthonormalised
  // against Z and among themselves in the small space
  if (lane == 0) {
    int na = 0;
    for (int c = 0; c < q; ++c)
      if (amask & (1u << c)) s.act[na++] = c;
    s.iv[0] = na;
  }
  __syncwarp();
  const int na = nx > 0 ? s.iv[0] : 0;
  __syncwarp();
  for (int e = lane; e < m * LB; e += 32) {
    const int i = e / LB, t = e % LB;
    s.Ys[i * LB + t] = (t < na && i >= nx) ? s.Zs[i * LB + s.act[t]] : zf0();
  }
  __syncwarp();
  // unit columns
  if (lane < na) {
    float nn = 0.f;
    for (int i = 0; i < m; ++i) nn += zabs2(s.Ys[i * LB + lane]);
    const float sc = nn > 0.f ? rsqrtf(nn) : 0.f;
    for (int i = 0; i < m; ++i) s.Ys[i * LB + lane] = zscale(s.Ys[i * LB + lane], sc);
  }
  __syncwarp();
  for (int pass = 0; pass < 2; ++pass) {
    // Gs = Z^dagger Ys (q x na), Ys -= Z Gs
    for (int e = lane; e < q * na; e += 32) {
      const int c = e / na, t = e % na;
      zf a = zf0();
      for (int i = 0; i < m; ++i) a = zfcma(s.Zs[i * LB + c], s.Ys[i * LB + t], a);
      s.Gs[c * LB + t] = a;
    }
    __syncwarp();
    for (int e = lane; e < m * na; e += 32) {
      const int i = e / na, t = e % na;
      zf a = s.Ys[i * LB + t];
      for (int c = 0; c < q; ++c) a = zsub(a, zmul(s.Zs[i * LB + c], s.Gs[c * LB + t]));
      s.Ys[i * LB + t] = a;
    }
    __syncwarp();
  }
  int npn = 0;
  for (int pass = 0; pass < 2 && na > 0; ++pass) {
    const int cnt = pass == 0 ? na : npn;
    if (cnt == 0) break;
    // Gram of the columns and Cholesky with dropping (lane 0)
    for (int e = lane; e < cnt * cnt; e += 32) {
      const int t = e / cnt, u = e % cnt;
      zf a = zf0();
      for (int i = 0; i < m; ++i) a = zfcma(s.Ys[i * LB + t], s.Ys[i * LB + u], a);
      s.Gs[t * LB + u] = a;
    }
    __syncwarp();
    if (lane == 0) {
      int nk = 0;
      const float thr2 = 1e-6f;
      for (int j = 0; j < cnt; ++j) {
        const float gjj = s.Gs[j * LB + j].x;
        zf row[LB];
        float piv = gjj;
        for (int t = 0; t < nk; ++t) {
          zf v = s.Gs[j * LB + s.kept[t]];
          for (int u = 0; u < t; ++u) v = zfnmac(row[u], s.L[t * LB + u], v);
          v = zscale(v, 1.0f / s.L[t * LB + t].x);
          row[t] = v;
          piv -= zabs2(v);
        }
        // relative to the unit norm the column had before the projections
        if (piv > thr2 * (pass == 0 ? 1.f : gjj) && isfinite(piv)) {
          for (int t = 0; t < nk; ++t) s.L[nk * LB + t] = row[t];
          s.L[nk * LB + nk] = make_float2(sqrtf(piv), 0.f);
          s.kept[nk++] = j;
        }
      }
      s.iv[1] = nk;
    }
    __syncwarp();
    const int nk = s.iv[1];
    __syncwarp();
    // Ys' = Ys[:, kept] L^-dagger, row by row (lanes over rows)
    for (int i = lane; i < m; i += 32) {
      zf v[LB];
#pragma unroll
      for (int t = 0; t < LB; ++t) v[t] = t < nk ? s.Ys[i * LB + s.kept[t]] : zf0();
#pragma unroll
      for (int t = 0; t < LB; ++t) {
        if (t < nk) {
          zf x = v[t];
#pragma unroll
          for (int u = 0; u < t; ++u) x = zfnmac(v[u], s.L[t * LB + u], x);
          v[t] = zscale(x, 1.0f / s.L[t * LB + t].x);
        }
      }
#pragma unroll
      for (int t = 0; t < LB; ++t) s.Ys[i * LB + t] = t < nk ? v[t] : zf0();
    }
    __syncwarp();
    npn = nk;
  }
  zf* Yg = w.Y + (size_t)k * LB * LM;
  for (int e = lane; e < npn * m; e += 32) {
    const int t = e / m, i = e % m;
    Yg[(size_t)t * LM + i] = s.Ys[i * LB + t];
  }
  if (lane == 0) stp->npn = npn;
}

// ------------------------------------------------------------ update, residuals, next W
__global__ void __launch_bounds__(UT, 2) lob_update_kernel(LobWs w, int n, int kb, int b, int nb,
                                                        int maxit, float tol, float tolb,
                                                        float floor2) {
  extern __shared__ float4 dyn_u[];
  const SmU sm = carve_u(dyn_u);
  __shared__ LobState st;
  __shared__ float rn2[LB];
  __shared__ int act[LB];
  __shared__ int flag;
  const int k = blockIdx.x, tid = threadIdx.x;
  if (tid == 0) st = w.st[k];
  __syncthreads();
  if (st.done) return;
  const int cur = st.cur, nxt = 1 - cur;
  const zf* S0 = w.S + blk_off(cur, k, kb, b, n);
  const zf* CS0 = w.CS + blk_off(cur, k, kb, b, n);
  zf* S = w.S + blk_off(nxt, k, kb, b, n);
  zf* CS = w.CS + blk_off(nxt, k, kb, b, n);
  const int m = st.nx + st.np + st.nw, npn = st.npn;
  const zf* Zg = w.Z + (size_t)k * LB * LM;
  const zf* Yg = w.Y + (size_t)k * LB * LM;
  for (int e = tid; e < m * LB; e += UT) {
    const int c = e / m, i = e % m;
    sm.Zs[i * LB + c] = c < b ? Zg[(size_t)c * LM + i] : zf0();
    sm.Ys[i * LB + c] = c < npn ? Yg[(size_t)c * LM + i] : zf0();
  }
  for (int i = tid; i < m; i += UT) sm.colA[i] = bcol(i, st.nx, st.np, b);
  __syncthreads();
  // X' = S Z, P' = S Y (then the same with C S) into the other buffer
  for (int pass = 0; pass < 2; ++pass) {
    const zf* src = pass ? CS0 : S0;
    zf* dst = pass ? CS : S;
    for (int r = tid; r < n; r += UT) {
      zf ax[LB], ap[LB];
#pragma unroll
      for (int c = 0; c < LB; ++c) {
        ax[c] = zf0();
        ap[c] = zf0();
      }
      // the next basis entry is loaded while this one is used (the loop is
      // otherwise one L2 round trip per step)
      zf vn = m > 0 ? src[(size_t)sm.colA[0] * n + r] : zf0();
      for (int i = 0; i < m; ++i) {
        const zf v = vn;
        if (i + 1 < m) vn = src[(size_t)sm.colA[i + 1] * n + r];
        const float4* zr = reinterpret_cast<const float4*>(sm.Zs + i * LB);
        const float4* yr = reinterpret_cast<const float4*>(sm.Ys + i * LB);
#pragma unroll
        for (int c2 = 0; c2 < LB / 2; ++c2) {
          const float4 z4 = zr[c2], y4 = yr[c2];
          ax[2 * c2] = zfma(v, make_float2(z4.x, z4.y), ax[2 * c2]);
          ax[2 * c2 + 1] = zfma(v, make_float2(z4.z, z4.w), ax[2 * c2 + 1]);
          ap[2 * c2] = zfma(v, make_float2(y4.x, y4.y), ap[2 * c2]);
          ap[2 * c2 + 1] = zfma(v, make_float2(y4.z, y4.w), ap[2 * c2 + 1]);
        }
      }
#pragma unroll
      for (int c = 0; c < LB; ++c) {
        if (c < b) dst[(size_t)c * n + r] = ax[c];
        if (c < npn) dst[(size_t)(b + c) * n + r] = ap[c];
      }
    }
  }
  __syncthreads();
  const int np = npn;
  // residuals R_c = C x_c - theta_c x_c into the W slot; squared norms
  {
    float p[LB];
#pragma unroll
    for (int c = 0; c < LB; ++c) p[c] = 0.f;
    for (int r = tid; r < n; r += UT) {
#pragma unroll
      for (int c = 0; c < LB; ++c) {
        if (c < b) {
          const zf x = S[(size_t)c * n + r], cx = CS[(size_t)c * n + r];
          const zf rr = zsub(cx, zscale(x, st.theta[c]));
          S[(size_t)(2 * b + c) * n + r] = rr;
          p[c] += zabs2(rr);
        }
      }
    }
    const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
    for (int c = 0; c < LB; ++c) {
      const float v = warp_sum(p[c]);
      if (lane == 0) sm.red[warp * LB + c] = v;
    }
    __syncthreads();
    if (tid < LB) {
      float sum = 0.f;
      for (int q = 0; q < UT / 32; ++q) sum += sm.red[q * LB + tid];
      rn2[tid] = sum;
    }
    __syncthreads();
  }
  if (tid == 0) {
    bool wanted = true;
    int na = 0;
    unsigned mask = 0u;
    float rmax = 0.f;
    // the FP64 certificate bounds the error of theta_c by about
    // ||r_c||^2 / (rho - theta_c), rho a shift in a gap near the block's top
    // (at most theta_{b-2} + 1%), against 2 tolb max(theta_c, floor2): wanted
    // columns meet that with theta_{b-2} for rho and a factor 8 to spare
    const float top = st.theta[b - 2];
    for (int c = 0; c < b; ++c) {
      const float scale = fmaxf(fabsf(st.theta[c]), floor2);
      const float ratio = sqrtf(rn2[c]) / scale;
      const bool ok = ratio <= tol &&
                      (c >= nb || rn2[c] <= 0.25f * tolb * scale * fmaxf(top - st.theta[c], 0.f));
      if (c < nb) {
        wanted = wanted && ok;
        rmax = fmaxf(rmax, ratio);
      }
      if (!ok) {
        act[na++] = c;
        mask |= 1u << c;
      }
    }
    st.cur = nxt;
    st.nx = b;
    st.np = np;
    st.it += 1;
    st.rmax = rmax;
    st.nact = na;
    st.amask = mask;
    // stagnation (the FP32 rounding floor): no 10 % gain in 12 iterations
    if (rmax < 0.9f * st.rbest) {
      st.rbest = rmax;
      st.itbest = st.it;
    }
    const bool stuck = st.it - st.itbest >= 12;
    const bool stop = wanted || st.it >= maxit || na == 0 || stuck;
    flag = stop ? 1 : 0;
    if (stop) st.done = 1;
  }
  __syncthreads();
  if (flag) {
    if (tid == 0) {
      w.st[k] = st;
      atomicAdd(w.ndone, 1);
    }
    return;
  }
  const int na = st.nact;
  // W_j = R_{act_j} / (diag(C) + shift), compacted
  const zf* C = w.C32 + (size_t)k * n * n;
  for (int r = tid; r < n; r += UT) {
    const float pr = 1.f / (C[(size_t)r * n + r].x + st.dshift);
    zf v[LB];
#pragma unroll
    for (int j = 0; j < LB; ++j) v[j] = j < na ? S[(size_t)(2 * b + act[j]) * n + r] : zf0();
#pragma unroll
    for (int j = 0; j < LB; ++j)
      if (j < na) S[(size_t)(2 * b + j) * n + r] = zscale(v[j], pr);
  }
  // against [X P], then among themselves
  for (int i = tid; i < b + np; i += UT) sm.colA[i] = i;   // X at 0..b-1, P at b..b+np-1
  if (tid < LB) sm.colB[tid] = 2 * b + tid;
  __syncthreads();
  const int nw = orth_block(S, b + np, na, n, 1e-6f, sm);
  // Gram of [X P]: [X P]^dagger [CX CP]
  for (int i = tid; i < b + np; i += UT) sm.colA[i] = i;
  __syncthreads();
  tall_gram(S, sm.colA, b + np, CS, sm.colA, b + np, n, sm);
  zf* axp = w.Axp + (size_t)k * LM * LM;
  for (int e = tid; e < (b + np) * (b + np); e += UT) {
    const int i = e % (b + np), j = e / (b + np);
    axp[(size_t)j * LM + i] = sm.G[i * LM + j];
  }
  if (tid == 0) {
    st.nw = nw;
    if (nw == 0) {
      st.done = 1;
      atomicAdd(w.ndone, 1);
    }
    w.st[k] = st;
  }
}

// X (FP32, current buffer) -> FP64 n x b block for the Rayleigh-Ritz tail
__global__ void lob_export_kernel(LobWs w, int n, int kb, int b, zd* X64, int* iters) {
  const int k = blockIdx.y;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const LobState* stp = w.st + k;
  const int cur = stp->cur;
  if (e < (size_t)n * b) {
    const zf v = w.S[blk_off(cur, k, kb, b, n) + e];
    X64[(size_t)k * n * b + e] = zmake((double)v.x, (double)v.y);
  }
  if (e == 0 && iters) iters[k] = stp->seedfail ? -1 : stp->it;
}

// y = (I_2 (x) L_R^dagger) u for starting vectors given in plane-wave
// displacement coefficients: u [k][v][n] (complex64) -> y [k][v][n].  With
// Mp >= 0 the input holds only the waves |alpha|, |beta| <= Mp
// (2 (2Mp+1)^2 coefficients per vector, same ordering rules); the others are 0.
__global__ void lob_to_reduced_kernel(const float2* u, const zd* LR, int N, int M, int Mp,
                                      float2* y) {
  extern __shared__ double2 ush[];
  const int kv = blockIdx.x, n = 2 * N;
  if (Mp < 0) {
    const float2* uk = u + (size_t)kv * n;
    for (int r = threadIdx.x; r < n; r += blockDim.x) ush[r] = zmake(uk[r].x, uk[r].y);
  } else {
    const int wl = 2 * Mp + 1, Nl = wl * wl;
    const float2* uk = u + (size_t)kv * 2 * Nl;
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
      const int I = r / N, a = r % N;
      const int al = a / (2 * M + 1) - M, be = a % (2 * M + 1) - M;
      zd v = zmake(0.0, 0.0);
      if (al >= -Mp && al <= Mp && be >= -Mp && be <= Mp) {
        const float2 f = uk[I * Nl + (al + Mp) * wl + (be + Mp)];
        v = zmake(f.x, f.y);
      }
      ush[r] = v;
    }
  }
  __syncthreads();
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const int I = r / N, i = r % N;
    zd acc = zmake(0.0, 0.0);
    const zd* col = LR + (size_t)i * N;   // column i of L_R, rows t >= i
    for (int t = i; t < N; ++t) acc = zfmac(ush[I * N + t], col[t], acc);
    y[(size_t)kv * n + r] = make_float2((float)acc.x, (float)acc.y);
  }
}

// Ritz vectors of the tail mapped back to displacement coefficients:
// u = (I_2 (x) L_R^-dagger) X w_j for j < nbands.  Problem k uses
// L_R^-1 at LinvR + (k / kper) * lstride (one factor per cell).  Output row
// rows[k] (or k) of [row][j][len]: all n coefficients (Mp < 0) or only the
// waves |alpha|, |beta| <= Mp (len = 2 (2Mp+1)^2).
__global__ void lob_vectors_kernel(const zd* X64, const zd* Wc, const zd* LinvR, long lstride,
                                   int kper, int N, int M, int Mp, int b, int nbands,
                                   const int* rows, float2* out) {
  extern __shared__ double2 ysh[];
  const int k = blockIdx.y, j = blockIdx.x, n = 2 * N;
  const zd* x = X64 + (size_t)k * n * b;
  const zd* wj = Wc + (size_t)k * b * b + (size_t)j * b;
  const zd* Li = LinvR + (size_t)(k / kper) * lstride;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    zd acc = zmake(0.0, 0.0);
    for (int l = 0; l < b; ++l) acc = zfma(x[r + (size_t)l * n], wj[l], acc);
    ysh[r] = acc;
  }
  __syncthreads();
  const int wl = 2 * Mp + 1;
  const int len = Mp < 0 ? n : 2 * wl * wl;
  const size_t row = rows ? (size_t)rows[k] : (size_t)k;
  for (int o = threadIdx.x; o < len; o += blockDim.x) {
    int r = o;
    if (Mp >= 0) {
      const int I = o / (wl * wl), a = o % (wl * wl);
      const int al = a / wl - Mp, be = a % wl - Mp;
      r = I * N + (al + M) * (2 * M + 1) + (be + M);
    }
    const int I = r / N, i = r % N;
    zd acc = zmake(0.0, 0.0);
    const zd* col = Li + (size_t)i * N;   // column i of L_R^-1, rows t >= i
    for (int t = i; t < N; ++t) acc = zfmac(ysh[I * N + t], col[t], acc);
    out[(row * nbands + j) * len + o] = make_float2((float)acc.x, (float)acc.y);
  }
}

}  // namespace

size_t bs_lob_part_elems(int n) { return (size_t)((n + CWT - 1) / CWT) * LB * LM; }
size_t bs_lob_small_elems() { return (size_t)LM * LM; }

// 16 columns (nbands plus at least four guard vectors) where n allows: the
// guards keep the top Ritz value, the gap reference of the residual bound,
// well above the wanted ones.  Even and no larger than the block the FP64
// Rayleigh-Ritz workspace of the mixed path holds (its Jacobi sweeps pair
// the columns).
int bs_lob_block(int nbands, int n) {
  int b = LB;
  (void)nbands;
  const int g = bs_mixed_guard(nbands, n);
  if (b > g) b = g;
  if (b & 1) --b;
  return b;
}

int bs_launch_lobpcg(const LobWs& w, int n, int kb, int b, int nb, int maxit, float tol,
                     float tolb, float floor2, int check_every, cudaStream_t s) {
  const size_t su = smu_bytes(), se = sme_bytes();
  cudaFuncSetAttribute(lob_seed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)su);
  cudaFuncSetAttribute(lob_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)su);
  cudaFuncSetAttribute(lob_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)se);
  if (b < 2 || b > LB || nb > b || n < b + 1) {
    bs_set_error("LOBPCG: block size %d outside [2, %d] or n = %d too small", b, LB, n);
    return BS_EINVAL;
  }
  cudaError_t ce = cudaMemsetAsync(w.ndone, 0, sizeof(int), s);
  if (ce != cudaSuccess) return bs_cuda_status(ce, "LOBPCG counter");
  lob_seed_kernel<<<kb, UT, su, s>>>(w, n, kb, b);
  BS_CHECK_LAUNCH("lob_seed_kernel");
  const int nrb = (n + CWT - 1) / CWT;
  // maxit + 1 updates: the last one only evaluates the residuals of the
  // final block and marks every k finished
  for (int it = 0; it < maxit + 1; ++it) {
    lob_cw_kernel<<<dim3(nrb, kb), CWT, 0, s>>>(w, n, kb, b);
    BS_CHECK_LAUNCH("lob_cw_kernel");
    lob_eig_kernel<<<kb, 32, se, s>>>(w, n, kb, b);
    BS_CHECK_LAUNCH("lob_eig_kernel");
    lob_update_kernel<<<kb, UT, su, s>>>(w, n, kb, b, nb, maxit, tol, tolb, floor2);
    BS_CHECK_LAUNCH("lob_update_kernel");
    if (check_every > 0 && (it + 1) % check_every == 0) {
      int hdone = 0;
      ce = cudaMemcpyAsync(&hdone, w.ndone, sizeof(int), cudaMemcpyDeviceToHost, s);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
      if (ce != cudaSuccess) return bs_cuda_status(ce, "LOBPCG progress");
      if (hdone >= kb) break;
    }
  }
  return BS_OK;
}

int bs_launch_lob_export(const LobWs& w, int n, int kb, int b, zd* X64, int* iters, cudaStream_t s) {
  const size_t tot = (size_t)n * b;
  lob_export_kernel<<<dim3((unsigned)((tot + 255) / 256), kb), 256, 0, s>>>(w, n, kb, b, X64, iters);
  BS_CHECK_LAUNCH("lob_export_kernel");
  return BS_OK;
}

int bs_launch_lob_to_reduced(const float2* u, const zd* LR, int N, int M, int Mp, int kb, int nvec,
                             float2* y, cudaStream_t s) {
  if (Mp > M) {
    bs_set_error("starting vectors with Mp = %d > M = %d", Mp, M);
    return BS_EINVAL;
  }
  const size_t sh = (size_t)2 * N * sizeof(double2);
  if (sh > 48 * 1024)
    cudaFuncSetAttribute(lob_to_reduced_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  lob_to_reduced_kernel<<<kb * nvec, 256, sh, s>>>(u, LR, N, M, Mp, y);
  BS_CHECK_LAUNCH("lob_to_reduced_kernel");
  return BS_OK;
}

int bs_launch_lob_vectors(const zd* X64, const zd* Wc, const zd* LinvR, long lstride, int kper,
                          int N, int M, int Mp, int b, int nbands, int kb, const int* rows,
                          float2* out, cudaStream_t s) {
  const size_t sh = (size_t)2 * N * sizeof(double2);
  if (sh > 48 * 1024)
    cudaFuncSetAttribute(lob_vectors_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  lob_vectors_kernel<<<dim3(nbands, kb), 256, sh, s>>>(X64, Wc, LinvR, lstride, kper, N, M, Mp, b,
                                                       nbands, rows, out);
  BS_CHECK_LAUNCH("lob_vectors_kernel");
  return BS_OK;
}
