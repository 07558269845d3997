// Batched FP64 Householder reduction of Hermitian matrices to real
// symmetric tridiagonal form (the first stage of the eigensolve of
// Eq. (eigenvalueproblem) once the pencil is reduced to standard form).
//
// Step j (j = 0 .. n-2) with reflector H_j = I - tau v v^dagger (tau real,
// v[j+1] = 1) needs p = tau B v on the trailing block B = A[j+1:, j+1:],
// w = p - (tau/2)(v^dagger p) v and the rank-2 update B -= v w^dagger + w v^dagger.
// One launch per step does, for every matrix of the batch, the rank-2
// update of step j-1 fused with p of step j over 64 x 64 tiles of the
// lower triangle (each element is read and written once per step), and
// the last tile of each matrix to finish (an arrival counter, no waiting)
// reduces the tile partials, forms w, applies the update to column j+1
// and builds the next reflector.  The arithmetic is FP64 and FMA bound on
// GB300, so the tile loop is written for FP64 issue, not for bandwidth.
#include "bs_internal.h"

namespace {

constexpr int TS = 64;    // tile edge
constexpr int NT = 256;   // threads per CTA (8 warps)

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double t = lane < NT / 32 ? sh[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) sh[NT / 32] = t;
  }
  __syncthreads();
  return sh[NT / 32];
}

__device__ __forceinline__ zd ldg_cg(const zd* p) { return __ldcg(p); }

// Reflector of column c below the diagonal: x = A[c+1:n, c].  Writes v
// (v[c+1] = 1), tau and the tridiagonal off-diagonal |beta| = ||x||.
__device__ void householder(const zd* a, int n, int c, zd* v, double* tau_out, double* e_out,
                            double* sh) {
  const int tid = threadIdx.x, r0 = c + 1;
  double s = 0.0;
  for (int r = r0 + 1 + tid; r < n; r += NT) {
    zd x = ldg_cg(a + r + (size_t)c * n);
    s = fma(x.x, x.x, fma(x.y, x.y, s));
  }
  s = block_sum(s, sh);
  const zd alpha = ldg_cg(a + r0 + (size_t)c * n);
  const double aa = hypot(alpha.x, alpha.y);
  const double nu = sqrt(fma(aa, aa, s));
  double tau = 0.0;
  zd scale = zmake(0.0, 0.0);
  if (nu > 0.0) {
    const zd beta = aa > 0.0 ? zscale(alpha, -nu / aa) : zmake(-nu, 0.0);
    tau = (aa + nu) / nu;
    const zd den = zsub(alpha, beta);
    const double d2 = den.x * den.x + den.y * den.y;
    scale = zmake(den.x / d2, -den.y / d2);
  }
  for (int r = r0 + 1 + tid; r < n; r += NT) v[r] = zmul(ldg_cg(a + r + (size_t)c * n), scale);
  if (tid == 0) {
    v[r0] = zmake(1.0, 0.0);
    *tau_out = tau;
    *e_out = nu;
  }
}

__global__ void __launch_bounds__(NT) tridiag_init_kernel(const zd* __restrict__ A, int n,
                                                          zd* __restrict__ vec,
                                                          double* __restrict__ de,
                                                          double* __restrict__ tau,
                                                          unsigned* __restrict__ count) {
  __shared__ double sh[NT / 32 + 1];
  const int b = blockIdx.x;
  const zd* a = A + (size_t)b * n * n;
  zd* vb = vec + (size_t)b * 3 * n;
  for (int r = threadIdx.x; r < 3 * n; r += NT) vb[r] = zmake(0.0, 0.0);
  __syncthreads();
  double* d = de + (size_t)b * 2 * n;
  if (threadIdx.x == 0) {
    d[0] = a[0].x;
    count[b] = 0u;
    tau[b] = 0.0;
  }
  if (n > 1) householder(a, n, 0, vb, tau + b, d + n, sh);
}

__device__ __forceinline__ void tri_index(int l, int& bi, int& bk) {
  int r = (int)((sqrt(8.0 * l + 1.0) - 1.0) * 0.5);
  while ((r + 1) * (r + 2) / 2 <= l) ++r;
  while (r * (r + 1) / 2 > l) --r;
  bi = r;
  bk = l - r * (r + 1) / 2;
}

__global__ void __launch_bounds__(NT, 2) tridiag_step_kernel(zd* __restrict__ A, int n, int j,
                                                             zd* __restrict__ vec,
                                                             zd* __restrict__ part,
                                                             double* __restrict__ de,
                                                             double* __restrict__ tau,
                                                             unsigned* __restrict__ count,
                                                             int ntl) {
  // Thread (tx, ty) owns rows R*TS + tx + 16v and columns S*TS + ty + 16u,
  // u, v = 0..3: its 16 elements give 4 row and 4 column partials of p,
  // reduced once per tile through shared memory.
  __shared__ zd vpS[TS], wpS[TS], vcS[TS];
  __shared__ zd rowred[TS / 4][TS];   // [ty][row]
  __shared__ zd colred[TS / 4][TS];   // [tx][col]
  __shared__ double sh[NT / 32 + 1];
  __shared__ int is_last;

  const int b = blockIdx.y, tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int nt = (n + TS - 1) / TS, t0 = (j + 1) / TS, r0 = j + 1;
  zd* a = A + (size_t)b * n * n;
  zd* vb = vec + (size_t)b * 3 * n;
  zd* vcur = vb + (size_t)(j & 1) * n;
  zd* vprev = vb + (size_t)((j + 1) & 1) * n;
  zd* w = vb + 2 * (size_t)n;
  zd* pt = part + (size_t)b * nt * n;

  int bi, bk;
  tri_index(blockIdx.x, bi, bk);
  const int R = t0 + bi, S = t0 + bk;
  const int rbase = R * TS, sbase = S * TS;

  if (tid < TS) {
    const int s = sbase + tid;
    const bool ok = s < n && s >= r0;
    vpS[tid] = ok ? vprev[s] : zmake(0.0, 0.0);
    wpS[tid] = ok ? w[s] : zmake(0.0, 0.0);
    vcS[tid] = ok ? vcur[s] : zmake(0.0, 0.0);
  }
  zd vpr[4], wpr[4], vcr[4], racc[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const int r = rbase + tx + 16 * v;
    const bool ok = r < n && r >= r0;
    vpr[v] = ok ? vprev[r] : zmake(0.0, 0.0);
    wpr[v] = ok ? w[r] : zmake(0.0, 0.0);
    vcr[v] = ok ? vcur[r] : zmake(0.0, 0.0);
    racc[v] = zmake(0.0, 0.0);
  }
  __syncthreads();

#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int sl = ty + 16 * u, s = sbase + sl;
    const zd vps = vpS[sl], wps = wpS[sl], vcs = vcS[sl];
    zd cacc = zmake(0.0, 0.0);
    const bool sok = s >= r0;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int r = rbase + tx + 16 * v;
      if (sok && r < n && r >= s) {
        zd* ap = a + r + (size_t)s * n;
        zd x = *ap;
        x = zfnmac(vpr[v], wps, x);
        x = zfnmac(wpr[v], vps, x);
        if (r == s) x.y = 0.0;
        *ap = x;
        racc[v] = zfma(x, vcs, racc[v]);
        if (r != s) cacc = zfma(zconj(x), vcr[v], cacc);
      }
    }
    colred[tx][sl] = cacc;
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) rowred[ty][tx + 16 * v] = racc[v];
  __syncthreads();
  if (tid < 2 * TS) {
    const bool isrow = tid < TS;
    const int l = isrow ? tid : tid - TS;
    zd acc = zmake(0.0, 0.0);
#pragma unroll
    for (int q = 0; q < TS / 4; ++q) acc = zadd(acc, isrow ? rowred[q][l] : colred[q][l]);
    if (R == S) {
      // diagonal tile: row and column partials of the same index meet here
      if (isrow) rowred[0][l] = acc;
      else colred[0][l] = acc;
    } else if (isrow) {
      if (rbase + l < n) pt[(size_t)S * n + rbase + l] = acc;
    } else {
      pt[(size_t)R * n + sbase + l] = acc;
    }
  }
  if (R == S) {
    __syncthreads();
    if (tid < TS && rbase + tid < n) pt[(size_t)R * n + rbase + tid] = zadd(rowred[0][tid], colred[0][tid]);
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) is_last = (atomicAdd(count + b, 1u) == (unsigned)(ntl - 1));
  __syncthreads();
  if (!is_last) return;
  __threadfence();

  // ---- epilogue: one CTA per matrix
  const double tj = tau[b];
  double kp = 0.0;
  for (int rr = r0 + tid; rr < n; rr += NT) {
    zd p = zmake(0.0, 0.0);
    for (int t = t0; t < nt; ++t) p = zadd(p, ldg_cg(pt + (size_t)t * n + rr));
    p = zscale(p, tj);
    w[rr] = p;
    const zd v = vcur[rr];
    kp = fma(v.x, p.x, fma(v.y, p.y, kp));
  }
  const double K = 0.5 * tj * block_sum(kp, sh);
  for (int rr = r0 + tid; rr < n; rr += NT) {
    const zd v = vcur[rr];
    w[rr] = zsub(w[rr], zscale(v, K));
  }
  __syncthreads();
  const zd wj = w[r0], vj = vcur[r0];
  for (int rr = r0 + tid; rr < n; rr += NT) {
    zd* ap = a + rr + (size_t)r0 * n;
    zd x = ldg_cg(ap);
    x = zfnmac(vcur[rr], wj, x);
    x = zfnmac(w[rr], vj, x);
    if (rr == r0) x.y = 0.0;
    *ap = x;
  }
  __syncthreads();
  double* d = de + (size_t)b * 2 * n;
  if (tid == 0) {
    d[r0] = a[r0 + (size_t)r0 * n].x;
    count[b] = 0u;
  }
  if (r0 + 1 < n) householder(a, n, r0, vprev, tau + b, d + n + r0, sh);
}

}  // namespace

size_t bs_tridiag_vec_elems(int n) { return 3 * (size_t)n; }
size_t bs_tridiag_part_elems(int n) { return (size_t)((n + TS - 1) / TS) * n; }

int bs_launch_tridiag(zd* A, int n, int batch, zd* vec, zd* part, double* de, double* tau,
                      unsigned* count, cudaStream_t s) {
  tridiag_init_kernel<<<batch, NT, 0, s>>>(A, n, vec, de, tau, count);
  BS_CHECK_LAUNCH("tridiag_init_kernel");
  const int nt = (n + TS - 1) / TS;
  for (int j = 0; j + 1 < n; ++j) {
    const int m = nt - (j + 1) / TS;
    const int ntl = m * (m + 1) / 2;
    tridiag_step_kernel<<<dim3(ntl, batch), NT, 0, s>>>(A, n, j, vec, part, de, tau, count, ntl);
    BS_CHECK_LAUNCH("tridiag_step_kernel");
  }
  return BS_OK;
}
