// Batched Householder reduction of Hermitian matrices to tridiagonal form
// (the first stage of the eigensolve of Eq. (eigenvalueproblem) once the
// pencil is reduced to standard form), in FP64 (the plain path) or FP32
// (the reduction of the mixed path, refined afterwards in FP64).
//
// Step j (j = 0 .. n-2) with reflector H_j = I - tau v v^dagger (tau real,
// v[j+1] = 1) needs p = tau B v on the trailing block B = A[j+1:, j+1:],
// w = p - (tau/2)(v^dagger p) v and the rank-2 update B -= v w^dagger + w v^dagger.
// One launch per step does, for every matrix of the batch, the rank-2
// update of step j-1 fused with p of step j over 64 x 64 tiles of the
// lower triangle (each element is read and written once per step), and
// the last tile of each matrix to finish (an arrival counter, no waiting)
// reduces the tile partials, forms w, applies the update to column j+1
// and builds the next reflector.  In FP64 the loop is bound by the FP64
// pipe of GB300, so it is written for FP64 issue: 16 FMAs per element and
// one shared-memory reduction of the row and column partials per tile.
#include <algorithm>

#include "bs_internal.h"

namespace {

constexpr int TSMAX = 64;  // largest tile edge (the default)
constexpr int TSMIN = 32;  // smallest tile edge (sizes the partial-sum buffer)
constexpr int NT = 256;    // threads per CTA (8 warps), a 16 x 16 thread grid

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

template <typename C>
__device__ __forceinline__ C ldg_cg(const C* p) { return __ldcg(p); }

// Reflector of column c below the diagonal, x = A[c+1:n, c]: H x = beta e1
// with beta = -(x0/|x0|) ||x||, tau = (|x0| + ||x||)/||x||, v = x / (x0 - beta).
// The scalars are formed in FP64 for both precisions.  Writes v to the
// vector buffer and to A[c+2:n, c], tau_j, beta_j and |beta_j|.
template <typename R>
__device__ void householder(typename Cplx<R>::T* a, int n, int c, typename Cplx<R>::T* v,
                            double* tau_out, zd* beta_out, double* e_out, double* sh) {
  typedef typename Cplx<R>::T C;
  const int tid = threadIdx.x, r0 = c + 1;
  double s = 0.0;
  for (int r = r0 + 1 + tid; r < n; r += NT) {
    const C x = ldg_cg(a + r + (size_t)c * n);
    s = fma((double)x.x, (double)x.x, fma((double)x.y, (double)x.y, s));
  }
  s = block_sum(s, sh);
  const C al = ldg_cg(a + r0 + (size_t)c * n);
  const zd alpha = zmake(al.x, al.y);
  const double aa = hypot(alpha.x, alpha.y);
  const double nu = sqrt(fma(aa, aa, s));
  double tau = 0.0;
  zd scale = zmake(0.0, 0.0), beta = zmake(0.0, 0.0);
  if (nu > 0.0) {
    beta = aa > 0.0 ? zscale(alpha, -nu / aa) : zmake(-nu, 0.0);
    tau = (aa + nu) / nu;
    const zd den = zsub(alpha, beta);
    const double d2 = den.x * den.x + den.y * den.y;
    scale = zmake(den.x / d2, -den.y / d2);
  }
  for (int r = r0 + 1 + tid; r < n; r += NT) {
    C* ap = a + r + (size_t)c * n;
    const C x = ldg_cg(ap);
    const zd y = zmul(zmake(x.x, x.y), scale);
    const C vr = Cplx<R>::make((R)y.x, (R)y.y);
    v[r] = vr;
    *ap = vr;
  }
  if (tid == 0) {
    v[r0] = Cplx<R>::make((R)1, (R)0);
    *tau_out = tau;
    *beta_out = beta;
    *e_out = nu;
  }
}

template <typename R>
__global__ void __launch_bounds__(NT) tridiag_init_kernel(typename Cplx<R>::T* __restrict__ A,
                                                          int n,
                                                          typename Cplx<R>::T* __restrict__ vec,
                                                          double* __restrict__ de,
                                                          double* __restrict__ tau,
                                                          zd* __restrict__ beta,
                                                          unsigned* __restrict__ count) {
  typedef typename Cplx<R>::T C;
  __shared__ double sh[NT / 32 + 1];
  const int b = blockIdx.x;
  C* a = A + (size_t)b * n * n;
  C* vb = vec + (size_t)b * 3 * n;
  for (int r = threadIdx.x; r < 3 * n; r += NT) vb[r] = Cplx<R>::make((R)0, (R)0);
  __syncthreads();
  double* d = de + (size_t)b * 2 * n;
  if (threadIdx.x == 0) {
    d[0] = a[0].x;
    count[b] = 0u;
    tau[(size_t)b * n] = 0.0;
    beta[(size_t)b * n] = zmake(0.0, 0.0);
  }
  if (n > 1) householder<R>(a, n, 0, vb, tau + (size_t)b * n, beta + (size_t)b * n, d + n, sh);
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

// FP32: 3 CTAs per SM (memory latency needs warps); FP64: 2 (its pipe is the limit).
// TS = 64 (4 x 4 elements per thread) or 32 (2 x 2): the tile edge is tuned per n.
template <typename R, int TS>
__global__ void __launch_bounds__(NT, sizeof(R) == 4 ? 3 : 2) tridiag_step_kernel(typename Cplx<R>::T* __restrict__ A,
                                                             int n, int j,
                                                             typename Cplx<R>::T* __restrict__ vec,
                                                             typename Cplx<R>::T* __restrict__ part,
                                                             double* __restrict__ de,
                                                             double* __restrict__ tau,
                                                             zd* __restrict__ beta,
                                                             unsigned* __restrict__ count,
                                                             int ntl) {
  typedef typename Cplx<R>::T C;
  // Thread (tx, ty) owns rows R*TS + tx + 16v and columns S*TS + ty + 16u,
  // u, v < EPT: its EPT^2 elements give EPT row and EPT column partials of p,
  // reduced once per tile through shared memory.
  constexpr int EPT = TS / 16;
  __shared__ C vpS[TS], wpS[TS], vcS[TS];
  __shared__ C rowred[16][TS];   // [ty][row]
  __shared__ C colred[16][TS];   // [tx][col]
  __shared__ double sh[NT / 32 + 1];
  __shared__ int is_last;

  const int b = blockIdx.y, tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int nt = (n + TS - 1) / TS, t0 = (j + 1) / TS, r0 = j + 1;   // TS: template
  const C zero = Cplx<R>::make((R)0, (R)0);
  C* a = A + (size_t)b * n * n;
  C* vb = vec + (size_t)b * 3 * n;
  C* vcur = vb + (size_t)(j & 1) * n;
  C* vprev = vb + (size_t)((j + 1) & 1) * n;
  C* w = vb + 2 * (size_t)n;
  C* pt = part + (size_t)b * nt * n;

  int bi, bk;
  tri_index(blockIdx.x, bi, bk);
  const int Rt = t0 + bi, St = t0 + bk;
  const int rbase = Rt * TS, sbase = St * TS;

  if (tid < TS) {
    const int s = sbase + tid;
    const bool ok = s < n && s >= r0;
    vpS[tid] = ok ? vprev[s] : zero;
    wpS[tid] = ok ? w[s] : zero;
    vcS[tid] = ok ? vcur[s] : zero;
  }
  C vpr[EPT], wpr[EPT], vcr[EPT], racc[EPT];
#pragma unroll
  for (int v = 0; v < EPT; ++v) {
    const int r = rbase + tx + 16 * v;
    const bool ok = r < n && r >= r0;
    vpr[v] = ok ? vprev[r] : zero;
    wpr[v] = ok ? w[r] : zero;
    vcr[v] = ok ? vcur[r] : zero;
    racc[v] = zero;
  }
  __syncthreads();

  // FP32: all 16 loads first (the stores below could alias them as far as
  // the compiler knows, which would serialise one load latency per element
  // in a loop that is otherwise light).  FP64: interleaved, the FP64 pipe
  // hides the latency and the registers are needed for the accumulators.
  constexpr bool kHoist = sizeof(R) == 4;
  C xs[EPT][EPT];
  if constexpr (kHoist) {
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
      const int s = sbase + ty + 16 * u;
#pragma unroll
      for (int v = 0; v < EPT; ++v) {
        const int r = rbase + tx + 16 * v;
        xs[u][v] = (s >= r0 && r < n && r >= s) ? a[r + (size_t)s * n] : zero;
      }
    }
  }
#pragma unroll
  for (int u = 0; u < EPT; ++u) {
    const int sl = ty + 16 * u, s = sbase + sl;
    const C vps = vpS[sl], wps = wpS[sl], vcs = vcS[sl];
    C cacc = zero;
    const bool sok = s >= r0;
#pragma unroll
    for (int v = 0; v < EPT; ++v) {
      const int r = rbase + tx + 16 * v;
      if (sok && r < n && r >= s) {
        C x;
        if constexpr (kHoist) x = xs[u][v];
        else x = a[r + (size_t)s * n];
        x = zfnmac(vpr[v], wps, x);
        x = zfnmac(wpr[v], vps, x);
        if (r == s) x.y = (R)0;
        a[r + (size_t)s * n] = x;
        racc[v] = zfma(x, vcs, racc[v]);
        if (r != s) cacc = zfma(zconj(x), vcr[v], cacc);
      }
    }
    colred[tx][sl] = cacc;
  }
#pragma unroll
  for (int v = 0; v < EPT; ++v) rowred[ty][tx + 16 * v] = racc[v];
  __syncthreads();
  if (tid < 2 * TS) {
    const bool isrow = tid < TS;
    const int l = isrow ? tid : tid - TS;
    C acc = zero;
#pragma unroll
    for (int q = 0; q < 16; ++q) acc = zadd(acc, isrow ? rowred[q][l] : colred[q][l]);
    if (Rt == St) {
      // diagonal tile: row and column partials of the same index meet here
      if (isrow) rowred[0][l] = acc;
      else colred[0][l] = acc;
    } else if (isrow) {
      if (rbase + l < n) pt[(size_t)St * n + rbase + l] = acc;
    } else {
      pt[(size_t)Rt * n + sbase + l] = acc;
    }
  }
  if (Rt == St) {
    __syncthreads();
    if (tid < TS && rbase + tid < n)
      pt[(size_t)Rt * n + rbase + tid] = zadd(rowred[0][tid], colred[0][tid]);
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) is_last = (atomicAdd(count + b, 1u) == (unsigned)(ntl - 1));
  __syncthreads();
  if (!is_last) return;
  __threadfence();

  // ---- epilogue: one CTA per matrix
  const R tj = (R)tau[(size_t)b * n + j];
  double kp = 0.0;
  for (int rr = r0 + tid; rr < n; rr += NT) {
    C p = zero;
    for (int t = t0; t < nt; ++t) p = zadd(p, ldg_cg(pt + (size_t)t * n + rr));
    p = zscale(p, tj);
    w[rr] = p;
    const C v = vcur[rr];
    kp = fma((double)v.x, (double)p.x, fma((double)v.y, (double)p.y, kp));
  }
  const R K = (R)(0.5 * (double)tj * block_sum(kp, sh));
  for (int rr = r0 + tid; rr < n; rr += NT) {
    const C v = vcur[rr];
    w[rr] = zsub(w[rr], zscale(v, K));
  }
  __syncthreads();
  const C wj = w[r0], vj = vcur[r0];
  for (int rr = r0 + tid; rr < n; rr += NT) {
    C* ap = a + rr + (size_t)r0 * n;
    C x = ldg_cg(ap);
    x = zfnmac(vcur[rr], wj, x);
    x = zfnmac(w[rr], vj, x);
    if (rr == r0) x.y = (R)0;
    *ap = x;
  }
  __syncthreads();
  double* d = de + (size_t)b * 2 * n;
  if (tid == 0) {
    d[r0] = (double)a[r0 + (size_t)r0 * n].x;
    count[b] = 0u;
  }
  if (r0 + 1 < n)
    householder<R>(a, n, r0, vprev, tau + (size_t)b * n + r0, beta + (size_t)b * n + r0,
                   d + n + r0, sh);
}

}  // namespace

size_t bs_tridiag_vec_elems(int n) { return 3 * (size_t)n; }
size_t bs_tridiag_part_elems(int n) { return (size_t)((n + TSMIN - 1) / TSMIN) * n; }

template <typename R, int TS>
static int launch_steps(typename Cplx<R>::T* A, int n, int batch, typename Cplx<R>::T* vec,
                        typename Cplx<R>::T* part, double* de, double* tau, zd* beta,
                        unsigned* count, cudaStream_t s) {
  tridiag_init_kernel<R><<<batch, NT, 0, s>>>(A, n, vec, de, tau, beta, count);
  BS_CHECK_LAUNCH("tridiag_init_kernel");
  const int nt = (n + TS - 1) / TS;
  for (int j = 0; j + 1 < n; ++j) {
    const int m = nt - (j + 1) / TS;
    const int ntl = m * (m + 1) / 2;
    tridiag_step_kernel<R, TS><<<dim3(ntl, batch), NT, 0, s>>>(A, n, j, vec, part, de, tau, beta,
                                                               count, ntl);
    BS_CHECK_LAUNCH("tridiag_step_kernel");
  }
  return BS_OK;
}

// FP64, n <= 600: 64-tiles while a step has enough of them to fill the GPU,
// then 32-tiles (four times as many CTAs) for the small trailing blocks of
// the last steps.  Each step writes and reduces its own partial sums, so the
// tile edge may change from one step to the next.  Larger matrices keep
// 64-tiles throughout (their tail is a negligible share of the steps).
static int launch_steps_fp64(zd* A, int n, int batch, zd* vec, zd* part, double* de, double* tau,
                             zd* beta, unsigned* count, cudaStream_t s) {
  if (n > 600) return launch_steps<double, 64>(A, n, batch, vec, part, de, tau, beta, count, s);
  tridiag_init_kernel<double><<<batch, NT, 0, s>>>(A, n, vec, de, tau, beta, count);
  BS_CHECK_LAUNCH("tridiag_init_kernel");
  const long fill = 2L * 2 * bs_sm_count();   // two waves of the 64-tile kernel (2 CTAs per SM)
  const int nt64 = (n + 63) / 64, nt32 = (n + 31) / 32;
  for (int j = 0; j + 1 < n; ++j) {
    const int m64 = nt64 - (j + 1) / 64;
    const int ntl64 = m64 * (m64 + 1) / 2;
    if ((long)ntl64 * batch >= fill) {
      tridiag_step_kernel<double, 64><<<dim3(ntl64, batch), NT, 0, s>>>(A, n, j, vec, part, de,
                                                                         tau, beta, count, ntl64);
    } else {
      const int m32 = nt32 - (j + 1) / 32;
      const int ntl32 = m32 * (m32 + 1) / 2;
      tridiag_step_kernel<double, 32><<<dim3(ntl32, batch), NT, 0, s>>>(A, n, j, vec, part, de,
                                                                         tau, beta, count, ntl32);
    }
    BS_CHECK_LAUNCH("tridiag_step_kernel");
  }
  return BS_OK;
}

template <typename R>
int bs_launch_tridiag(typename Cplx<R>::T* A, int n, int batch, typename Cplx<R>::T* vec,
                      typename Cplx<R>::T* part, double* de, double* tau, zd* beta,
                      unsigned* count, cudaStream_t s, int tile) {
  if (tile == 0) tile = 64;
  // The whole batch runs in every step launch.  (Reducing it in L2-sized
  // groups one after another was measured slower for FP32: the per-step
  // launch and epilogue latency then repeats once per group.)
  if (tile == 32)
    return launch_steps<R, 32>(A, n, batch, vec, part, de, tau, beta, count, s);
  if constexpr (sizeof(R) == 8)
    return launch_steps_fp64(A, n, batch, vec, part, de, tau, beta, count, s);
  return launch_steps<R, 64>(A, n, batch, vec, part, de, tau, beta, count, s);
}

template int bs_launch_tridiag<double>(zd*, int, int, zd*, zd*, double*, double*, zd*, unsigned*,
                                       cudaStream_t, int);
template int bs_launch_tridiag<float>(zf*, int, int, zf*, zf*, double*, double*, zd*, unsigned*,
                                      cudaStream_t, int);
