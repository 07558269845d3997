// Householder tridiagonalisation (FP32) with each matrix resident in the
// shared memory of one thread-block cluster for all of its n - 1 steps.
//
// The per-step-launch reduction (tridiag.cu) streams the trailing triangle
// through HBM once per step and pays a launch and a serial epilogue per
// step; for the eigen dimensions of a ragged batch (n <= 608) the whole
// lower triangle fits in the distributed shared memory of a cluster of
// 1..8 CTAs, so this kernel keeps it there and synchronises with cluster
// barriers instead.  Measured on a 256-cell ragged batch (n = 242..578) it is
// 5x slower than the per-step kernel: each matrix's n steps become a serial
// chain of four cluster barriers plus DSMEM round trips, while the per-step
// kernel hides its latency behind thousands of matrices per launch.  It stays
// as an explicit choice (bs_batch_set_tile) for few, small matrices.
//
// Layout: 32 x 32 tiles of the lower triangle, tile l = I(I+1)/2 + J (J <= I)
// owned by CTA l % CS at slot l / CS; element (r, s) of a tile at
// r * 32 + (s ^ r) (XOR swizzle: both row-wise and column-wise warp accesses
// are conflict-free).  Step j (r0 = j + 1), same arithmetic and outputs as
// tridiag.cu (real tau, H = I - tau v v^dagger, v[r0] = 1):
//   A  each CTA, on its tiles with rows, columns >= r0: the rank-2 update of
//      step j-1 and the row / column partials of p = B v_j (warps own whole
//      block rows, then whole block columns: deterministic sums);
//   -- cluster barrier --
//   B  every CTA sums all CTAs' partials (fixed order), forms w_j, updates
//      column r0 on its tiles and the norm partial of the next reflector;
//   -- cluster barrier --
//   C  every CTA forms the reflector scalars (FP64, identical everywhere);
//      owners scale their part of column r0 into v_{j+1};
//   -- cluster barrier --
//   D  every CTA gathers the full v_{j+1}.
// At the end the tiles (now holding the reflectors below the subdiagonal)
// go back to the matrix in global memory.
#include <cooperative_groups.h>

#include "bs_internal.h"

namespace cg = cooperative_groups;

namespace {

constexpr int TS = 32;
constexpr int CT = 256;
constexpr int NW = CT / 32;
constexpr int MAX_CS = 8;
constexpr size_t SMEM_LIMIT = 227 * 1024 - 1024;

struct Geo {
  int n, nt, nl, CS, tpc, npad;
};

__host__ __device__ inline size_t smem_bytes(int tpc, int npad) {
  // tiles, then V[2], W, prow, pcol (complex float), then 2 + CS doubles
  return (size_t)tpc * TS * TS * sizeof(zf) + 5 * (size_t)npad * sizeof(zf) +
         (4 + 2 * MAX_CS) * sizeof(double);
}

__device__ __forceinline__ int tri_base(int I) { return I * (I + 1) / 2; }

__device__ __forceinline__ zf* tile_ptr(zf* tiles, int l, int CS) {
  return tiles + (size_t)(l / CS) * TS * TS;
}
__device__ __forceinline__ int sw(int r, int s) { return r * TS + (s ^ r); }

__device__ __forceinline__ double warp_sumd(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sum over the CTA (identical order in every CTA of the cluster)
__device__ double cta_sum(double v, double* red) {
  v = warp_sumd(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int q = 0; q < NW; ++q) t += red[q];
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(CT, 1)
tridiag_cluster_kernel(zf* __restrict__ A, int n, int nt, int CS, int tpc, int npad,
                       double* __restrict__ de, double* __restrict__ tau_g,
                       zd* __restrict__ beta_g) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int b = blockIdx.x / CS;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nl = nt * (nt + 1) / 2;
  zf* tiles = reinterpret_cast<zf*>(smraw);
  zf* V0 = tiles + (size_t)tpc * TS * TS;
  zf* V1 = V0 + npad;
  zf* W = V1 + npad;
  zf* prow = W + npad;
  zf* pcol = prow + npad;
  double* scal = reinterpret_cast<double*>(pcol + npad);   // [0..NW) reduction scratch
  double* nrm_part = scal + NW;                             // this CTA's norm partial
  double* alpha_slot = nrm_part + 1;                        // re, im of alpha (owner only)
  zf* a = A + (size_t)b * n * n;
  double* d = de + (size_t)b * 2 * n;
  double* e = d + n;
  const zf zero = make_float2(0.f, 0.f);

  // load the owned tiles (outside the matrix: zero)
  for (int q = 0; q < tpc; ++q) {
    const int l = q * CS + rank;
    if (l >= nl) break;
    int I = (int)((sqrtf(8.f * l + 1.f) - 1.f) * 0.5f);
    while (tri_base(I + 1) <= l) ++I;
    while (tri_base(I) > l) --I;
    const int J = l - tri_base(I);
    zf* t = tiles + (size_t)q * TS * TS;
    for (int e2 = tid; e2 < TS * TS; e2 += CT) {
      const int r = e2 % TS, s = e2 / TS;
      const int gr = I * TS + r, gs = J * TS + s;
      t[sw(r, s)] = (gr < n && gs < n && gr >= gs) ? a[gr + (size_t)gs * n] : zero;
    }
  }
  for (int i = tid; i < npad; i += CT) {
    V0[i] = zero;
    V1[i] = zero;
    W[i] = zero;
  }
  __syncthreads();

  // reflector of column c (rows >= c+1) from the current tiles; vout gets v
  // (rows >= c+1, v[c+1] = 1), tau_c / beta_c / e_c to global (rank 0).
  // Contains two cluster barriers.
  auto reflector = [&](int c, zf* vout, double& tau_out) {
    const int rA = c + 1;               // alpha row
    const int J = c / TS, sl = c % TS;
    double s2 = 0.0;
    // norm partial over owned elements (r, c), r >= c + 2
    for (int I = J; I < nt; ++I) {
      const int l = tri_base(I) + J;
      if (l % CS != rank) continue;
      const zf* t = tile_ptr(tiles, l, CS);
      for (int rl = tid; rl < TS; rl += CT) {
        const int r = I * TS + rl;
        if (r >= rA + 1 && r < n) {
          const zf x = t[sw(rl, sl)];
          s2 += (double)x.x * x.x + (double)x.y * x.y;
        }
        if (r == rA) {
          const zf x = t[sw(rl, sl)];
          alpha_slot[0] = x.x;
          alpha_slot[1] = x.y;
        }
      }
    }
    s2 = cta_sum(s2, scal);
    if (tid == 0) nrm_part[0] = s2;
    cluster.sync();
    // every CTA: the same scalars
    double tot = 0.0;
    for (int q = 0; q < CS; ++q) tot += *cluster.map_shared_rank(nrm_part, q);
    const int lA = tri_base(rA / TS) + J;
    const double* al = cluster.map_shared_rank(alpha_slot, lA % CS);
    const zd alpha = zmake(al[0], al[1]);
    const double aa = hypot(alpha.x, alpha.y);
    const double nu = sqrt(fma(aa, aa, tot));
    double tau = 0.0;
    zd scale = zmake(0.0, 0.0), beta = zmake(0.0, 0.0);
    if (nu > 0.0) {
      beta = aa > 0.0 ? zscale(alpha, -nu / aa) : zmake(-nu, 0.0);
      tau = (aa + nu) / nu;
      const zd den = zsub(alpha, beta);
      const double dd = den.x * den.x + den.y * den.y;
      scale = zmake(den.x / dd, -den.y / dd);
    }
    tau_out = tau;
    if (rank == 0 && tid == 0) {
      tau_g[(size_t)b * n + c] = tau;
      beta_g[(size_t)b * n + c] = beta;
      e[c] = nu;
    }
    // owners scale their part of the column into v (tile and vout)
    for (int I = J; I < nt; ++I) {
      const int l = tri_base(I) + J;
      if (l % CS != rank) continue;
      zf* t = tile_ptr(tiles, l, CS);
      for (int rl = tid; rl < TS; rl += CT) {
        const int r = I * TS + rl;
        if (r >= rA + 1 && r < n) {
          const zf x = t[sw(rl, sl)];
          const zd y = zmul(zmake(x.x, x.y), scale);
          const zf v = make_float2((float)y.x, (float)y.y);
          t[sw(rl, sl)] = v;
          vout[r] = v;
        }
      }
    }
    cluster.sync();
    // gather v (rows >= c + 2) from the owners
    for (int r = rA + 1 + tid; r < n; r += CT) {
      const int l = tri_base(r / TS) + J;
      const int own = l % CS;
      if (own != rank) vout[r] = *cluster.map_shared_rank(vout + r, own);
    }
    if (tid == 0) vout[rA] = make_float2(1.f, 0.f);
    __syncthreads();
  };

  if (rank == 0 && tid == 0) {
    const zf* t0 = tile_ptr(tiles, 0, CS);
    d[0] = (double)t0[sw(0, 0)].x;
    tau_g[(size_t)b * n] = 0.0;
    beta_g[(size_t)b * n] = zmake(0.0, 0.0);
  }
  double tau_cur = 0.0;
  if (n > 1) reflector(0, V0, tau_cur);
  // keep the cluster together before the first step reads remote buffers
  cluster.sync();

  for (int j = 0; j + 1 < n; ++j) {
    const int r0 = j + 1, t0 = r0 / TS;
    zf* vcur = (j & 1) ? V1 : V0;
    zf* vprev = (j & 1) ? V0 : V1;   // v_{j-1}; becomes v_{j+1}
    const bool upd = j >= 1;
    // ---- A: update of step j-1 and partials of p = B v_j
    // pass 1 (lane = row): warp w takes block rows I = t0 + w, t0 + w + NW, ...
    for (int I = t0 + warp; I < nt; I += NW) {
      const int r = I * TS + lane;
      const bool rok = r >= r0 && r < n;
      const zf vr_p = rok ? vprev[r] : zero, wr_p = rok ? W[r] : zero;
      zf racc = zero;
      for (int J = t0; J <= I; ++J) {
        const int l = tri_base(I) + J;
        if (l % CS != rank) continue;
        zf* t = tile_ptr(tiles, l, CS);
#pragma unroll 4
        for (int sl = 0; sl < TS; ++sl) {
          const int s = J * TS + sl;
          if (!rok || s < r0 || s > r) continue;
          zf x = t[sw(lane, sl)];
          if (upd) {
            x = zfnmac(vr_p, W[s], x);
            x = zfnmac(wr_p, vprev[s], x);
            if (r == s) x.y = 0.f;
            t[sw(lane, sl)] = x;
          }
          racc = zfma(x, vcur[s], racc);
        }
      }
      prow[I * TS + lane] = racc;
    }
    __syncthreads();
    // pass 2 (lane = column): warp w takes block columns J = t0 + w, ...
    for (int J = t0 + warp; J < nt; J += NW) {
      const int s = J * TS + lane;
      const bool sok = s >= r0 && s < n;
      zf cacc = zero;
      for (int I = J; I < nt; ++I) {
        const int l = tri_base(I) + J;
        if (l % CS != rank) continue;
        const zf* t = tile_ptr(tiles, l, CS);
#pragma unroll 4
        for (int rl = 0; rl < TS; ++rl) {
          const int r = I * TS + rl;
          if (!sok || r <= s || r >= n) continue;
          const zf x = t[sw(rl, lane)];
          cacc = zfma(zconj(x), vcur[r], cacc);
        }
      }
      pcol[J * TS + lane] = cacc;
    }
    // block rows / columns below t0 are not written this step: zero the
    // entries the reduction reads that no warp produced
    for (int i = tid; i < t0 * TS; i += CT) {
      prow[i] = zero;
      pcol[i] = zero;
    }
    cluster.sync();
    // ---- B: p, w_j, column r0
    double kp = 0.0;
    for (int r = r0 + tid; r < n; r += CT) {
      zf p = zero;
      for (int q = 0; q < CS; ++q) {
        p = zadd(p, *cluster.map_shared_rank(prow + r, q));
        p = zadd(p, *cluster.map_shared_rank(pcol + r, q));
      }
      p = zscale(p, (float)tau_cur);
      W[r] = p;
      const zf v = vcur[r];
      kp = fma((double)v.x, (double)p.x, fma((double)v.y, (double)p.y, kp));
    }
    const float K = (float)(0.5 * tau_cur * cta_sum(kp, scal));
    for (int r = r0 + tid; r < n; r += CT) W[r] = zsub(W[r], zscale(vcur[r], K));
    __syncthreads();
    {
      const zf wj = W[r0], vj = vcur[r0];
      const int J = r0 / TS, sl = r0 % TS;
      for (int I = J; I < nt; ++I) {
        const int l = tri_base(I) + J;
        if (l % CS != rank) continue;
        zf* t = tile_ptr(tiles, l, CS);
        for (int rl = tid; rl < TS; rl += CT) {
          const int r = I * TS + rl;
          if (r < r0 || r >= n) continue;
          zf x = t[sw(rl, sl)];
          x = zfnmac(vcur[r], wj, x);
          x = zfnmac(W[r], vj, x);
          if (r == r0) {
            x.y = 0.f;
            d[r0] = (double)x.x;
          }
          t[sw(rl, sl)] = x;
        }
      }
    }
    __syncthreads();
    // ---- C, D: the next reflector (two cluster barriers inside); the
    // last step has none, but keeps the barrier count of the others
    if (r0 + 1 < n) {
      reflector(r0, vprev, tau_cur);
    } else {
      cluster.sync();
      cluster.sync();
    }
    // every CTA has finished reading this step's partials and v before the
    // next step overwrites them
    cluster.sync();
  }

  // the tiles (reflectors below the subdiagonal) back to the matrix
  for (int q = 0; q < tpc; ++q) {
    const int l = q * CS + rank;
    if (l >= nl) break;
    int I = (int)((sqrtf(8.f * l + 1.f) - 1.f) * 0.5f);
    while (tri_base(I + 1) <= l) ++I;
    while (tri_base(I) > l) --I;
    const int J = l - tri_base(I);
    const zf* t = tiles + (size_t)q * TS * TS;
    for (int e2 = tid; e2 < TS * TS; e2 += CT) {
      const int r = e2 % TS, s = e2 / TS;
      const int gr = I * TS + r, gs = J * TS + s;
      if (gr < n && gs < n && gr >= gs) a[gr + (size_t)gs * n] = t[sw(r, s)];
    }
  }
}

bool geometry(int n, Geo& g) {
  g.n = n;
  g.nt = (n + TS - 1) / TS;
  g.nl = g.nt * (g.nt + 1) / 2;
  g.npad = g.nt * TS;
  for (int CS = 1; CS <= MAX_CS; CS *= 2) {
    const int tpc = (g.nl + CS - 1) / CS;
    if (smem_bytes(tpc, g.npad) <= SMEM_LIMIT) {
      g.CS = CS;
      g.tpc = tpc;
      return true;
    }
  }
  return false;
}

}  // namespace

bool bs_tridiag_cluster_fits(int n) {
  Geo g;
  return n >= 2 && geometry(n, g);
}

int bs_launch_tridiag_cluster(zf* A, int n, int batch, double* de, double* tau, zd* beta,
                              cudaStream_t s) {
  Geo g;
  if (n < 2 || !geometry(n, g)) {
    bs_set_error("cluster tridiagonalisation: n = %d does not fit a cluster", n);
    return BS_EINVAL;
  }
  const size_t sm = smem_bytes(g.tpc, g.npad);
  cudaError_t e = cudaFuncSetAttribute(tridiag_cluster_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return bs_cuda_status(e, "cluster tridiagonalisation attribute");
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(batch * g.CS));
  cfg.blockDim = dim3(CT);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = g.CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, tridiag_cluster_kernel, A, n, g.nt, g.CS, g.tpc, g.npad, de, tau,
                         beta);
  if (e != cudaSuccess) return bs_cuda_status(e, "cluster tridiagonalisation launch");
  BS_CHECK_LAUNCH("tridiag_cluster_kernel");
  return BS_OK;
}
