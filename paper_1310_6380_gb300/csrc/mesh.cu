// Form factors of a mesh cell: the centroid rule of Sec. III over arbitrary
// elements (the paper's triangle meshes) instead of pixels,
//   ghat_f(d) = sum_e w_f(e) exp(-i G_d . c_e),  d in [-2M, 2M]^2,
// with w = area times each per-phase material field (1/(lam+mu), 1/mu, rho,
// or the seven of an anisotropic cell) and w = area for a last field, whose
// form factors give I1 = int conj(f_a) f_b (a mesh does not make it
// diagonal).  With the centroid c_e = s_e h1 + t_e h2 the phase separates into
// exp(-2 pi i da s_e) exp(-2 pi i db t_e), so each field is the contraction
// over elements of a (2M+1) x nel table (da >= 0 only: ghat(-d) = conj ghat(d)
// for real fields) with a D x nel table.  It runs in FP64 on the CUDA cores:
// element chunks per CTA, tables staged per tile of elements in shared
// memory, a fixed-order reduction over chunks; the cost is (nf + 1)(2M+1) D nel
// complex products (7 MFLOP for a 1000-element isotropic mesh at M = 5).
#include <algorithm>

#include "bs_internal.h"

namespace {

constexpr int MT = 256;   // threads per CTA
constexpr int TE = 32;    // elements per shared-memory tile
constexpr int PPT = 8;    // (da, db) pairs per thread: (2M+1)(4M+1) <= 1891 <= 8 * 256

int mesh_chunks(int nel) { return std::max(1, std::min(152, (nel + 255) / 256)); }

// part[f][ch][r][db] = sum_{e in chunk ch} w_f(e) exp(-2 pi i (r s_e + (db - 2M) t_e)), r = 0..2M
__global__ void __launch_bounds__(MT)
mesh_partial_kernel(const double* __restrict__ cen, const double* __restrict__ area,
                    const uint16_t* __restrict__ phase, const double* __restrict__ tab, int np,
                    int nf, int nel, int M, int nch, zd* __restrict__ part) {
  extern __shared__ zd sm[];
  const int R = 2 * M + 1, D = 4 * M + 1, npair = R * D;
  zd* Ea = sm;              // [TE][R]: w_f exp(-2 pi i r s)
  zd* Eb = sm + TE * R;     // [TE][D]: exp(-2 pi i (db - 2M) t)
  const int ch = blockIdx.x, f = blockIdx.y, tid = threadIdx.x;
  const long e0 = (long)nel * ch / nch, e1 = (long)nel * (ch + 1) / nch;
  zd acc[PPT];
#pragma unroll
  for (int i = 0; i < PPT; ++i) acc[i] = zmake(0.0, 0.0);
  for (long t0 = e0; t0 < e1; t0 += TE) {
    __syncthreads();
    for (int idx = tid; idx < TE * (R + D); idx += MT) {
      const int el = idx / (R + D), row = idx % (R + D);
      const long e = t0 + el;
      zd v = zmake(0.0, 0.0);
      if (e < e1) {
        double w = 1.0, x;
        if (row < R) {
          const double a = area[e];
          w = f < nf ? a * tab[(size_t)f * np + phase[e]] : a;
          x = 2.0 * row * cen[2 * e];
        } else {
          x = 2.0 * (row - R - 2 * M) * cen[2 * e + 1];
        }
        x -= 2.0 * floor(0.5 * x);           // exp(-i pi x) depends on x mod 2 only
        double sn, cs;
        sincospi(x, &sn, &cs);
        v = zmake(w * cs, -w * sn);
      }
      if (row < R)
        Ea[el * R + row] = v;
      else
        Eb[el * D + row - R] = v;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
      const int p = tid + i * MT;
      if (p < npair) {
        const int r = p / D, db = p % D;
        zd a = acc[i];
        for (int el = 0; el < TE; ++el) a = zfma(Ea[el * R + r], Eb[el * D + db], a);
        acc[i] = a;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < PPT; ++i) {
    const int p = tid + i * MT;
    if (p < npair) part[((size_t)f * nch + ch) * npair + p] = acc[i];
  }
}

// ghat[f][2M + r][db] = sum over chunks (in order); the rows da < 2M, and the
// half row da = 2M, db < 2M, are the conjugates of the mirrored entries
__global__ void mesh_reduce_kernel(const zd* __restrict__ part, int M, int nch,
                                   zd* __restrict__ ghat) {
  const int R = 2 * M + 1, D = 4 * M + 1, npair = R * D;
  const int f = blockIdx.y;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npair) return;
  const int r = p / D, db = p % D;
  if (r == 0 && db < 2 * M) return;       // written as a mirror below
  zd v = zmake(0.0, 0.0);
  for (int ch = 0; ch < nch; ++ch) {
    const zd x = part[((size_t)f * nch + ch) * npair + p];
    v.x += x.x;
    v.y += x.y;
  }
  zd* g = ghat + (size_t)f * D * D;
  g[(size_t)(2 * M + r) * D + db] = v;
  if (r > 0 || db > 2 * M) g[(size_t)(2 * M - r) * D + (4 * M - db)] = zconj(v);
}

}  // namespace

size_t bs_mesh_partial_elems(int M, int nel, int nfields) {
  return (size_t)nfields * mesh_chunks(nel) * (2 * M + 1) * (4 * M + 1);
}

int bs_launch_mesh_assembly(bs_cell* c, cudaStream_t s) {
  const int M = c->M, R = 2 * M + 1, D = 4 * M + 1, nch = mesh_chunks(c->nel);
  if (R * D > PPT * MT) {
    bs_set_error("mesh form factors: M = %d exceeds the kernel's pair capacity", M);
    return BS_EINVAL;
  }
  const size_t smem = (size_t)TE * (R + D) * sizeof(zd);
  cudaFuncSetAttribute(mesh_partial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem);
  TRY_LAUNCH(bs_launch_table(c, s));
  const int nfl = c->nf + 1;     // the material fields and the constant 1
  mesh_partial_kernel<<<dim3(nch, nfl), MT, smem, s>>>(c->d_cen, c->d_area, c->d_phase,
                                                      c->d_table, c->nphase, c->nf, c->nel, M,
                                                      nch, c->d_mpart);
  BS_CHECK_LAUNCH("mesh_partial_kernel");
  mesh_reduce_kernel<<<dim3((R * D + 127) / 128, nfl), 128, 0, s>>>(c->d_mpart, M, nch,
                                                                   c->d_ghat);
  BS_CHECK_LAUNCH("mesh_reduce_kernel");
  return BS_OK;
}
