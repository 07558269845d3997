// Form-factor assembly (material fields + separable Fourier sums) and the
// plane-wave (Toeplitz) expansion of the form factors.
//
// The compliance and density integrals of Eqs. (eo) and (ep), evaluated
// with the centroid rule of Sec. III on a P x P pixel map, depend on the
// plane-wave pair (a, b) only through the difference d = a - b and
// factor over the two lattice directions:
//   ghat(da, db) = (V/P^2) sum_p sum_q g[p][q] E[da][p] E[db][q],
//   E[d][p] = exp(-2 pi i d (p + 1/2) / P),
// because G_d . x_pq = 2 pi (da (p+1/2) + db (q+1/2)) / P for any lattice
// (q^i . h^j = 2 pi delta_ij, Eq. (1)).  For isotropic plane strain the
// compliance Gram matrix needs only the fields 1/(lam+mu) and 1/mu (the
// combinations D1111 +- D1122 and 4 D1212 of the Sec. IV compliance), and
// Omega needs rho.
#include "bs_internal.h"

namespace {

// a1: per-phase material table: 1/(lam+mu), 1/mu, rho
__global__ void table_kernel(const double* __restrict__ lam, const double* __restrict__ mu,
                             const double* __restrict__ rho, int nphase, double* __restrict__ tab) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nphase) return;
  tab[i] = 1.0 / (lam[i] + mu[i]);
  tab[nphase + i] = 1.0 / mu[i];
  tab[2 * nphase + i] = rho[i];
}

// E[d][p] = exp(-i pi dd (2p+1) / P), dd = d - 2M; the angle is reduced
// exactly in integers before sincospi.
__global__ void exp_table_kernel(int P, int M, int D, zd* __restrict__ E) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= D * P) return;
  int d = i / P, p = i % P;
  long long dd = d - 2 * M;
  long long m = (dd * (2 * p + 1)) % (2LL * P);
  if (m < 0) m += 2LL * P;
  double s, c;
  sincospi((double)m / (double)P, &s, &c);
  E[i] = zmake(c, -s);
}

// Stage 1 (Y[f][p][d] = sum_q g_f[p][q] E[d][q]) runs as an exact-slice
// tensor-core contraction, see slices.cu.

// Stage 2: ghat[f][da][db] = w * sum_p E[da][p] Y[f][p][db]
__global__ void stage2_kernel(int P, int D, double w, const zd* __restrict__ E,
                              const zd* __restrict__ Y, zd* __restrict__ ghat) {
  int da = blockIdx.x, f = blockIdx.y;
  const zd* e = E + (size_t)da * P;
  const zd* y = Y + (size_t)f * P * D;
  for (int db = threadIdx.x; db < D; db += blockDim.x) {
    zd acc = zmake(0.0, 0.0);
    for (int p = 0; p < P; ++p) acc = zfma(e[p], y[(size_t)p * D + db], acc);
    ghat[((size_t)f * D + da) * D + db] = zscale(acc, w);
  }
}

// T[f][a + b N] = ghat[f][alpha_a - alpha_b + 2M][beta_a - beta_b + 2M]
__global__ void toeplitz_kernel(const zd* __restrict__ ghat, int M, int N, int D, int nf,
                                zd* __restrict__ T) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t NN = (size_t)N * N;
  if (i >= (size_t)nf * NN) return;
  int f = (int)(i / NN);
  size_t r = i % NN;
  int a = (int)(r % N), b = (int)(r / N);
  int W = 2 * M + 1;
  int aa = a / W, ab = a % W, ba = b / W, bb = b % W;   // (alpha + M, beta + M)
  T[i] = ghat[((size_t)f * D + (aa - ba + 2 * M)) * D + (ab - bb + 2 * M)];
}

}  // namespace

// Per-phase fields of an isotropic cell (an anisotropic cell's table is
// written by bs_set_stiffness): the raw lam/mu/rho copies sit right after
// the nf derived rows.
int bs_launch_table(bs_cell* c, cudaStream_t s) {
  if (c->aniso) return BS_OK;
  const double* raw = c->d_table + (size_t)c->nf * c->nphase;
  table_kernel<<<(c->nphase + 127) / 128, 128, 0, s>>>(raw, raw + c->nphase, raw + 2 * c->nphase,
                                                       c->nphase, c->d_table);
  BS_CHECK_LAUNCH("table_kernel");
  return BS_OK;
}

int bs_launch_assembly(bs_cell* c, cudaStream_t s) {
  int P = c->P, D = c->D;
  TRY_LAUNCH(bs_launch_table(c, s));
  exp_table_kernel<<<(D * P + 255) / 256, 256, 0, s>>>(P, c->M, D, c->d_E);
  BS_CHECK_LAUNCH("exp_table_kernel");
  // first stage (the bulk: nf P^2 D complex-by-real products) on the tensor cores
  TRY_LAUNCH(bs_launch_fields_tc(c, s));
  stage2_kernel<<<dim3(D, c->nf), 64, 0, s>>>(P, D, c->V / ((double)P * P), c->d_E, c->d_Y,
                                              c->d_ghat);
  BS_CHECK_LAUNCH("stage2_kernel");
  return BS_OK;
}

int bs_launch_toeplitz(bs_cell* c, cudaStream_t s) {
  const size_t NN = (size_t)c->N * c->N, tot = (size_t)c->nf * NN;
  toeplitz_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(c->d_ghat, c->M, c->N, c->D,
                                                                 c->nf, c->d_T);
  BS_CHECK_LAUNCH("toeplitz_kernel");
  if (c->mesh) {
    // the Gram matrix of the plane waves under the centroid rule (the last field, 1)
    toeplitz_kernel<<<(unsigned)((NN + 255) / 256), 256, 0, s>>>(
        c->d_ghat + (size_t)c->nf * c->D * c->D, c->M, c->N, c->D, 1, c->d_I1);
    BS_CHECK_LAUNCH("toeplitz_kernel I1");
  }
  return BS_OK;
}
