// 3-D voxelated cells (the paper's outlook: three displacement and six
// stress components, 9 (2M+1)^3 unknowns), FP64 path.
//
// Form factors: ghat_f(d) = (V/P^3) sum_pqr g_f[p][q][r] E[da][p] E[db][q] E[dc][r]
// with E[d][p] = exp(-i pi (d - 2M)(2p + 1)/P), three separable stages on the
// CUDA cores, for g = 1/(3 lam + 2 mu), 1/mu, rho.
//
// Isotropic Phi in an orthonormal stress basis (Sec. IV in 3-D): the
// hydrostatic direction (1,1,1,0,0,0)/sqrt3 sees T_h = T[1/(3 lam + 2 mu)],
// the two deviatoric normal directions (1,-1,0)/sqrt2, (1,1,-2)/sqrt6 see
// T[1/(2 mu)] = T_m / 2 and the three shears (with the Voigt factor 2 of
// Eq. (ep)) see T_m = T[1/mu].  With H (v_c x I) = i V [diag h_c[l]]_l, where
// h_c[l] = sum_j alpha_{c,l,j} K_j, T_X^-1 = Z_X Z_X^dagger and
// F_X^a = L_R^-1 diag(s_a) Z_X (s_0 = 1, s_j = G_j), block (l, l') of
//   C(k) = L_Omega^-1 H Phi^-1 H^* L_Omega^-dagger
// is V^2 sum_X sum_{jj'} B_X[l][l'][j][j'] (k_j F^0 + F^j)(k_j' F^0 + F^j')^dagger
// with B_X = sum over the directions c of X of s_c alpha_{c,l,j} alpha_{c,l',j'}
// (s = 1, 2, 2, 1, 1, 1).  So C(k) has ten k-monomials (1, k_i, k_i^2,
// k_i k_j), combinations of the twenty products P_X^{ab} = F_X^a F_X^b^dagger,
// which run as exact-slice tensor-core contractions like the 2-D ones.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "bs_internal.h"

struct bs_cell3 {
  int P, M, N, n, D, nphase;
  double h[3][3], q[3][3], V;
  bool assembled;
  uint16_t* d_phase;   // P^3
  double* d_tab;       // 3 x nphase: 1/(3 lam + 2 mu), 1/mu, rho
  zd* d_E;             // D x P
  zd* d_Y1;            // 3 x P^2 x D
  zd* d_Y2;            // 3 x P x D^2
  zd* d_ghat;          // 3 x D^3
  zd* d_T;             // 3 x N x N (h, mu, rho), Cholesky in place
  zd* d_Linv;          // 3 x N x N
  zd* d_LinvR2;        // L_R^-1 twice
  double* d_G;         // 3 x N
  zd* d_F;             // 2 x 4 x N x N
  zd* d_Pp;            // 2 x 10 x N x N
  zd* d_Cm;            // 10 x n x n
  double* d_coef;      // 10 x 3 x 3 x 2 x 4 x 4 monomial coefficients
  int* d_info;
  uint16_t *d_mA, *d_mB;
  float* d_mD;
  int *d_meA, *d_meB;
  // per-k workspace
  int kcap, wcap;
  zd *d_C, *d_vec, *d_part, *d_beta;
  double *d_de, *d_tau, *d_Q, *d_w;
  unsigned* d_count;
  int* d_stat;
  BandWs* band;        // two-stage reduction workspace (allocated on first use)
};

namespace {

constexpr int NMONO = 10;

__global__ void exp3_kernel(int P, int M, int D, zd* __restrict__ E) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= D * P) return;
  const int d = i / P, p = i % P;
  const long long dd = d - 2 * M;
  long long m = (dd * (2 * p + 1)) % (2LL * P);
  if (m < 0) m += 2LL * P;
  double s, c;
  sincospi((double)m / (double)P, &s, &c);
  E[i] = zmake(c, -s);
}

// Y1[f][(p P + q) D + dc] = sum_r g_f[p][q][r] E[dc][r]
__global__ void ff3_stage1(const uint16_t* __restrict__ phase, const double* __restrict__ tab,
                           int np, int P, int D, const zd* __restrict__ E, zd* __restrict__ Y1) {
  const size_t tot = (size_t)3 * P * P * D;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= tot) return;
  const int dc = (int)(i % D);
  const size_t pq = (i / D) % ((size_t)P * P);
  const int f = (int)(i / ((size_t)P * P * D));
  const uint16_t* ph = phase + pq * P;
  const double* t = tab + (size_t)f * np;
  const zd* e = E + (size_t)dc * P;
  zd acc = zmake(0.0, 0.0);
  for (int r = 0; r < P; ++r) {
    const double g = t[ph[r]];
    acc.x = fma(g, e[r].x, acc.x);
    acc.y = fma(g, e[r].y, acc.y);
  }
  Y1[i] = acc;
}

// Y2[f][(p D + db) D + dc] = sum_q E[db][q] Y1[f][(p P + q) D + dc]
__global__ void ff3_stage2(const zd* __restrict__ Y1, int P, int D, const zd* __restrict__ E,
                           zd* __restrict__ Y2) {
  const size_t tot = (size_t)3 * P * D * D;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= tot) return;
  const int dc = (int)(i % D), db = (int)((i / D) % D);
  const int p = (int)((i / ((size_t)D * D)) % P), f = (int)(i / ((size_t)P * D * D));
  const zd* y = Y1 + ((size_t)f * P * P + (size_t)p * P) * D + dc;
  const zd* e = E + (size_t)db * P;
  zd acc = zmake(0.0, 0.0);
  for (int q = 0; q < P; ++q) acc = zfma(e[q], y[(size_t)q * D], acc);
  Y2[i] = acc;
}

// ghat[f][(da D + db) D + dc] = w sum_p E[da][p] Y2[f][(p D + db) D + dc]
__global__ void ff3_stage3(const zd* __restrict__ Y2, int P, int D, double w,
                           const zd* __restrict__ E, zd* __restrict__ ghat) {
  const size_t D3 = (size_t)D * D * D, tot = 3 * D3;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= tot) return;
  const size_t dbc = i % ((size_t)D * D);
  const int da = (int)((i / ((size_t)D * D)) % D), f = (int)(i / D3);
  const zd* y = Y2 + (size_t)f * P * D * D + dbc;
  const zd* e = E + (size_t)da * P;
  zd acc = zmake(0.0, 0.0);
  for (int p = 0; p < P; ++p) acc = zfma(e[p], y[(size_t)p * D * D], acc);
  ghat[i] = zscale(acc, w);
}

// T[f][a + b N] = ghat[f][alpha_a - alpha_b][beta_a - beta_b][gamma_a - gamma_b] (+2M each)
__global__ void toeplitz3_kernel(const zd* __restrict__ ghat, int M, int N, int D,
                                 zd* __restrict__ T) {
  const size_t NN = (size_t)N * N;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * NN) return;
  const int f = (int)(i / NN);
  const size_t r = i % NN;
  const int a = (int)(r % N), b = (int)(r / N), W = 2 * M + 1;
  const int aa = a / (W * W), ab = (a / W) % W, ac = a % W;
  const int ba = b / (W * W), bb = (b / W) % W, bc = b % W;
  T[i] = ghat[(size_t)f * D * D * D +
              ((size_t)(aa - ba + 2 * M) * D + (ab - bb + 2 * M)) * D + (ac - bc + 2 * M)];
}

__device__ __forceinline__ int pidx4(int a, int b) {   // a <= b < 4
  return a == 0 ? b : a == 1 ? 3 + b : a == 2 ? 5 + b : 9;
}

// Cm[t][e] = V2 sum_{X,a,b} coef[t][l][l'][X][a][b] P_X^{ab}(i, j),
// P^{ab} = (P^{ba})^dagger for a > b
__global__ void monomial3_kernel(const zd* __restrict__ Pp, const double* __restrict__ coef,
                                 int N, double V2, zd* __restrict__ Cm) {
  const int n = 3 * N;
  const size_t nn = (size_t)n * n, NN = (size_t)N * N;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nn) return;
  const int r = (int)(e % n), c = (int)(e / n);
  const int l = r / N, lp = c / N, i = r % N, j = c % N;
  zd m[NMONO];
#pragma unroll
  for (int t = 0; t < NMONO; ++t) m[t] = zmake(0.0, 0.0);
  for (int X = 0; X < 2; ++X)
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        const double* cf = coef + (((size_t)(l * 3 + lp) * 2 + X) * 4 + a) * 4 + b;
        // coef[t] stride: 3 * 3 * 2 * 4 * 4 = 288
        bool any = false;
#pragma unroll
        for (int t = 0; t < NMONO; ++t) any = any || cf[(size_t)t * 288] != 0.0;
        if (!any) continue;
        zd p;
        if (a <= b)
          p = Pp[((size_t)X * 10 + pidx4(a, b)) * NN + i + (size_t)j * N];
        else
          p = zconj(Pp[((size_t)X * 10 + pidx4(b, a)) * NN + j + (size_t)i * N]);
#pragma unroll
        for (int t = 0; t < NMONO; ++t) {
          const double w = cf[(size_t)t * 288];
          m[t].x = fma(w, p.x, m[t].x);
          m[t].y = fma(w, p.y, m[t].y);
        }
      }
#pragma unroll
  for (int t = 0; t < NMONO; ++t) Cm[(size_t)t * nn + e] = zscale(m[t], V2);
}

constexpr int KB3 = 32;

// C(k) = sum_t c_t(k) Cm[t], c = (1, k1, k2, k3, k1^2, k2^2, k3^2, k1 k2, k1 k3, k2 k3)
__global__ void builder3_kernel(const zd* __restrict__ Cm, int n, const double* __restrict__ Q,
                                int nk, const double* __restrict__ qv, zd* __restrict__ C) {
  __shared__ double coef[KB3][NMONO];
  const size_t nn = (size_t)n * n;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = e < nn && (int)(e % n) >= (int)(e / n);
  zd m[NMONO];
  if (live) {
#pragma unroll
    for (int t = 0; t < NMONO; ++t) m[t] = Cm[t * nn + e];
  }
  for (int k0 = 0; k0 < nk; k0 += KB3) {
    const int kb = min(KB3, nk - k0);
    __syncthreads();
    if (threadIdx.x < kb) {
      const double* Qk = Q + 3 * (k0 + threadIdx.x);
      double k[3];
      for (int d = 0; d < 3; ++d) k[d] = Qk[0] * qv[d] + Qk[1] * qv[3 + d] + Qk[2] * qv[6 + d];
      double* cf = coef[threadIdx.x];
      cf[0] = 1.0;
      cf[1] = k[0];
      cf[2] = k[1];
      cf[3] = k[2];
      cf[4] = k[0] * k[0];
      cf[5] = k[1] * k[1];
      cf[6] = k[2] * k[2];
      cf[7] = k[0] * k[1];
      cf[8] = k[0] * k[2];
      cf[9] = k[1] * k[2];
    }
    __syncthreads();
    if (!live) continue;
    for (int b = 0; b < kb; ++b) {
      double re = m[0].x, im = m[0].y;
#pragma unroll
      for (int t = 1; t < NMONO; ++t) {
        re = fma(coef[b][t], m[t].x, re);
        im = fma(coef[b][t], m[t].y, im);
      }
      C[(size_t)(k0 + b) * nn + e] = zmake(re, im);
    }
  }
}

// ---- host helpers
bool dev_ptr3(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int fetch3(void* dst, const void* src, size_t bytes) {
  if (dev_ptr3(src)) {
    cudaError_t e = cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bs_cuda_status(e, "3-D cell fetch");
  } else {
    memcpy(dst, src, bytes);
  }
  return BS_OK;
}

template <typename T>
int alloc3(T** p, size_t count, const char* what) {
  *p = nullptr;
  if (count == 0) return BS_OK;
  if (cudaMalloc((void**)p, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    bs_set_error("cudaMalloc(%s, %zu bytes) failed", what, count * sizeof(T));
    return BS_ENOMEM;
  }
  return BS_OK;
}

#define CK3(call, where)                                        \
  do {                                                          \
    cudaError_t e__ = (call);                                   \
    if (e__ != cudaSuccess) return bs_cuda_status(e__, where);  \
  } while (0)

// Monomial coefficients coef[t][l][l'][X][a][b] (t < 10, l, l' < 3, X < 2, a, b < 4)
std::vector<double> monomial_coefficients() {
  const int comp[6][2] = {{0, 0}, {1, 1}, {2, 2}, {1, 2}, {0, 2}, {0, 1}};
  const double r3 = 1.0 / sqrt(3.0), r2 = 1.0 / sqrt(2.0), r6 = 1.0 / sqrt(6.0);
  // stress directions: vector, scale s_c, Gram block X (0: T_h, 1: T_m)
  const double v[6][6] = {{r3, r3, r3, 0, 0, 0}, {r2, -r2, 0, 0, 0, 0},
                          {r6, r6, -2 * r6, 0, 0, 0}, {0, 0, 0, 1, 0, 0},
                          {0, 0, 0, 0, 1, 0}, {0, 0, 0, 0, 0, 1}};
  const double sc[6] = {1, 2, 2, 1, 1, 1};
  const int X_of[6] = {0, 1, 1, 1, 1, 1};
  double alpha[6][3][3] = {};   // [c][l][j]
  for (int c = 0; c < 6; ++c)
    for (int q = 0; q < 6; ++q) {
      const int m = comp[q][0], nn = comp[q][1];
      for (int l = 0; l < 3; ++l) {
        if (l == m) alpha[c][l][nn] += v[c][q];
        if (l == nn && m != nn) alpha[c][l][m] += v[c][q];
      }
    }
  std::vector<double> coef((size_t)NMONO * 288, 0.0);
  auto at = [&](int t, int l, int lp, int X, int a, int b) -> double& {
    return coef[(size_t)t * 288 + (((l * 3 + lp) * 2 + X) * 4 + a) * 4 + b];
  };
  const int quad[3][3] = {{4, 7, 8}, {7, 5, 9}, {8, 9, 6}};
  for (int c = 0; c < 6; ++c)
    for (int l = 0; l < 3; ++l)
      for (int lp = 0; lp < 3; ++lp)
        for (int j = 0; j < 3; ++j)
          for (int jp = 0; jp < 3; ++jp) {
            const double w = sc[c] * alpha[c][l][j] * alpha[c][lp][jp];
            if (w == 0.0) continue;
            const int X = X_of[c];
            at(0, l, lp, X, j + 1, jp + 1) += w;        // F^j F^j'^dagger
            at(1 + j, l, lp, X, 0, jp + 1) += w;        // k_j F^0 F^j'^dagger
            at(1 + jp, l, lp, X, j + 1, 0) += w;        // k_j' F^j F^0^dagger
            at(quad[j][jp], l, lp, X, 0, 0) += w;       // k_j k_j' F^0 F^0^dagger
          }
  return coef;
}

void free_ws3(bs_cell3* c) {
  if (c->band) {
    bs_band_ws_free(c->band);
    delete c->band;
    c->band = nullptr;
  }
  cudaFree(c->d_C);
  cudaFree(c->d_vec);
  cudaFree(c->d_part);
  cudaFree(c->d_beta);
  cudaFree(c->d_de);
  cudaFree(c->d_tau);
  cudaFree(c->d_Q);
  cudaFree(c->d_w);
  cudaFree(c->d_count);
  cudaFree(c->d_stat);
  c->d_C = c->d_vec = c->d_part = c->d_beta = nullptr;
  c->d_de = c->d_tau = c->d_Q = c->d_w = nullptr;
  c->d_count = nullptr;
  c->d_stat = nullptr;
  c->kcap = c->wcap = 0;
}

int ensure_ws3(bs_cell3* c, int kb, int nb) {
  if (kb <= c->kcap && nb <= c->wcap) return BS_OK;
  kb = std::max(kb, c->kcap);
  nb = std::max(nb, c->wcap);
  cudaDeviceSynchronize();
  free_ws3(c);
  const int n = c->n;
  int r = BS_OK;
  if (!r) r = alloc3(&c->d_C, (size_t)kb * n * n, "C(k)");
  if (!r) r = alloc3(&c->d_vec, (size_t)kb * bs_tridiag_vec_elems(n), "tridiag vectors");
  if (!r) r = alloc3(&c->d_part, (size_t)kb * bs_tridiag_part_elems(n), "tridiag partials");
  if (!r) r = alloc3(&c->d_de, (size_t)kb * 2 * n, "tridiagonal");
  if (!r) r = alloc3(&c->d_tau, (size_t)kb * n, "tau");
  if (!r) r = alloc3(&c->d_beta, (size_t)kb * n, "beta");
  if (!r) r = alloc3(&c->d_count, (size_t)kb, "counters");
  if (!r) r = alloc3(&c->d_Q, (size_t)kb * 3, "Q");
  if (!r) r = alloc3(&c->d_w, (size_t)kb * nb, "omega");
  if (!r) r = alloc3(&c->d_stat, (size_t)kb, "status");
  if (r) {
    free_ws3(c);
    return r;
  }
  c->kcap = kb;
  c->wcap = nb;
  return BS_OK;
}

int check3(bs_cell3* c, cudaStream_t s) {
  int info[2] = {0, 0};
  CK3(cudaMemcpyAsync(info, c->d_info, 2 * sizeof(int), cudaMemcpyDeviceToHost, s), "info");
  CK3(cudaStreamSynchronize(s), "sync");
  if (info[0]) {
    bs_set_error("Cholesky of a Gram matrix failed (not positive definite)");
    return BS_ENOTPD;
  }
  if (info[1]) {
    bs_set_error("a tensor-core pipeline wait reached its limit");
    return BS_ECUDA;
  }
  return BS_OK;
}

}  // namespace

extern "C" int bs_destroy_cell3(bs_cell3* c) {
  if (!c) return BS_OK;
  cudaDeviceSynchronize();
  free_ws3(c);
  void* bufs[] = {c->d_phase, c->d_tab, c->d_E, c->d_Y1, c->d_Y2, c->d_ghat, c->d_T, c->d_Linv,
                  c->d_LinvR2, c->d_G, c->d_F, c->d_Pp, c->d_Cm, c->d_coef, c->d_info, c->d_mA,
                  c->d_mB, c->d_mD, c->d_meA, c->d_meB};
  for (void* b : bufs) cudaFree(b);
  delete c;
  return BS_OK;
}

extern "C" int bs_create_cell3(const bs_cell3_desc* d, bs_cell3** out) {
  if (!d || !out) {
    bs_set_error("bs_create_cell3: NULL argument");
    return BS_EINVAL;
  }
  *out = nullptr;
  const int P = d->P, M = d->M, np = d->nphase;
  if (P < 1 || P > 128 || M < 0 || M > 5 || 2 * M + 1 > P || np < 1 || np > 65536 ||
      !d->phase || !d->lam || !d->mu || !d->rho) {
    bs_set_error("bs_create_cell3: need 1 <= P <= 128, 0 <= M <= 5, 2M+1 <= P, 1 <= nphase <= "
                 "65536 and non-NULL arrays (P=%d M=%d nphase=%d)", P, M, np);
    return BS_EINVAL;
  }
  double h[3][3];
  for (int i = 0; i < 3; ++i) {
    h[0][i] = d->h1[i];
    h[1][i] = d->h2[i];
    h[2][i] = d->h3[i];
  }
  // q^i = 2 pi (h_j x h_k) / (h_i . (h_j x h_k))  (Eq. (1))
  auto cross = [](const double* a, const double* b, double* o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
  };
  double c12[3], c23[3], c31[3];
  cross(h[1], h[2], c23);
  cross(h[2], h[0], c31);
  cross(h[0], h[1], c12);
  const double vol = h[0][0] * c23[0] + h[0][1] * c23[1] + h[0][2] * c23[2];
  if (!(fabs(vol) > 0.0) || !isfinite(vol)) {
    bs_set_error("bs_create_cell3: h1, h2, h3 are not a basis");
    return BS_EINVAL;
  }
  std::vector<double> raw(3 * (size_t)np), tab(3 * (size_t)np);
  int r = fetch3(raw.data(), d->lam, np * sizeof(double));
  if (!r) r = fetch3(raw.data() + np, d->mu, np * sizeof(double));
  if (!r) r = fetch3(raw.data() + 2 * np, d->rho, np * sizeof(double));
  if (r) return r;
  for (int i = 0; i < np; ++i) {
    const double lam = raw[i], mu = raw[np + i], rho = raw[2 * np + i];
    if (!isfinite(lam) || !isfinite(mu) || !isfinite(rho) || !(mu > 0.0) ||
        !(3.0 * lam + 2.0 * mu > 0.0) || !(rho > 0.0)) {
      bs_set_error("bs_create_cell3: phase %d has lam=%g mu=%g rho=%g (need mu > 0, "
                   "3 lam + 2 mu > 0, rho > 0, finite)", i, lam, mu, rho);
      return BS_EINVAL;
    }
    tab[i] = 1.0 / (3.0 * lam + 2.0 * mu);
    tab[np + i] = 1.0 / mu;
    tab[2 * np + i] = rho;
  }
  const size_t P3 = (size_t)P * P * P;
  std::vector<uint16_t> ph(P3);
  r = fetch3(ph.data(), d->phase, P3 * sizeof(uint16_t));
  if (r) return r;
  for (size_t i = 0; i < P3; ++i)
    if (ph[i] >= np) {
      bs_set_error("bs_create_cell3: voxel %zu has phase %u >= nphase %d", i, ph[i], np);
      return BS_EINVAL;
    }
  bs_cell3* c = new bs_cell3;
  memset(c, 0, sizeof(*c));
  c->P = P;
  c->M = M;
  const int W = 2 * M + 1;
  c->N = W * W * W;
  c->n = 3 * c->N;
  c->D = 4 * M + 1;
  c->nphase = np;
  c->V = fabs(vol);
  memcpy(c->h, h, sizeof(h));
  for (int i = 0; i < 3; ++i) {
    c->q[0][i] = 2.0 * M_PI * c23[i] / vol;
    c->q[1][i] = 2.0 * M_PI * c31[i] / vol;
    c->q[2][i] = 2.0 * M_PI * c12[i] / vol;
  }
  const int N = c->N, D = c->D, n = c->n;
  const size_t NN = (size_t)N * N, nn = (size_t)n * n;
  if (!r) r = alloc3(&c->d_phase, P3, "phase");
  if (!r) r = alloc3(&c->d_tab, 3 * (size_t)np, "table");
  if (!r) r = alloc3(&c->d_E, (size_t)D * P, "E");
  if (!r) r = alloc3(&c->d_Y1, 3 * (size_t)P * P * D, "Y1");
  if (!r) r = alloc3(&c->d_Y2, 3 * (size_t)P * D * D, "Y2");
  if (!r) r = alloc3(&c->d_ghat, 3 * (size_t)D * D * D, "ghat");
  if (!r) r = alloc3(&c->d_T, 3 * NN, "T");
  if (!r) r = alloc3(&c->d_Linv, 3 * NN, "Linv");
  if (!r) r = alloc3(&c->d_LinvR2, 2 * NN, "L_R^-1 pair");
  if (!r) r = alloc3(&c->d_G, 3 * (size_t)N, "G");
  if (!r) r = alloc3(&c->d_F, 8 * NN, "F");
  if (!r) r = alloc3(&c->d_Pp, 20 * NN, "P");
  if (!r) r = alloc3(&c->d_Cm, NMONO * nn, "Cm");
  if (!r) r = alloc3(&c->d_coef, (size_t)NMONO * 288, "monomial coefficients");
  if (!r) r = alloc3(&c->d_info, 4, "info");
  size_t ma = 0, mb = 0, md = 0;
  bs_zgemm_tc_elems(N, 2, &ma, &mb, &md);
  if (!r) r = alloc3(&c->d_mA, ma, "digit planes A");
  if (!r) r = alloc3(&c->d_mB, mb, "digit planes B");
  if (!r) r = alloc3(&c->d_mD, md, "digit-pair products");
  if (!r) r = alloc3(&c->d_meA, 2 * (size_t)N, "exponents A");
  if (!r) r = alloc3(&c->d_meB, 2 * (size_t)N, "exponents B");
  if (r) {
    bs_destroy_cell3(c);
    return r;
  }
  std::vector<double> G(3 * (size_t)N);
  for (int a = 0; a < N; ++a) {
    const int al = a / (W * W) - M, be = (a / W) % W - M, ga = a % W - M;
    for (int j = 0; j < 3; ++j)
      G[(size_t)j * N + a] = al * c->q[0][j] + be * c->q[1][j] + ga * c->q[2][j];
  }
  const std::vector<double> coef = monomial_coefficients();
  cudaError_t e = cudaMemcpy(c->d_phase, ph.data(), P3 * 2, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_tab, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->d_G, G.data(), G.size() * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(c->d_coef, coef.data(), coef.size() * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(c->d_info, 0, 4 * sizeof(int));
  if (e != cudaSuccess) {
    r = bs_cuda_status(e, "bs_create_cell3 upload");
    bs_destroy_cell3(c);
    return r;
  }
  *out = c;
  return BS_OK;
}

extern "C" int bs_assemble3(bs_cell3* c, void* stream) {
  if (!c) {
    bs_set_error("bs_assemble3: NULL cell");
    return BS_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int P = c->P, D = c->D, N = c->N, n = c->n;
  const size_t NN = (size_t)N * N, nn = (size_t)n * n;
  CK3(cudaMemsetAsync(c->d_info, 0, 2 * sizeof(int), s), "bs_assemble3");
  exp3_kernel<<<(D * P + 255) / 256, 256, 0, s>>>(P, c->M, D, c->d_E);
  BS_CHECK_LAUNCH("exp3_kernel");
  size_t tot = (size_t)3 * P * P * D;
  ff3_stage1<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(c->d_phase, c->d_tab, c->nphase, P, D,
                                                          c->d_E, c->d_Y1);
  BS_CHECK_LAUNCH("ff3_stage1");
  tot = (size_t)3 * P * D * D;
  ff3_stage2<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(c->d_Y1, P, D, c->d_E, c->d_Y2);
  BS_CHECK_LAUNCH("ff3_stage2");
  tot = (size_t)3 * D * D * D;
  ff3_stage3<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
      c->d_Y2, P, D, c->V / ((double)P * P * P), c->d_E, c->d_ghat);
  BS_CHECK_LAUNCH("ff3_stage3");
  toeplitz3_kernel<<<(unsigned)((3 * NN + 255) / 256), 256, 0, s>>>(c->d_ghat, c->M, N, D,
                                                                   c->d_T);
  BS_CHECK_LAUNCH("toeplitz3_kernel");
  TRY_LAUNCH(bs_launch_cholesky(c->d_T, N, 3, (long)NN, c->d_info, s));
  TRY_LAUNCH(bs_launch_trinv(c->d_T, c->d_Linv, N, 3, (long)NN, s));
  // F_X^a = L_R^-1 diag(s_a) L_X^-dagger for X in {h, m} (batch of 2), a = 0..3
  const zd* LinvR = c->d_Linv + 2 * NN;
  CK3(cudaMemcpyAsync(c->d_LinvR2, LinvR, NN * sizeof(zd), cudaMemcpyDeviceToDevice, s), "copy");
  CK3(cudaMemcpyAsync(c->d_LinvR2 + NN, LinvR, NN * sizeof(zd), cudaMemcpyDeviceToDevice, s),
      "copy");
  int* err = c->d_info + 1;
  for (int a = 0; a < 4; ++a) {
    const double* sc = a == 0 ? nullptr : c->d_G + (size_t)(a - 1) * N;
    TRY_LAUNCH(bs_launch_zgemm_tc(c->d_LinvR2, (long)NN, sc, c->d_Linv, (long)NN,
                                  c->d_F + (size_t)a * NN, (long)(4 * NN), N, 2, c->d_mA, c->d_mB,
                                  c->d_mD, c->d_meA, c->d_meB, err, s));
  }
  // P_X^{ab} = F_X^a F_X^b^dagger, a <= b
  int t = 0;
  for (int a = 0; a < 4; ++a)
    for (int b = a; b < 4; ++b, ++t)
      TRY_LAUNCH(bs_launch_zgemm_tc(c->d_F + (size_t)a * NN, (long)(4 * NN), nullptr,
                                    c->d_F + (size_t)b * NN, (long)(4 * NN),
                                    c->d_Pp + (size_t)t * NN, (long)(10 * NN), N, 2, c->d_mA,
                                    c->d_mB, c->d_mD, c->d_meA, c->d_meB, err, s));
  monomial3_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(c->d_Pp, c->d_coef, N,
                                                               c->V * c->V, c->d_Cm);
  BS_CHECK_LAUNCH("monomial3_kernel");
  c->assembled = true;
  return BS_OK;
}

extern "C" int bs_solve_k3(bs_cell3* c, const double* Q, int nk, int nbands, double* omega_out,
                           int* status_out, void* stream) {
  if (!c || nk < 0 || (nk > 0 && (!Q || !omega_out))) {
    bs_set_error("bs_solve_k3: NULL argument or nk < 0");
    return BS_EINVAL;
  }
  if (!c->assembled) {
    bs_set_error("bs_solve_k3: call bs_assemble3 first");
    return BS_ESTATE;
  }
  if (nbands < 1 || nbands > c->n) {
    bs_set_error("bs_solve_k3: nbands=%d outside [1, %d]", nbands, c->n);
    return BS_EINVAL;
  }
  if (nk == 0) return BS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int n = c->n;
  const bool q_dev = dev_ptr3(Q), w_dev = dev_ptr3(omega_out);
  const bool st_dev = status_out && dev_ptr3(status_out);
  // wavevectors per chunk: about 4 GB of C(k)
  const int cap = (int)std::max<size_t>(1, std::min<size_t>((size_t)nk, (4ull << 30) /
                                                            ((size_t)n * n * sizeof(zd))));
  TRY_LAUNCH(ensure_ws3(c, cap, nbands));
  std::vector<double> qv(9);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) qv[i * 3 + j] = c->q[i][j];
  double* d_qv = nullptr;
  CK3(cudaMalloc(&d_qv, 9 * sizeof(double)), "bs_solve_k3 q");
  CK3(cudaMemcpy(d_qv, qv.data(), 9 * sizeof(double), cudaMemcpyHostToDevice), "bs_solve_k3 q");
  int r = BS_OK;
  for (int k0 = 0; k0 < nk && !r; k0 += cap) {
    const int kb = std::min(cap, nk - k0);
    cudaError_t e = cudaMemcpyAsync(c->d_Q, Q + 3 * (size_t)k0, 3 * kb * sizeof(double),
                                    q_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
      r = bs_cuda_status(e, "bs_solve_k3 Q");
      break;
    }
    const size_t nn = (size_t)n * n;
    builder3_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(c->d_Cm, n, c->d_Q, kb, d_qv,
                                                                 c->d_C);
    e = cudaGetLastError();
    bs_count_launch();
    if (e != cudaSuccess) {
      r = bs_cuda_status(e, "builder3_kernel");
      break;
    }
    if (bs_use_band(n)) {
      if (!c->band) c->band = new BandWs();
      r = bs_band_ws_alloc(c->band, n, c->kcap, BS_SLICES_BAND);
      BandBisect bis{nbands, c->d_w, c->d_stat};
      if (!r) r = bs_launch_eig_band(c->d_C, n, kb, *c->band, c->d_de, c->d_info + 1, s, &bis);
    } else {
      r = bs_launch_tridiag<double>(c->d_C, n, kb, c->d_vec, c->d_part, c->d_de, c->d_tau,
                                    c->d_beta, c->d_count, s);
      if (!r) r = bs_launch_bisect(c->d_de, n, kb, nbands, c->d_w, c->d_stat, s);
    }
    if (r) break;
    e = cudaMemcpyAsync(omega_out + (size_t)k0 * nbands, c->d_w, (size_t)kb * nbands * 8,
                        w_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && status_out)
      e = cudaMemcpyAsync(status_out + k0, c->d_stat, kb * sizeof(int),
                          st_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) r = bs_cuda_status(e, "bs_solve_k3 output");
    if (!r && (!w_dev || (status_out && !st_dev))) r = check3(c, s);
  }
  cudaStreamSynchronize(s);
  cudaFree(d_qv);
  return r;
}

extern "C" int bs_form_factors3(bs_cell3* c, double* out, void* stream) {
  if (!c || !out) {
    bs_set_error("bs_form_factors3: NULL argument");
    return BS_EINVAL;
  }
  if (!c->assembled) {
    bs_set_error("bs_form_factors3: call bs_assemble3 first");
    return BS_ESTATE;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t D3 = (size_t)c->D * c->D * c->D;
  CK3(cudaMemcpyAsync(out, c->d_ghat, 3 * D3 * sizeof(zd),
                      dev_ptr3(out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s),
      "bs_form_factors3");
  CK3(cudaStreamSynchronize(s), "bs_form_factors3 sync");
  return BS_OK;
}

extern "C" int bs_reduced_matrix3(bs_cell3* c, const double* Q, double* out, void* stream) {
  if (!c || !Q || !out) {
    bs_set_error("bs_reduced_matrix3: NULL argument");
    return BS_EINVAL;
  }
  if (!c->assembled) {
    bs_set_error("bs_reduced_matrix3: call bs_assemble3 first");
    return BS_ESTATE;
  }
  cudaStream_t s = (cudaStream_t)stream;
  TRY_LAUNCH(ensure_ws3(c, 1, 1));
  std::vector<double> qv(9), Qh(3);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) qv[i * 3 + j] = c->q[i][j];
  TRY_LAUNCH(fetch3(Qh.data(), Q, 3 * sizeof(double)));
  double* d_qv = nullptr;
  CK3(cudaMalloc(&d_qv, 9 * sizeof(double)), "q");
  cudaMemcpy(d_qv, qv.data(), 9 * 8, cudaMemcpyHostToDevice);
  cudaMemcpy(c->d_Q, Qh.data(), 3 * 8, cudaMemcpyHostToDevice);
  const size_t nn = (size_t)c->n * c->n;
  builder3_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(c->d_Cm, c->n, c->d_Q, 1, d_qv,
                                                               c->d_C);
  bs_count_launch();
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, c->d_C, nn * sizeof(zd),
                        dev_ptr3(out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  cudaFree(d_qv);
  if (e != cudaSuccess) return bs_cuda_status(e, "bs_reduced_matrix3");
  return check3(c, s);
}

extern "C" int bs_cell3_dims(const bs_cell3* c, int* N, int* n) {
  if (!c) {
    bs_set_error("bs_cell3_dims: NULL cell");
    return BS_EINVAL;
  }
  if (N) *N = c->N;
  if (n) *n = c->n;
  return BS_OK;
}
