// A general in-plane stiffness per phase: the full compliance Gram matrix of
// Eq. (ep).  With the Voigt compliance S = C^-1 of each phase (strain
// (e11, e22, 2 e12) = S (s11, s22, s12)), the paper's Phi entries with their
// factors 2 and 4 are exactly the Toeplitz blocks of the Voigt entries,
//   Phi = [T[S11] T[S12] T[S13]; T[S12] T[S22] T[S23]; T[S13] T[S23] T[S33]],
// which is no longer block diagonal in any stress basis.  So the isotropic
// shortcut is replaced by one Cholesky factor Phi = L L^dagger of the
// 3N x 3N matrix, Z = L^-dagger (Phi^-1 = Z Z^dagger), and
//   W(k) = L_Omega^-1 H(k) Z = k1 W1 + k2 W2 + W0,
// H(k) = i V [diag K1, 0, diag K2; 0, diag K2, diag K1] (Eq. (eh)), so that
//   W1 = A_R [Z1; Z3],  W2 = A_R [Z3; Z2],
//   W0 = A_R [G1 Z1 + G2 Z3; G2 Z2 + G1 Z3]     (rows r of Z: Z_r, diag G scaling)
// with A_R = L_R^-1 (V applied with the monomials; L_R^-1 I1 on a mesh), and
//   C(k) = W W^dagger = sum over a <= b of k_a k_b (W_a W_b^dagger + h.c.),
// the same six k-monomials as the isotropic path (k_0 = 1).  The products
// (18 N^3 complex multiply-adds for the W_i and 72 N^3 for the monomials,
// once per cell) run as exact-slice tensor-core contractions, FP64-accurate
// like the isotropic path's, while 6N <= 4096; beyond that as FP64 complex
// GEMMs on the CUDA cores.
#include "bs_internal.h"

namespace {

// Voigt entry (r, c) -> material field index of the table (S11, S22, rho, S12, S13, S23, S33)
__device__ __forceinline__ int voigt_field(int r, int c) {
  const int lo = r < c ? r : c, hi = r < c ? c : r;
  if (lo == hi) return lo == 0 ? 0 : lo == 1 ? 1 : 6;
  return lo == 0 ? (hi == 1 ? 3 : 4) : 5;
}

// Phi[(rN + a) + (cN + b) 3N] = T_f(a, b), f = voigt_field(r, c)
__global__ void phi_build_kernel(const zd* __restrict__ T, int N, zd* __restrict__ Phi) {
  const size_t n3 = 3 * (size_t)N, NN = (size_t)N * N;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n3 * n3) return;
  const int R = (int)(i % n3), C = (int)(i / n3);
  const int r = R / N, a = R % N, c = C / N, b = C % N;
  Phi[i] = T[(size_t)voigt_field(r, c) * NN + a + (size_t)b * N];
}

// Yw[t] (2N x 3N, column-major, ld 2N) = rows of H_t Z / (i V), Z = L^-dagger:
// Z(r', c) = conj(L^-1(c, r')); with trans set, Yw[t]^dagger instead (3N x 2N,
// ld 3N), the B operand of the tensor-core products
__global__ void yw_kernel(const zd* __restrict__ LPhi, const double* __restrict__ G, int N,
                          int trans, zd* __restrict__ Yw) {
  const size_t n2 = 2 * (size_t)N, n3 = 3 * (size_t)N;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n2 * n3) return;
  const int t = blockIdx.y;
  const int rho = (int)(i % n2), c = (int)(i / n2);
  auto Z = [&](int rr) { return zconj(LPhi[(size_t)c + (size_t)rr * n3]); };
  const bool top = rho < N;
  const int a = top ? rho : rho - N;
  zd v;
  if (t == 1) {
    v = Z(top ? a : 2 * N + a);
  } else if (t == 2) {
    v = Z(top ? 2 * N + a : N + a);
  } else {
    const double g1 = G[a], g2 = G[N + a];
    v = top ? zadd(zscale(Z(a), g1), zscale(Z(2 * N + a), g2))
            : zadd(zscale(Z(N + a), g2), zscale(Z(2 * N + a), g1));
  }
  if (trans)
    Yw[(size_t)t * n2 * n3 + (size_t)c + (size_t)rho * n3] = zconj(v);
  else
    Yw[(size_t)t * n2 * n3 + i] = v;
}

// Cm[t] = V2 (P_ab + P_ab^dagger) (a < b) or V2 P_aa, monomials 1, k1, k2, k1^2, k1 k2, k2^2
__global__ void cm_aniso_kernel(const zd* __restrict__ Pab, int n, double V2,
                                zd* __restrict__ Cm) {
  const size_t nn = (size_t)n * n;
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nn) return;
  const int r = (int)(e % n), c = (int)(e / n);
  const size_t et = (size_t)c + (size_t)r * n;
  // products in the order (0,0), (0,1), (0,2), (1,1), (1,2), (2,2)
  const bool sym[6] = {false, true, true, false, true, false};
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    const zd* P = Pab + (size_t)t * nn;
    zd v = P[e];
    if (sym[t]) v = zadd(v, zconj(P[et]));
    Cm[(size_t)t * nn + e] = zscale(v, V2);
  }
}

// R3[:, j] = [K1 u1; K2 u2; K2 u1 + K1 u2] of column j = (k, v)
__global__ void stress_rhs3_kernel(const zd* __restrict__ U, const double* __restrict__ Q,
                                   const double* __restrict__ Gv, int N, int nvec, int m,
                                   double q1x, double q1y, double q2x, double q2y,
                                   zd* __restrict__ R3) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)N * m) return;
  const int a = (int)(i % N);
  const int j = (int)(i / N);
  const int k = j / nvec;
  const double Q1 = Q[2 * k], Q2 = Q[2 * k + 1];
  const double K1 = Q1 * q1x + Q2 * q2x + Gv[a];
  const double K2 = Q1 * q1y + Q2 * q2y + Gv[N + a];
  const zd u1 = U[(size_t)j * 2 * N + a], u2 = U[(size_t)j * 2 * N + N + a];
  zd* r = R3 + (size_t)j * 3 * N;
  r[a] = zscale(u1, K1);
  r[N + a] = zscale(u2, K2);
  r[2 * N + a] = zadd(zscale(u1, K2), zscale(u2, K1));
}

// S = i vs X
__global__ void scale_i_kernel(const zd* __restrict__ X, size_t cnt, double vs,
                               zd* __restrict__ S) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cnt) return;
  const zd x = X[i];
  S[i] = zmake(-vs * x.y, vs * x.x);
}

}  // namespace

int bs_launch_gram_aniso(bs_cell* c, cudaStream_t s) {
  const int N = c->N;
  const size_t NN = (size_t)N * N, n3 = 3 * (size_t)N;
  // R = T[rho] (slot 2): Cholesky in place and its inverse, where the isotropic path keeps them
  TRY_LAUNCH(bs_launch_cholesky(c->d_T + 2 * NN, N, 1, (long)NN, c->d_info, s));
  TRY_LAUNCH(bs_launch_trinv(c->d_T + 2 * NN, c->d_Linv + 2 * NN, N, 1, (long)NN, s));
  phi_build_kernel<<<(unsigned)((n3 * n3 + 255) / 256), 256, 0, s>>>(c->d_T, N, c->d_Phi);
  BS_CHECK_LAUNCH("phi_build_kernel");
  TRY_LAUNCH(bs_launch_cholesky(c->d_Phi, 3 * N, 1, (long)(n3 * n3), c->d_info, s));
  TRY_LAUNCH(bs_launch_trinv(c->d_Phi, c->d_LPhi, 3 * N, 1, (long)(n3 * n3), s));
  return BS_OK;
}

int bs_launch_monomials_aniso(bs_cell* c, cudaStream_t s) {
  const int N = c->N, n = 2 * N;
  const size_t NN = (size_t)N * N, n2n3 = (size_t)n * 3 * N, nn = (size_t)n * n;
  const zd one = zmake(1.0, 0.0);
  const zd* LinvR = c->d_Linv + 2 * NN;
  int* err = c->d_info + 1;
  // A_R = L_R^-1 (pixel grid) or L_R^-1 I1 (mesh; I1 is Hermitian)
  const zd* AR = LinvR;
  if (c->mesh) {
    TRY_LAUNCH(bs_launch_zgemm_tc(LinvR, 0, nullptr, c->d_I1, 0, c->d_LinvR2, (long)NN, N, 1,
                                  c->d_mA, c->d_mB, c->d_mD, c->d_meA, c->d_meB, err, s));
    AR = c->d_LinvR2;
  }
  const bool tc = bs_zgemm_tc_fits(3 * N);
  yw_kernel<<<dim3((unsigned)((n2n3 + 255) / 256), 3), 256, 0, s>>>(c->d_LPhi, c->d_G, N,
                                                                   tc ? 1 : 0, c->d_Yw);
  BS_CHECK_LAUNCH("yw_kernel");
  // W_t = diag(A_R, A_R) Yw_t: the top and bottom halves as a batch of two
  // (on the tensor cores B = Yw_t^dagger, halves 3N x N apart)
  for (int t = 0; t < 3; ++t) {
    if (tc)
      TRY_LAUNCH(bs_launch_zgemm_tc_rect(AR, N, 0, nullptr, c->d_Yw + t * n2n3, 3 * N,
                                         (long)(3 * NN), c->d_Wk + t * n2n3, n, N, N, 3 * N, N, 2,
                                         c->d_mA, c->d_mB, c->d_mD, c->d_meA, c->d_meB, err, s));
    else
      TRY_LAUNCH(bs_launch_zgemm(false, false, N, 3 * N, N, one, AR, N, 0, c->d_Yw + t * n2n3, n,
                                 N, nullptr, 0, c->d_Wk + t * n2n3, n, N, 2, c->mesh ? 0 : 1, s));
  }
  const int pa[6] = {0, 0, 0, 1, 1, 2}, pb[6] = {0, 1, 2, 1, 2, 2};
  for (int t = 0; t < 6; ++t) {
    if (tc)
      TRY_LAUNCH(bs_launch_zgemm_tc_rect(c->d_Wk + pa[t] * n2n3, n, 0, nullptr,
                                         c->d_Wk + pb[t] * n2n3, n, 0, c->d_Pab + t * nn, n, 0, n,
                                         n, 3 * N, 1, c->d_mA, c->d_mB, c->d_mD, c->d_meA,
                                         c->d_meB, err, s));
    else
      TRY_LAUNCH(bs_launch_zgemm(false, true, n, n, 3 * N, one, c->d_Wk + pa[t] * n2n3, n, 0,
                                 c->d_Wk + pb[t] * n2n3, n, 0, nullptr, 0, c->d_Pab + t * nn, n,
                                 0, 1, 0, s));
  }
  const double V2 = c->mesh ? 1.0 : c->V * c->V;
  cm_aniso_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(c->d_Pab, n, V2, c->d_Cm);
  BS_CHECK_LAUNCH("cm_aniso_kernel");
  return BS_OK;
}

// S = -Phi^-1 H^* U = i vs L^-dagger L^-1 [K1 u1; K2 u2; K2 u1 + K1 u2] (vs = V, or 1 on a
// mesh where U already holds I1 U); R3 and Y3 hold 3N x (kc nvec) each
int bs_launch_stress_aniso(bs_cell* c, const zd* U, const double* Q, int kc, int nvec, zd* R3,
                           zd* Y3, zd* S, cudaStream_t s) {
  const int N = c->N, m = kc * nvec;
  const size_t tot = (size_t)N * m;
  const zd one = zmake(1.0, 0.0);
  stress_rhs3_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
      U, Q, c->d_G, N, nvec, m, c->q1[0], c->q1[1], c->q2[0], c->q2[1], R3);
  BS_CHECK_LAUNCH("stress_rhs3_kernel");
  TRY_LAUNCH(bs_launch_zgemm(false, false, 3 * N, m, 3 * N, one, c->d_LPhi, 3 * N, 0, R3, 3 * N,
                             0, nullptr, 0, Y3, 3 * N, 0, 1, 1, s));
  TRY_LAUNCH(bs_launch_zgemm(true, false, 3 * N, m, 3 * N, one, c->d_LPhi, 3 * N, 0, Y3, 3 * N,
                             0, nullptr, 0, R3, 3 * N, 0, 1, 4, s));
  const size_t cnt = 3 * tot;
  scale_i_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(R3, cnt, c->mesh ? 1.0 : c->V, S);
  BS_CHECK_LAUNCH("scale_i_kernel");
  return BS_OK;
}
