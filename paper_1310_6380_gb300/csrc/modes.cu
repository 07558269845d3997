// Mode shapes: the stress coefficients of a Bloch mode and the fields of a
// plane-wave expansion on a grid of the unit cell.
//
// Stress (second block row of Eq. (equationshomogeneousMatrix), Phi S + H^* U = 0):
// with H = i V [diag K1, 0, diag K2; 0, diag K2, diag K1] (Eq. (eh) on the pixel
// grid, where int conj(f_a) f_b = V delta_ab) and the isotropic Phi of Eq. (ep),
// which in the rotated stress basis (S11 +- S22)/sqrt2, S12 is
// diag(T_k/2, T_m/2, T_m) (T_k = T[1/(lam+mu)], T_m = T[1/mu]),
//   S11 = i V [T_k^-1 (K1 u1 + K2 u2) + T_m^-1 (K1 u1 - K2 u2)]
//   S22 = i V [T_k^-1 (K1 u1 + K2 u2) - T_m^-1 (K1 u1 - K2 u2)]
//   S12 = i V  T_m^-1 (K2 u1 + K1 u2),
// where T_X^-1 = L_X^-dagger L_X^-1 uses the triangular inverses that the
// assembly keeps.  On a mesh cell the centroid rule does not make the plane
// waves orthogonal, H = i I1 diag(K) with I1 = int conj(f_a) f_b, and V u
// becomes I1 u in the right-hand sides.  All of it is FP64: two complex products per Gram solve,
// every (k, mode) a column of one batched product.
//
// Fields (Eq. (approximation2d)): F(x_pq) = sum_a c_a exp(i K_a . x_pq) at
// x_pq = ((p + 1/2)/G) h1 + ((q + 1/2)/G) h2.  With K_a = (Q1 + alpha) q^1 +
// (Q2 + beta) q^2 and q^i . h^j = 2 pi delta_ij the phase separates, so
//   F[p][q] = sum_alpha Ep[alpha][p] sum_beta c[alpha][beta] Eq[beta][q],
//   Ep[alpha][p] = exp(i pi (Q1 + alpha)(2p + 1)/G), Eq likewise with Q2, beta.
// The angles are reduced exactly in integers and evaluated in FP64; the two
// contractions run in FP32 (the output is complex64).  Each CTA owns one
// field: every thread keeps the column T[.][q] of the first contraction in
// registers, so the second streams rows p with shared-memory broadcasts of
// Ep and coalesced stores along q.  The kernel is bound by its stores and
// the FP32 pipe, not by any read.
#include <algorithm>
#include <vector>

#include "bs_internal.h"

namespace {

constexpr int FT = 256;   // most threads of a field CTA
constexpr int PB = 16;    // rows of Ep staged per shared-memory pass (a multiple of 4)

// E[k][0][a][p] = exp(i pi (Q1 + a - M)(2p + 1)/G), E[k][1][a][q] likewise with Q2;
// rows a >= 2M + 1 up to WP are zero (the padding of the unrolled contractions)
__global__ void field_table_kernel(const double* __restrict__ Q, int nk, int M, int WP, int G,
                                   zf* __restrict__ E) {
  const size_t tot = (size_t)nk * 2 * WP * G;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= tot) return;
  const int p = (int)(i % G);
  const int a = (int)((i / G) % WP);
  const int dir = (int)((i / ((size_t)G * WP)) % 2);
  const int k = (int)(i / ((size_t)G * WP * 2));
  if (a >= 2 * M + 1) {
    E[i] = make_float2(0.f, 0.f);
    return;
  }
  const long long al = a - M, odd = 2LL * p + 1, twoG = 2LL * G;
  long long m = (al * odd) % twoG;
  if (m < 0) m += twoG;
  double x = fmod(Q[2 * k + dir] * (double)odd / (double)G, 2.0);
  x += (double)m / (double)G;
  double s, c;
  sincospi(x, &s, &c);
  E[i] = make_float2((float)c, (float)s);
}

// out[j][p][q] for field j of the chunk, global field f0 + j of wavevector
// (f0 + j) / fpk; the table holds wavevectors kbase, kbase + 1, ...
// WP >= 2M + 1, WP % 4 == 0; rows of four outputs per thread for independent chains
template <int WP>
__global__ void __launch_bounds__(FT, 2)
field_kernel(const zd* __restrict__ coef, int M, int N, int G, long f0, int fpk, long kbase,
             const zf* __restrict__ E, zf* __restrict__ out) {
  __shared__ __align__(16) zf Ct[WP * WP];     // Ct[b][a] = c[a][b]
  __shared__ __align__(16) zf Es[PB][WP];
  const long f = f0 + blockIdx.x;
  const long k = f / fpk - kbase;
  const int W = 2 * M + 1;
  const int tid = threadIdx.x;
  const zd* c = coef + (size_t)blockIdx.x * N;
  for (int e = tid; e < WP * WP; e += blockDim.x) {
    const int b = e / WP, a = e % WP;
    zf v = make_float2(0.f, 0.f);
    if (a < W && b < W) {
      const zd x = c[a * W + b];
      v = make_float2((float)x.x, (float)x.y);
    }
    Ct[e] = v;
  }
  const zf* Ep = E + (size_t)k * 2 * WP * G;
  const zf* Eq = Ep + (size_t)WP * G;
  zf* o = out + (size_t)blockIdx.x * G * G;
  for (int q0 = 0; q0 < G; q0 += blockDim.x) {
    const int q = q0 + tid;
    const bool act = q < G;
    __syncthreads();   // Ct written; Es of the previous chunk consumed
    // first contraction: T[a] = sum_b c[a][b] Eq[b][q], kept in registers
    zf T[WP];
#pragma unroll
    for (int a = 0; a < WP; ++a) T[a] = make_float2(0.f, 0.f);
#pragma unroll
    for (int b = 0; b < WP; ++b) {
      const zf eb = act ? Eq[(size_t)b * G + q] : make_float2(0.f, 0.f);
      const float4* c4 = reinterpret_cast<const float4*>(&Ct[b * WP]);
#pragma unroll
      for (int a = 0; a < WP; a += 2) {
        const float4 v = c4[a / 2];
        T[a] = zfma(make_float2(v.x, v.y), eb, T[a]);
        T[a + 1] = zfma(make_float2(v.z, v.w), eb, T[a + 1]);
      }
    }
    // second contraction, PB rows per staging pass, four rows at a time
    for (int p0 = 0; p0 < G; p0 += PB) {
      __syncthreads();
      for (int e = tid; e < PB * WP; e += blockDim.x) {
        const int r = e / WP, a = e % WP;
        Es[r][a] = p0 + r < G ? Ep[(size_t)a * G + p0 + r] : make_float2(0.f, 0.f);
      }
      __syncthreads();
      if (act) {
        const int rows = min(PB, G - p0);
#pragma unroll
        for (int r = 0; r < PB; r += 4) {
          zf acc[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) acc[i] = make_float2(0.f, 0.f);
#pragma unroll
          for (int a = 0; a < WP; a += 2) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const float4 v = reinterpret_cast<const float4*>(&Es[r + i][0])[a / 2];
              acc[i] = zfma(make_float2(v.x, v.y), T[a], acc[i]);
              acc[i] = zfma(make_float2(v.z, v.w), T[a + 1], acc[i]);
            }
          }
#pragma unroll
          for (int i = 0; i < 4; ++i)
            if (r + i < rows) o[(size_t)(p0 + r + i) * G + q] = acc[i];
        }
      }
    }
  }
}

// Right-hand sides of the Gram solves for columns j = (k, v), j < m:
// Zk[:, j] = K1 u1 + K2 u2,  Zm[:, j] = K1 u1 - K2 u2,  Zm[:, m + j] = K2 u1 + K1 u2
__global__ void stress_rhs_kernel(const zd* __restrict__ U, const double* __restrict__ Q,
                                  const double* __restrict__ Gv, int N, int nvec, int m,
                                  double q1x, double q1y, double q2x, double q2y,
                                  zd* __restrict__ Zk, zd* __restrict__ Zm) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)N * m) return;
  const int a = (int)(i % N);
  const int j = (int)(i / N);
  const int k = j / nvec;
  const double Q1 = Q[2 * k], Q2 = Q[2 * k + 1];
  const double K1 = Q1 * q1x + Q2 * q2x + Gv[a];
  const double K2 = Q1 * q1y + Q2 * q2y + Gv[N + a];
  const zd u1 = U[(size_t)j * 2 * N + a], u2 = U[(size_t)j * 2 * N + N + a];
  const zd t1 = zscale(u1, K1), t2 = zscale(u2, K2);
  Zk[i] = zadd(t1, t2);
  Zm[i] = zsub(t1, t2);
  Zm[(size_t)m * N + i] = zadd(zscale(u1, K2), zscale(u2, K1));
}

// S[j] = i V (Xk + Xm, Xk - Xm, X12) for column j
__global__ void stress_combine_kernel(const zd* __restrict__ Xk, const zd* __restrict__ Xm,
                                      int N, int m, double V, zd* __restrict__ S) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)N * m) return;
  const int a = (int)(i % N);
  const int j = (int)(i / N);
  const zd xk = Xk[i], xm = Xm[i], x12 = Xm[(size_t)m * N + i];
  const zd p = zadd(xk, xm), d = zsub(xk, xm);
  zd* s = S + (size_t)j * 3 * N;
  s[a] = zmake(-V * p.y, V * p.x);
  s[N + a] = zmake(-V * d.y, V * d.x);
  s[2 * N + a] = zmake(-V * x12.y, V * x12.x);
}

bool dev_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

#define MCK(call, where)                                         \
  do {                                                           \
    cudaError_t e__ = (call);                                    \
    if (e__ != cudaSuccess) return bs_cuda_status(e__, where);   \
  } while (0)

// grow the cell's mode workspace to `bytes`
int mode_ws(bs_cell* c, size_t bytes) {
  if (c->mode_cap >= bytes) return BS_OK;
  if (c->d_mode) {
    cudaDeviceSynchronize();
    cudaFree(c->d_mode);
    c->d_mode = nullptr;
    c->mode_cap = 0;
  }
  cudaError_t e = cudaMalloc(&c->d_mode, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->d_mode = nullptr;
    bs_set_error("mode workspace: cudaMalloc of %zu bytes failed", bytes);
    return BS_ENOMEM;
  }
  c->mode_cap = bytes;
  return BS_OK;
}

template <int WP>
int launch_field(const zd* coef, long nf, int M, int N, int G, long f0, int fpk, long kbase,
                 const zf* E, zf* out, cudaStream_t s) {
  const int chunks = (G + FT - 1) / FT;
  const int per = (G + chunks - 1) / chunks;
  const int threads = std::min(FT, (per + 31) / 32 * 32);
  field_kernel<WP><<<(unsigned)nf, threads, 0, s>>>(coef, M, N, G, f0, fpk, kbase, E, out);
  BS_CHECK_LAUNCH("field_kernel");
  return BS_OK;
}

}  // namespace

void bs_free_mode_workspace(bs_cell* c) {
  if (c->d_mode) cudaFree(c->d_mode);
  c->d_mode = nullptr;
  c->mode_cap = 0;
}

// fields f0 .. f0 + nf - 1 (fpk per wavevector) of coefficients `coef` (the
// chunk's first field) into `out`; Q holds the wavevectors kbase .. kbase + nkt - 1
int bs_launch_mode_field(const zd* coef, const double* Q, long kbase, int nkt, long f0, long nf,
                         int fpk, int M, int G, zf* E, zf* out, cudaStream_t s) {
  const int W = 2 * M + 1, WP = (W + 3) / 4 * 4, N = W * W;
  const size_t te = (size_t)nkt * 2 * WP * G;
  field_table_kernel<<<(unsigned)((te + 255) / 256), 256, 0, s>>>(Q + 2 * kbase, nkt, M, WP, G, E);
  BS_CHECK_LAUNCH("field_table_kernel");
  switch (WP) {
    case 4: return launch_field<4>(coef, nf, M, N, G, f0, fpk, kbase, E, out, s);
    case 8: return launch_field<8>(coef, nf, M, N, G, f0, fpk, kbase, E, out, s);
    case 12: return launch_field<12>(coef, nf, M, N, G, f0, fpk, kbase, E, out, s);
    case 16: return launch_field<16>(coef, nf, M, N, G, f0, fpk, kbase, E, out, s);
    case 20: return launch_field<20>(coef, nf, M, N, G, f0, fpk, kbase, E, out, s);
    case 24: return launch_field<24>(coef, nf, M, N, G, f0, fpk, kbase, E, out, s);
    case 28: return launch_field<28>(coef, nf, M, N, G, f0, fpk, kbase, E, out, s);
    case 32: return launch_field<32>(coef, nf, M, N, G, f0, fpk, kbase, E, out, s);
  }
  bs_set_error("mode field: truncation M = %d outside [0, 15]", M);
  return BS_EINVAL;
}

int bs_launch_stress(bs_cell* c, const zd* U, const double* Q, int kc, int nvec, zd* Zk, zd* Zm,
                     zd* Y, zd* S, cudaStream_t s) {
  const int N = c->N, m = kc * nvec;
  const size_t NN = (size_t)N * N, tot = (size_t)N * m;
  const zd one = zmake(1.0, 0.0);
  // on a mesh H^* U needs I1 U (I1 = V I on a pixel grid, where V is applied at the end)
  const zd* Uin = U;
  if (c->mesh) {
    TRY_LAUNCH(bs_launch_zgemm(false, false, N, 2 * m, N, one, c->d_I1, N, 0, U, N, 0, nullptr, 0,
                               Y, N, 0, 1, 0, s));
    Uin = Y;
  }
  stress_rhs_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
      Uin, Q, c->d_G, N, nvec, m, c->q1[0], c->q1[1], c->q2[0], c->q2[1], Zk, Zm);
  BS_CHECK_LAUNCH("stress_rhs_kernel");
  const zd* Lk = c->d_Linv;
  const zd* Lm = c->d_Linv + NN;
  // T_k^-1 Zk = L_k^-dagger (L_k^-1 Zk): Y = L^-1 Z (lower), then Zk = L^-dagger Y
  TRY_LAUNCH(bs_launch_zgemm(false, false, N, m, N, one, Lk, N, 0, Zk, N, 0, nullptr, 0, Y, N, 0,
                             1, 1, s));
  TRY_LAUNCH(bs_launch_zgemm(true, false, N, m, N, one, Lk, N, 0, Y, N, 0, nullptr, 0, Zk, N, 0,
                             1, 4, s));
  TRY_LAUNCH(bs_launch_zgemm(false, false, N, 2 * m, N, one, Lm, N, 0, Zm, N, 0, nullptr, 0, Y,
                             N, 0, 1, 1, s));
  TRY_LAUNCH(bs_launch_zgemm(true, false, N, 2 * m, N, one, Lm, N, 0, Y, N, 0, nullptr, 0, Zm, N,
                             0, 1, 4, s));
  stress_combine_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(Zk, Zm, N, m,
                                                                     c->mesh ? 1.0 : c->V, S);
  BS_CHECK_LAUNCH("stress_combine_kernel");
  return BS_OK;
}

extern "C" int bs_stress_coefficients(bs_cell* c, const double* Q, int nk, int nvec,
                                      const double* U, double* S_out, void* stream) {
  if (!c || nk < 0 || nvec < 1 || nvec > 16384 || (nk > 0 && (!Q || !U || !S_out))) {
    bs_set_error("bs_stress_coefficients: NULL argument, nk < 0 or nvec outside [1, 16384]");
    return BS_EINVAL;
  }
  if (!c->assembled) {
    bs_set_error("bs_stress_coefficients: call bs_assemble first");
    return BS_ESTATE;
  }
  if (nk == 0) return BS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int N = c->N;
  const bool u_dev = dev_ptr(U), s_dev = dev_ptr(S_out), q_dev = dev_ptr(Q);
  // columns per chunk: whole wavevectors, each N x m block about 2^21 complex
  // entries (eleven such blocks, ~350 MB) and m <= 16384 (the product's grid)
  long kcl = std::min<long>((1L << 21) / ((long)N * nvec), 16384 / nvec);
  const int kc = (int)std::max<long>(1, std::min<long>(nk, kcl));
  const size_t m = (size_t)kc * nvec;
  const size_t zq = 2 * (size_t)kc, zu = 2 * (size_t)N * m, zs = 3 * (size_t)N * m;
  const size_t need = (zq + 2 * (6 * (size_t)N * m + zu + zs)) * sizeof(double);
  TRY_LAUNCH(mode_ws(c, need));
  double* dQ = c->d_mode;
  zd* Zk = (zd*)(dQ + zq);             // Zk, Zm: 3 N m contiguous (R3 of the anisotropic path)
  zd* Zm = Zk + (size_t)N * m;
  zd* Y = Zm + 2 * (size_t)N * m;      // 3 N m
  zd* dU = Y + 3 * (size_t)N * m;
  zd* dS = dU + (size_t)2 * N * m;
  for (int k0 = 0; k0 < nk; k0 += kc) {
    const int kb = std::min(kc, nk - k0);
    const size_t mb = (size_t)kb * nvec;
    MCK(cudaMemcpyAsync(dQ, Q + 2 * (size_t)k0, 2 * kb * sizeof(double),
                        q_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s),
        "bs_stress_coefficients Q");
    const zd* uk = (const zd*)U + (size_t)k0 * nvec * 2 * N;
    if (!u_dev) {
      MCK(cudaMemcpyAsync(dU, uk, mb * 2 * N * sizeof(zd), cudaMemcpyHostToDevice, s),
          "bs_stress_coefficients U");
      uk = dU;
    }
    zd* sk = s_dev ? (zd*)S_out + (size_t)k0 * nvec * 3 * N : dS;
    if (c->aniso) {
      const zd* ui = uk;
      if (c->mesh) {   // I1 U first (U as an N x 2 kb nvec matrix)
        TRY_LAUNCH(bs_launch_zgemm(false, false, N, 2 * (int)mb, N, zmake(1.0, 0.0), c->d_I1, N,
                                   0, uk, N, 0, nullptr, 0, Y, N, 0, 1, 0, s));
        ui = Y;
      }
      TRY_LAUNCH(bs_launch_stress_aniso(c, ui, dQ, kb, nvec, Zk, Y, sk, s));
    } else {
      TRY_LAUNCH(bs_launch_stress(c, uk, dQ, kb, nvec, Zk, Zm, Y, sk, s));
    }
    if (!s_dev)
      MCK(cudaMemcpyAsync((zd*)S_out + (size_t)k0 * nvec * 3 * N, dS, mb * 3 * N * sizeof(zd),
                          cudaMemcpyDeviceToHost, s),
          "bs_stress_coefficients S");
    if (!u_dev || !s_dev) MCK(cudaStreamSynchronize(s), "bs_stress_coefficients sync");
  }
  return BS_OK;
}

extern "C" int bs_mode_field(bs_cell* c, const double* Q, int nk, int nfield, const double* coef,
                             int G, float* out, void* stream) {
  if (!c || nk < 0 || nfield < 1 || G < 1 || G > 8192 ||
      (nk > 0 && (!Q || !coef || !out))) {
    bs_set_error("bs_mode_field: NULL argument, nk < 0, nfield < 1 or G outside [1, 8192]");
    return BS_EINVAL;
  }
  if (nk == 0) return BS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int N = c->N, M = c->M, W = 2 * M + 1, WP = (W + 3) / 4 * 4;
  const bool c_dev = dev_ptr(coef), o_dev = dev_ptr(out), q_dev = dev_ptr(Q);
  const long nf_all = (long)nk * nfield;
  const size_t gg = (size_t)G * G;
  // fields per chunk: about 256 MB of staged complex64 outputs when `out` is
  // host memory, 256 MB of staged coefficients when `coef` is, and a
  // phase table of at most 2^25 entries
  long fc = std::min<long>(nf_all, 1L << 30);
  if (!o_dev) fc = std::max<long>(1, std::min<long>(fc, (long)((32u << 20) / gg)));
  if (!c_dev) fc = std::max<long>(1, std::min<long>(fc, (long)((16u << 20) / N)));
  const long kt_max = std::max<long>(1, (long)((1u << 25) / (2 * (size_t)WP * G)));
  fc = std::max<long>(1, std::min<long>(fc, (kt_max - 1) * nfield));
  if (fc < 1) fc = 1;
  const long kt_cap = (fc + nfield - 1) / nfield + 1;      // wavevectors a chunk can span
  const size_t tq = 2 * (size_t)nk, te = (size_t)kt_cap * 2 * WP * G;
  const size_t tc = c_dev ? 0 : (size_t)fc * N, to = o_dev ? 0 : (size_t)fc * gg;
  const size_t need = tq * 8 + (te + 1) * 8 + tc * 16 + to * 8;
  TRY_LAUNCH(mode_ws(c, need));
  double* dQ = c->d_mode;
  zf* E = (zf*)(dQ + tq);
  zd* dC = (zd*)(E + te + (te & 1));
  zf* dO = (zf*)(dC + tc);
  MCK(cudaMemcpyAsync(dQ, Q, 2 * (size_t)nk * sizeof(double),
                      q_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s),
      "bs_mode_field Q");
  for (long f0 = 0; f0 < nf_all; f0 += fc) {
    const long nf = std::min(fc, nf_all - f0);
    const long kbase = f0 / nfield, klast = (f0 + nf - 1) / nfield;
    const zd* ck = (const zd*)coef + (size_t)f0 * N;
    if (!c_dev) {
      MCK(cudaMemcpyAsync(dC, ck, (size_t)nf * N * sizeof(zd), cudaMemcpyHostToDevice, s),
          "bs_mode_field coefficients");
      ck = dC;
    }
    zf* ok = o_dev ? (zf*)out + (size_t)f0 * gg : dO;
    TRY_LAUNCH(bs_launch_mode_field(ck, dQ, kbase, (int)(klast - kbase + 1), f0, nf, nfield, M, G,
                                    E, ok, s));
    if (!o_dev)
      MCK(cudaMemcpyAsync((zf*)out + (size_t)f0 * gg, dO, (size_t)nf * gg * sizeof(zf),
                          cudaMemcpyDeviceToHost, s),
          "bs_mode_field out");
    if (!c_dev || !o_dev) MCK(cudaStreamSynchronize(s), "bs_mode_field sync");
  }
  return BS_OK;
}
