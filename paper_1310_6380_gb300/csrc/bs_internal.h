// Internal declarations of libbs: the cell object, complex helpers and the
// kernel launchers shared by the translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "bandstructure.h"

// ------------------------------------------------------------------ complex
typedef double2 zd;   // complex double (re, im)
typedef float2 zf;    // complex float

__host__ __device__ __forceinline__ zd zmake(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ zd zadd(zd a, zd b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ zd zsub(zd a, zd b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ zd zconj(zd a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ zd zscale(zd a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ zd zmul(zd a, zd b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc + a * b
__host__ __device__ __forceinline__ zd zfma(zd a, zd b, zd acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
// acc + a * conj(b)
__host__ __device__ __forceinline__ zd zfmac(zd a, zd b, zd acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.y, b.x, acc.y);
  acc.y = fma(-a.x, b.y, acc.y);
  return acc;
}
// acc - a * b
__host__ __device__ __forceinline__ zd zfnma(zd a, zd b, zd acc) {
  acc.x = fma(-a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(-a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
  return acc;
}
// acc - a * conj(b)
__host__ __device__ __forceinline__ zd zfnmac(zd a, zd b, zd acc) {
  acc.x = fma(-a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(-a.y, b.x, acc.y);
  acc.y = fma(a.x, b.y, acc.y);
  return acc;
}

// float2 versions (FP32 reduction of the mixed path)
__host__ __device__ __forceinline__ zf zadd(zf a, zf b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ zf zsub(zf a, zf b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ zf zconj(zf a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ zf zscale(zf a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ zf zmul(zf a, zf b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ zf zfma(zf a, zf b, zf acc) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
  return acc;
}
__host__ __device__ __forceinline__ zf zfnmac(zf a, zf b, zf acc) {
  acc.x = fmaf(-a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(-a.y, b.x, acc.y);
  acc.y = fmaf(a.x, b.y, acc.y);
  return acc;
}

// complex type of a real precision
template <typename R> struct Cplx;
template <> struct Cplx<double> {
  typedef double2 T;
  static __host__ __device__ __forceinline__ T make(double a, double b) { return make_double2(a, b); }
};
template <> struct Cplx<float> {
  typedef float2 T;
  static __host__ __device__ __forceinline__ T make(float a, float b) { return make_float2(a, b); }
};

// phase indices of bs_phase_times
// PH_ASM_TC: the first-stage form-factor contraction on the tensor cores
// alone (inside PH_ASM)
enum { PH_ASM = 0, PH_GRAM = 1, PH_MONO = 2, PH_BUILD = 3, PH_TRID = 4, PH_BISECT = 5,
       PH_REFINE = 6, PH_ASM_TC = 7, PH_COUNT = 8 };
// number of SMs of the current device (queried once per device)
int bs_sm_count();

// ------------------------------------------------------------------ cell
struct LobState;

struct bs_cell {
  // geometry and truncation
  int P, M, N, n, D, nphase, precision;
  double h1[2], h2[2], q1[2], q2[2], V;
  bool assembled;

  // inputs (device copies)
  uint16_t* d_phase;   // P*P pixel phases, or nel element phases of a mesh
  bool mesh;           // subdomains are mesh elements (bs_create_cell_mesh)
  int nel;             // subdomains: P*P pixels or mesh elements
  double* d_cen;       // mesh: nel x 2 fractional centroids
  double* d_area;      // mesh: nel Cartesian areas
  zd* d_I1;            // mesh: N x N Gram matrix int conj(f_a) f_b (V I on a pixel grid)
  zd* d_mpart;         // mesh: per-chunk partial form factors
  // material fields: nf = 3 (isotropic: 1/(lam+mu), 1/mu, rho) or 7 (a general
  // in-plane stiffness: Voigt compliance S11, S22, rho, S12, S13, S23, S33);
  // d_table holds nf derived rows then the raw lam, mu, rho rows
  int nf;
  bool aniso;
  zd* d_Phi;           // aniso: 3N x 3N compliance Gram matrix, Cholesky in place
  zd* d_LPhi;          // aniso: its triangular inverse
  zd* d_Yw;            // aniso: 3 x 2N x 3N rows of H_i Z (Z = L_Phi^-dagger)
  zd* d_Wk;            // aniso: 3 x 2N x 3N W_i = L_Omega^-1 H_i Z
  zd* d_Pab;           // aniso: 6 x 2N x 2N products W_a W_b^dagger
  double* d_table;     // 3*nphase: 1/(lam+mu), 1/mu, rho

  // assembly
  zd* d_E;             // D x P separable exponential table, row-major [d][p]
  zd* d_Y;             // 3 x P x D first-stage contraction
  zd* d_ghat;          // 3 x D x D form factors [f][da][db] (4 for a mesh: the 4th is of 1)

  // k-independent Gram factors
  zd* d_T;             // 3 x N x N Toeplitz blocks (kappa, mu, rho), Cholesky in place
  zd* d_Linv;          // 3 x N x N inverses of the Cholesky factors (zeros above)
  double* d_G;         // 2 x N Cartesian components of G_a
  zd* d_F;             // 6 x N x N: F_X^a = L_R^-1 diag(G_a) L_X^-dagger
  zd* d_Pp;            // 12 x N x N: F_X^a F_X^b^dagger, a <= b
  zd* d_Cm;            // 6 x n x n monomial matrices of C(k)
  int* d_info;         // [0] Cholesky failure, [1] tensor-core pipeline timeout
  // exact-slice assembly operands
  uint16_t* d_sliceA;  // 3 S P x Kp digit planes of the fields
  uint16_t* d_sliceB;  // S 2D x Kp digit planes of the exponential table
  float* d_sliceD;     // (S 2D) x (3 S P) digit-pair products
  int* d_expA;         // 3 P row exponents
  int* d_expB;         // 2D row exponents
  // exact-slice workspace of the k-monomial products (batch of 2)
  uint16_t* d_mA;
  uint16_t* d_mB;
  float* d_mD;
  int* d_meA;
  int* d_meB;
  zd* d_LinvR2;        // L_R^-1 twice (the A operand of the batched F products)

  // per-k workspace (grown on demand)
  int kcap;            // matrices the workspace holds
  zd* d_C;             // kcap x n x n reduced matrices
  zd* d_vec;           // tridiagonalisation vectors
  zd* d_part;          // partial sums of the tridiagonalisation
  double* d_de;        // kcap x 2n tridiagonal (d, |e|)
  double* d_tau;       // kcap x n reflector scalars
  zd* d_beta;          // kcap x n tridiagonal off-diagonals (complex)
  // mixed path
  zf* d_C32;
  zf* d_vec32;
  zf* d_part32;
  double* d_lamT;
  double* d_scr;
  double* d_mY;
  zd* d_mphase;
  zf* d_X32;
  zd* d_X64;
  zd* d_CX;
  zd* d_mG;
  zd* d_H;
  zd* d_W;
  double* d_theta;
  uint16_t* d_cxA;     // Rayleigh-Ritz product digit planes of C(k)
  uint16_t* d_cxB;     // ... of X
  float* d_cxD;        // digit-pair products
  int* d_cxeA;
  int* d_cxeB;
  int bcap;            // guard-extended block size the mixed workspace holds
  double tol;          // relative omega tolerance the mixed path certifies
  double floor2;       // omega_floor^2 of the cell
  unsigned* d_count;   // kcap arrival counters
  double* d_Q;         // kcap x 2 wavevectors
  double* d_w;         // kcap x nbands_cap output
  int* d_stat;         // kcap
  int wcap;            // capacity of d_w per k
  // LOBPCG workspace (grown on demand)
  double* d_mode;      // mode-shape workspace (stress solves, field tables, staging)
  size_t mode_cap;     // its bytes
  int lcap;            // k the LOBPCG workspace holds
  int lbcap;           // block size it was sized for
  zf* d_lS;
  zf* d_lCS;
  zf* d_lA;
  zf* d_lpart;
  zf* d_lZ;
  zf* d_lY;
  LobState* d_lst;
  zf* d_lX0;
  int* d_lndone;
  int* d_liters;
  float2* d_lvec;
  float* d_lsig;       // inertia check: shifts, row scales, counters
  float* d_lsc;
  int* d_liw;

  // profiling: events around each phase of the last call
  struct BandWs* band;  // two-stage reduction workspace (allocated on first use)
  bool band_used;       // the last FP64 solve took the two-stage reduction

  bool prof;
  bool prof_ready[PH_COUNT];
  cudaEvent_t ev[PH_COUNT][2];
};

void bs_phase_begin(bs_cell* c, int ph, cudaStream_t s);
void bs_phase_end(bs_cell* c, int ph, cudaStream_t s);
void bs_count_launch();

// ------------------------------------------------------------------ errors
void bs_set_error(const char* fmt, ...);
int bs_cuda_status(cudaError_t e, const char* where);

#define TRY_LAUNCH(expr)     \
  do {                       \
    int r__ = (expr);        \
    if (r__) return r__;     \
  } while (0)

#define BS_CHECK_LAUNCH(where)                                   \
  do {                                                           \
    bs_count_launch();                                           \
    cudaError_t e__ = cudaGetLastError();                        \
    if (e__ != cudaSuccess) return bs_cuda_status(e__, where);   \
  } while (0)

// ------------------------------------------------------------------ launchers
// assemble.cu
int bs_launch_assembly(bs_cell* c, cudaStream_t s);
int bs_launch_toeplitz(bs_cell* c, cudaStream_t s);

// dense.cu
int bs_launch_cholesky(zd* A, int n, int batch, long stride, int* info, cudaStream_t s);
int bs_launch_trinv(const zd* L, zd* X, int n, int batch, long stride, cudaStream_t s);
// C[b] = alpha * opA(A[b]) * diag(sc) * opB(B[b]); tri bit0: opA lower, bit1: opB upper,
// bit2: opA upper
int bs_launch_zgemm(bool conjA, bool conjB, int m, int nn, int k, zd alpha,
                    const zd* A, int lda, long sA, const zd* B, int ldb, long sB,
                    const double* sc, long sS, zd* C, int ldc, long sC, int batch,
                    int tri, cudaStream_t s);
int bs_launch_monomials(bs_cell* c, cudaStream_t s);

// tc_gemm.cu / slices.cu: exact-slice contractions on tcgen05
#define BS_SLICES_ASM 7   // digit planes per operand in the assembly (~2^-46)
#define BS_SLICES_RR 7    // digit planes per operand in C X (~2^-46)
// D[z][n][m] = sum_k A[z][m][k] B[z][n][k]; BF16 operands, K % 8 == 0, K <= 4096
int bs_launch_slice_gemm(const uint16_t* A, const uint16_t* B, float* D, int M, int N, int K,
                         int batch, long sA, long sB, long ldd, long sD, int* err, cudaStream_t s);
// Digit orders of an exact-slice product.  The operands hold their S digit
// planes side by side along K, each Kp wide (Kp % 64 == 0): A row m is
// [A_0 | A_1 | ... | A_{S-1}], B row n the reverse [B_{S-1} | ... | B_0].  The
// order-u sum  sum_{s+t=u} A_s B_t^T  is then one contraction over A columns
// [0, (u+1) Kp) against B columns [(S-1-u) Kp, S Kp); it is split into slabs
// of at most BS_SLAB_K terms (the FP32 accumulator stays exact: every digit
// product is at most 2^12 in magnitude).  Orders u >= S are dropped: order S
// weighs at most (S - 1) 2^-7S of |A||B| per term, the size of the digits' own
// truncation (2^-7S per operand), so S = 7 keeps about 2^-46.
#define BS_SLAB_MAX 64
#define BS_SLAB_K 4032
struct SliceSlabs {
  int nq;                    // slabs
  int order[BS_SLAB_MAX];    // digit order u of slab q
  int a0[BS_SLAB_MAX];       // first A column
  int b0[BS_SLAB_MAX];       // first B column
  int len[BS_SLAB_MAX];      // columns (a multiple of 64)
};
// the slabs of S digits of width Kp for an M x N product over `batch`
// entries (cut finer while the launch would have fewer than two CTAs per
// SM); false when they do not fit BS_SLAB_MAX
bool bs_slice_slabs(int S, int Kp, int M, int N, int batch, SliceSlabs* q);
// (entry, slab) output planes to allocate for any batch up to `batch`
size_t bs_slice_planes(int S, int Kp, int M, int N, int batch);
// D[z][q][n][m] = sum_{k < len_q} A[z][m][a0_q + k] B[z][n][b0_q + k] for every
// slab q of (S, Kp); A: batch x M x S Kp, B: batch x N x S Kp
int bs_launch_slice_orders(const uint16_t* A, const uint16_t* B, float* D, int M, int N, int S,
                           int Kp, int batch, int* err, cudaStream_t s);
int bs_launch_fields_tc(bs_cell* c, cudaStream_t s);
size_t bs_fields_tc_elems(int P, int D, int nf, size_t* nA, size_t* nB, size_t* nD);
int bs_launch_cx_tc(const zd* C, const zd* X, int n, int b, int kb, uint16_t* sA, uint16_t* sB,
                    float* sD, int* eA, int* eB, zd* Y, int* err, cudaStream_t s);
void bs_cx_tc_elems(int n, int b, int kb, size_t* nA, size_t* nB, size_t* nD);
// C[z] = A[z] diag(sc) B[z]^dagger for complex N x N column-major matrices (2N <= 4096)
void bs_zgemm_tc_elems(int N, int batch, size_t* nA, size_t* nB, size_t* nD);
int bs_launch_zgemm_tc(const zd* A, long sA, const double* sc, const zd* B, long sB, zd* C, long sC,
                       int N, int batch, uint16_t* wA, uint16_t* wB, float* wD, int* eA, int* eB,
                       int* err, cudaStream_t s);
// the same for column-major A (M x K, leading dimension lda), B (Nc x K) and
// C (M x Nc); exponents eA: batch M, eB: batch Nc; needs 2K <= 4096
bool bs_zgemm_tc_fits(int K);
void bs_zgemm_tc_rect_elems(int M, int Nc, int K, int batch, size_t* nA, size_t* nB, size_t* nD);
int bs_launch_zgemm_tc_rect(const zd* A, int lda, long sA, const double* sc, const zd* B, int ldb,
                            long sB, zd* C, int ldc, long sC, int M, int Nc, int K, int batch,
                            uint16_t* wA, uint16_t* wB, float* wD, int* eA, int* eB, int* err,
                            cudaStream_t s);

// builder.cu
// ---- two-stage reduction to tridiagonal form (band.cu)
#define BS_BAND_NB 8        // half-width of the intermediate band
#define BS_SLICES_BAND 8    // digit planes per operand in its contractions (~2^-53)
#define BS_BAND_PARTS 4     // parts of the batch on concurrent streams (2: 178, 3: 172, 4: 170 ms on config 1)
struct BandWs {
  int n = 0, kb = 0, S = 0;
  zd* V = nullptr;          // kb x (n - nb) x nb reflectors of the current panel
  zd* X = nullptr;          // kb x (n - nb) x nb: A22 V
  zd* W = nullptr;          // kb x (n - nb) x nb
  zd* T = nullptr;          // kb x nb x nb
  uint16_t* wA = nullptr;   // digit planes
  uint16_t* wB = nullptr;
  float* wD = nullptr;      // digit-order sums
  int* eA = nullptr;
  int* eB = nullptr;
  zd* band = nullptr;       // kb x n x 2nb band storage (when it does not fit in shared memory)
  int* dsc = nullptr;       // kb x 2 x nb largest FP64 exponent fields of V's and W's columns
  zd* zpart = nullptr;      // kb x chunks x nb x nb partial sums of V^dagger X
  // per-kernel-group timing of the last reduction (bs_reduction_times):
  // event pairs [group][step] around the panel QR, A22 V, the W formation,
  // the rank-2 update and the bulge chase
  bool prof = false;
  cudaEvent_t* ev = nullptr;
  int evcap = 0;            // event pairs per group
  int nsteps = 0;           // steps recorded by the last reduction
  int timed = 0;            // matrices of the half whose launches the events bracket
  // the batch runs in BS_BAND_PARTS parts, each on a high-priority stream
  // (the chain of panel steps); the fork and join events, and the per-part
  // sizes of the digit buffers
  cudaStream_t sp[BS_BAND_PARTS] = {};
  cudaEvent_t fork = nullptr, join[BS_BAND_PARTS] = {};
  // look-ahead: per part a low-priority stream for the bulk of the trailing
  // update, and the events that order the two (operands packed, update done)
  cudaStream_t sb[BS_BAND_PARTS] = {};
  cudaEvent_t epr[BS_BAND_PARTS] = {}, eru[BS_BAND_PARTS] = {};
  size_t hA = 0, hB = 0, hD = 0, hE = 0;
};
#define BS_BAND_AUTO_MIN 400   // BS_REDUCE_AUTO takes the two-stage reduction from this n on
#define BS_BAND_GROUPS 5
int bs_band_times(BandWs& w, double ms[BS_BAND_GROUPS]);
bool bs_band_supported(int n);
bool bs_use_band(int n);
int bs_band_ws_alloc(BandWs* w, int n, int kb, int S);
void bs_band_ws_free(BandWs* w);
// optional: the Sturm multisection of each part, run on the part's stream
// right after its bulge chase (omega: kb x nbands, stat: kb)
struct BandBisect {
  int nbands;
  double* omega;
  int* stat;
};
int bs_launch_eig_band(zd* A, int n, int kb, BandWs& w, double* de, int* err, cudaStream_t s,
                       const BandBisect* bis = nullptr);
void bs_band_tc_elems(int n, int nb, int kb, int S, size_t* nA, size_t* nB, size_t* nD,
                      size_t* nE);
int bs_launch_band_pack_trail(const zd* A, int n, int o, int m, int kb, uint16_t* wA, int* eA,
                              cudaStream_t s);
int bs_launch_band_av(int m, const zd* V, int ldv, long sv, int nb, int kb, int S, uint16_t* wA,
                      uint16_t* wB, float* wD, int* eA, int* eB, zd* X, int ldx, long sx,
                      int* err, cudaStream_t s);
int bs_launch_band_pack_rank2(const zd* V, const zd* W, int ld, long sv, const int* dsc, int m,
                              int nb, int kb, int S, uint16_t* wA, uint16_t* wB, int* ex,
                              cudaStream_t s);
int bs_rank2_column_tiles(int m);
int bs_launch_rank2_update(const uint16_t* dA, const uint16_t* dB, const int* ex, int m, int kb,
                           zd* A, int n, int o, int ct0, int nct, int* err, cudaStream_t s);


int bs_launch_builder(const zd* Cm, int n, const double* Q, int nk, double q1x, double q1y,
                      double q2x, double q2y, zd* C, cudaStream_t s);

// tridiag.cu: Householder reduction in precision R (double or float).  On
// return column j of A below row j+1 holds v_j (v_j[j+1] = 1 implied),
// de = [d | |beta|], tau[b*n + j] = tau_j and beta[b*n + j] = beta_j, the
// (j+1, j) entry of the unitarily reduced (complex) tridiagonal.
size_t bs_tridiag_vec_elems(int n);
size_t bs_tridiag_part_elems(int n);
// tile: 64 (default) or 32 (tile edge of the fused update + matrix-vector
// step); 0 means 64
template <typename R>
int bs_launch_tridiag(typename Cplx<R>::T* A, int n, int batch, typename Cplx<R>::T* vec,
                      typename Cplx<R>::T* part, double* de, double* tau, zd* beta,
                      unsigned* count, cudaStream_t s, int tile = 64);

// mixed.cu: FP32 reduction + FP64 Rayleigh-Ritz refinement
struct MixedWs {
  zd* C64 = nullptr;        // kb x n x n full Hermitian C(k)
  zf* C32 = nullptr;        // kb x n x n, lower triangle; reflectors after the reduction
  double* de = nullptr;     // kb x 2n tridiagonal
  double* tau = nullptr;    // kb x n
  zd* beta = nullptr;       // kb x n
  double* lamT = nullptr;   // kb x (b+1) eigenvalues of T
  double* scratch = nullptr;// kb x b x 5n inverse-iteration factors
  double* Y = nullptr;      // kb x b x n tridiagonal eigenvectors
  zd* phase = nullptr;      // kb x n diagonal unitary scaling
  zf* X32 = nullptr;        // kb x b x n back-transformed vectors (FP32)
  zd* X64 = nullptr;        // kb x n x b (column-major) FP64 copy
  zd* CX = nullptr;         // kb x n x b
  zd* G = nullptr;          // kb x b x b
  zd* H = nullptr;          // kb x b x b
  zd* W = nullptr;          // kb x b x b Ritz coefficients
  double* theta = nullptr;  // kb x b Ritz values
  uint16_t* cxA = nullptr;  // C X digit planes and products (tensor cores)
  uint16_t* cxB = nullptr;
  float* cxD = nullptr;
  int* cxeA = nullptr;
  int* cxeB = nullptr;
  int* err = nullptr;       // tensor-core pipeline timeout flag
  double* errb = nullptr;   // optional: kb x nbands certified error bounds of theta
  float* csig = nullptr;    // LOBPCG tail: kb count shifts chosen by the certificate
  int* cexp = nullptr;      // and the eigenvalue counts expected below them (-1: none)
};
#define BS_MIXED_MAX_BANDS 24
int bs_mixed_guard(int nbands, int n);
// full32: write the whole FP32 matrix (the LOBPCG path), else its lower triangle
int bs_launch_builder_mixed(const zd* Cm, int n, const double* Q, int nk, double q1x, double q1y,
                            double q2x, double q2y, zd* C64, zf* C32, cudaStream_t s,
                            bool full32 = false);
int bs_launch_mixed_refine(const MixedWs& w, int n, int kb, int nbands, int b, double tol,
                           double floor2, double* omega, int* stat, cudaStream_t s);
// C32 lower triangle (FP32) from the full FP64 C of kb matrices
int bs_launch_c64_to_c32(const zd* C64, zf* C32, int n, int kb, cudaStream_t s);

// lobpcg.cu: block LOBPCG (FP32) with soft locking, batched over k
#define BS_LOB_MAX_BLOCK 16
struct LobState {
  int done;        // 1: no further iterations (converged, limit or breakdown)
  int it;          // updates taken
  int nx, np, nw;  // columns of X, P and W in the current basis
  int cur;         // which of the two basis buffers is current
  int npn;         // P columns of the next update
  int nact;        // unconverged columns of X
  unsigned amask;  // bit c: column c of X is unconverged
  int seedfail;    // the starting block could not be made full rank
  float dshift;    // preconditioner shift (1e-3 of the mean diagonal of C)
  float rmax;      // largest relative FP32 residual of the wanted columns
  float rbest;     // smallest rmax so far, and the iteration it was reached
  int itbest;
  float theta[BS_LOB_MAX_BLOCK];
};
struct LobWs {
  const zf* C32;   // kb x n x n full Hermitian FP32 C(k), column-major
  zf* S;           // 2 x kb x 3b x n basis blocks X | P | W (column-major)
  zf* CS;          // 2 x kb x 3b x n C times the basis blocks
  zf* Axp;         // kb x (3B)^2 Gram block of [X P] (B = BS_LOB_MAX_BLOCK)
  zf* part;        // kb x bs_lob_part_elems(n) partial S^dagger C W per row block
  zf* Z;           // kb x B x 3B Ritz coefficients
  zf* Y;           // kb x B x 3B coefficients of the P directions
  LobState* st;    // kb
  const zf* X0;    // kb x nvec x n starting vectors (reduced basis) or nullptr
  int nvec;
  int* ndone;      // finished-k counter
};
size_t bs_lob_part_elems(int n);
size_t bs_lob_small_elems();
int bs_lob_block(int nbands, int n);
// seed + iterations (check_every > 0: stop early once every k has finished,
// reading the counter every check_every iterations; 0: fixed count)
// tol: relative FP32 residual of every column; tolb: the residual bound the
// FP64 stage certifies (wanted columns only)
int bs_launch_lobpcg(const LobWs& w, int n, int kb, int b, int nb, int maxit, float tol,
                     float tolb, float floor2, int check_every, cudaStream_t s);
int bs_launch_lob_export(const LobWs& w, int n, int kb, int b, zd* X64, int* iters, cudaStream_t s);
// Mp < 0: u holds all n coefficients per vector; Mp >= 0: only the waves
// |alpha|, |beta| <= Mp, 2 (2Mp+1)^2 per vector
int bs_launch_lob_to_reduced(const float2* u, const zd* LR, int N, int M, int Mp, int kb, int nvec,
                             float2* y, cudaStream_t s);
// Iteration limits (bs_set_iteration_limits): LOBPCG iterations and FP64
// multisection sweeps of the Sturm bisection (defaults BS_LOB_MAXIT, 128)
int bs_lob_maxit();
int bs_bisect_sweeps();
// Shift of the eigenvalue-count certificate in the gap above Ritz value i
// (theta ascending, FP64): usable when theta_{i+1} - theta_i >= 2e-3 of its
// size; sigma sits in that gap, at most 1% above theta_i, rounded to FP32
// (the precision of the count), and i + 1 eigenvalues should lie below it.
__host__ __device__ inline bool bs_shift_at(const double* t, int i, double floor2, float* sigma) {
  const double g = t[i + 1] - t[i];
  if (!(g == g && g < 1e308 && g >= 2e-3 * (t[i + 1] > floor2 ? t[i + 1] : floor2))) return false;
  const double h = 0.02 * (t[i] > floor2 ? t[i] : floor2);
  *sigma = (float)(t[i] + 0.5 * (g < h ? g : h));
  return true;
}
// The default shift: the highest usable gap with i in [nb - 1, b - 2];
// *expect = i + 1, or -1 (returns false) when there is none.
__host__ __device__ inline bool bs_count_shift(const double* t, int b, int nb, double floor2,
                                               float* sigma, int* expect) {
  for (int i = b - 2; i >= nb - 1; --i)
    if (bs_shift_at(t, i, floor2, sigma)) {
      *expect = i + 1;
      return true;
    }
  *sigma = 0.f;
  *expect = -1;
  return false;
}
// inertia.cu: eigenvalue-count certificate (FP32 LDL^dagger of the scaled
// C - sigma I, sigma in a gap above the wanted Ritz values); A (lower part of
// C(k), overwritten), sigma (kb), sc (kb x n) floats and iwork (3 kb ints)
// scratch; stat[k] = BS_ENOCONV where the count fails; outcome optional
// shift_given: sigma (kb) and iwork[kb..2kb) (expected counts, -1 for none)
// are already set (by the residual certificate of the Rayleigh-Ritz tail,
// which picks the cut), else they are taken from bs_count_shift
int bs_launch_inertia_check(zf* A, int n, int kb, const double* theta, int b, int nb,
                            double floor2, float* sigma, float* sc, int* iwork, int* stat,
                            int* outcome, cudaStream_t s, bool shift_given = false);
// dense FP64 solve of nf host wavevectors on an assembled cell (host outputs)
int bs_cell_dense_fp64(bs_cell* c, const double* Q, int nf, int nbands, double* om, int* st,
                       cudaStream_t s);
// u = (I_2 (x) L_R^-dagger) X w_j (problem k: L_R^-1 at LinvR + (k / kper) lstride);
// rows (or identity) place problem k's nbands vectors; Mp >= 0 keeps only the
// low-order waves
int bs_launch_lob_vectors(const zd* X64, const zd* Wc, const zd* LinvR, long lstride, int kper,
                          int N, int M, int Mp, int b, int nbands, int kb, const int* rows,
                          float2* out, cudaStream_t s);
// mixed.cu: the FP64 Rayleigh-Ritz tail on a given FP64 block X64 (CX, G, H,
// small eigenproblem, Lehmann lower bounds from the residual Gram); the
// bound on the next eigenvalue comes from the eigenvalues of T (lamT) or,
// when lamT is null, from the shift of the count certificate, which the
// caller must then run (bs_launch_inertia_check)
int bs_launch_rr_tail(const MixedWs& w, int n, int kb, int nbands, int b, double tol,
                      double floor2, double* omega, int* stat, cudaStream_t s);

// bisect.cu
// lowest nbands eigenvalues of batch tridiagonals packed as [b][d(n) | e(n-1), pad];
// writes omega = sqrt(max(lambda, 0)) when want_omega, else lambda
int bs_launch_bisect(const double* de, int n, int batch, int nbands, double* omega, int* stat,
                     cudaStream_t s, bool want_omega = true, double stop_rel = 0.0);

// modes.cu: stress coefficients and plane-wave fields on a grid
void bs_free_mode_workspace(bs_cell* c);
int bs_launch_stress(bs_cell* c, const zd* U, const double* Q, int kc, int nvec, zd* Zk, zd* Zm,
                     zd* Y, zd* S, cudaStream_t s);
int bs_launch_mode_field(const zd* coef, const double* Q, long kbase, int nkt, long f0, long nf,
                         int fpk, int M, int G, zf* E, zf* out, cudaStream_t s);

// mesh.cu: form factors of a mesh cell (centroid rule over its elements)
size_t bs_mesh_partial_elems(int M, int nel, int nfields);
int bs_launch_mesh_assembly(bs_cell* c, cudaStream_t s);

// assemble.cu: per-phase derived table of an isotropic cell
int bs_launch_table(bs_cell* c, cudaStream_t s);

// aniso.cu: a general in-plane stiffness per phase (the full Phi of Eq. (ep))
int bs_launch_gram_aniso(bs_cell* c, cudaStream_t s);
int bs_launch_monomials_aniso(bs_cell* c, cudaStream_t s);
int bs_launch_stress_aniso(bs_cell* c, const zd* U, const double* Q, int kc, int nvec, zd* R3,
                           zd* Y3, zd* S, cudaStream_t s);
