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
// acc - a * conj(b)
__host__ __device__ __forceinline__ zd zfnmac(zd a, zd b, zd acc) {
  acc.x = fma(-a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(-a.y, b.x, acc.y);
  acc.y = fma(a.x, b.y, acc.y);
  return acc;
}

// ------------------------------------------------------------------ cell
struct bs_cell {
  // geometry and truncation
  int P, M, N, n, D, nphase, precision;
  double h1[2], h2[2], q1[2], q2[2], V;
  bool assembled;

  // inputs (device copies)
  uint16_t* d_phase;   // P*P
  double* d_table;     // 3*nphase: 1/(lam+mu), 1/mu, rho

  // assembly
  zd* d_E;             // D x P separable exponential table, row-major [d][p]
  zd* d_Y;             // 3 x P x D first-stage contraction
  zd* d_ghat;          // 3 x D x D form factors [f][da][db]

  // k-independent Gram factors
  zd* d_T;             // 3 x N x N Toeplitz blocks (kappa, mu, rho), Cholesky in place
  zd* d_Linv;          // 3 x N x N inverses of the Cholesky factors (zeros above)
  double* d_G;         // 2 x N Cartesian components of G_a
  zd* d_F;             // 6 x N x N: F_X^a = L_R^-1 diag(G_a) L_X^-dagger
  zd* d_Pp;            // 12 x N x N: F_X^a F_X^b^dagger, a <= b
  zd* d_Cm;            // 6 x n x n monomial matrices of C(k)
  int* d_info;         // [0] Cholesky failure flags

  // per-k workspace (grown on demand)
  int kcap;            // matrices the workspace holds
  zd* d_C;             // kcap x n x n reduced matrices
  zd* d_vec;           // tridiagonalisation vectors
  zd* d_part;          // partial sums of the tridiagonalisation
  double* d_de;        // kcap x 2n tridiagonal (d, |e|)
  double* d_tau;       // kcap
  unsigned* d_count;   // kcap arrival counters
  double* d_Q;         // kcap x 2 wavevectors
  double* d_w;         // kcap x nbands_cap output
  int* d_stat;         // kcap
  int wcap;            // capacity of d_w per k

  // profiling: events around each phase of the last call
  bool prof;
  bool prof_ready[6];
  cudaEvent_t ev[6][2];
};

// phase indices of bs_phase_times
enum { PH_ASM = 0, PH_GRAM = 1, PH_MONO = 2, PH_BUILD = 3, PH_TRID = 4, PH_BISECT = 5 };
void bs_phase_begin(bs_cell* c, int ph, cudaStream_t s);
void bs_phase_end(bs_cell* c, int ph, cudaStream_t s);
void bs_count_launch();

// ------------------------------------------------------------------ errors
void bs_set_error(const char* fmt, ...);
int bs_cuda_status(cudaError_t e, const char* where);

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
// C[b] = alpha * opA(A[b]) * diag(sc) * opB(B[b]); tri bit0: opA lower, bit1: opB upper
int bs_launch_zgemm(bool conjA, bool conjB, int m, int nn, int k, zd alpha,
                    const zd* A, int lda, long sA, const zd* B, int ldb, long sB,
                    const double* sc, long sS, zd* C, int ldc, long sC, int batch,
                    int tri, cudaStream_t s);
int bs_launch_monomials(bs_cell* c, cudaStream_t s);

// builder.cu
int bs_launch_builder(const zd* Cm, int n, const double* Q, int nk, double q1x, double q1y,
                      double q2x, double q2y, zd* C, cudaStream_t s);

// tridiag.cu
size_t bs_tridiag_vec_elems(int n);
size_t bs_tridiag_part_elems(int n);
int bs_launch_tridiag(zd* A, int n, int batch, zd* vec, zd* part, double* de, double* tau,
                      unsigned* count, cudaStream_t s);

// bisect.cu
// lowest nbands eigenvalues of batch tridiagonals packed as [b][d(n) | e(n-1), pad];
// writes omega = sqrt(max(lambda, 0)) when want_omega, else lambda
int bs_launch_bisect(const double* de, int n, int batch, int nbands, double* omega, int* stat,
                     cudaStream_t s, bool want_omega = true);
