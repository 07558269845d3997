// A batch of independent unit cells with uneven truncations, solved
// together on the mixed path (the "thousands of cells" regime the paper
// points to for band-structure optimisation).
//
// Cells are grouped by their truncation M (all cells of a group share the
// eigen dimension n).  Each cell is assembled in turn on one worker cell per
// group (its inputs stay resident for the whole batch; only the worker's
// k-independent state is rebuilt per cell) and its C(k) for all of its
// wavevectors is written into the group's chunk buffers.  Every chunk of
// cells is then reduced and refined as ONE batch of (cell, k) matrices:
// the FP32 Householder reduction, the eigenvalue shifts, inverse iteration,
// the FP64 Rayleigh-Ritz with tensor-core products and the residual bounds.
// The whole sequence can be captured in a CUDA graph on the first solve and
// replayed afterwards.  The reduction's tile edge (32 or 64) is chosen per
// group by timing both on the group's first chunk.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "bs_internal.h"

namespace {

#define CK(call, where)                                        \
  do {                                                         \
    cudaError_t e__ = (call);                                  \
    if (e__ != cudaSuccess) return bs_cuda_status(e__, where); \
  } while (0)

template <typename T>
int balloc(T** p, size_t count, const char* what) {
  *p = nullptr;
  if (count == 0) return BS_OK;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    bs_set_error("cudaMalloc(%s, %zu bytes) failed: %s", what, count * sizeof(T),
                 cudaGetErrorString(e));
    return BS_ENOMEM;
  }
  return BS_OK;
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

// dst[0] |= src[0], dst[1] |= src[1]: a worker cell's status flags into the group's
__global__ void or_flags_kernel(const int* __restrict__ src, int* __restrict__ dst) {
  if (threadIdx.x < 2 && src[threadIdx.x]) atomicOr(dst + threadIdx.x, src[threadIdx.x]);
}

// rows [k][0..w) of src go to dst rows idx[k]: per-cell outputs back in caller order
__global__ void scatter_rows_kernel(const double* __restrict__ src, const int* __restrict__ idx,
                                    int rows, int w, double* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * w) return;
  dst[(size_t)idx[i / w] * w + i % w] = src[i];
}
__global__ void scatter_int_kernel(const int* __restrict__ src, const int* __restrict__ idx,
                                   int rows, int w, int* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * w) return;
  dst[(size_t)idx[i / w] * w + i % w] = src[i];
}

}  // namespace

constexpr int kWorkers = 16;  // cells assembled concurrently per truncation group

struct BatchGroup {
  int M, N, n, b;
  std::vector<int> cells;     // caller indices
  bs_cell* workers[kWorkers]; // each assembles one cell at a time, on its own stream
  cudaStream_t wstream[kWorkers];
  cudaEvent_t wdone[kWorkers];
  cudaEvent_t fork;
  // double buffering: chunk c is assembled into buffer set c & 1 while the
  // main stream reduces chunk c - 1 from the other set
  zd* C64b[2];
  zf* C32b[2];
  zf* lX0b[2];
  zd* lLinvb[2];
  cudaEvent_t adone[2][kWorkers];   // worker w finished assembling into set p
  cudaEvent_t rdone[2];             // the reduction that read set p is done
  // Gram factors of a whole chunk at once: the workers write each cell's
  // three Toeplitz blocks into gT, one stream factors them all (Cholesky and
  // triangular inverse, batched over cells x 3) and the workers take the
  // factors back for the monomials
  zd* gT;                           // chunk x 3 x N x N
  zd* gLinv;                        // chunk x 3 x N x N
  cudaStream_t gstream;
  cudaEvent_t tdone[kWorkers];      // worker w wrote its cells' Toeplitz blocks
  cudaEvent_t gdone;                // the chunk's factors are ready
  bool used[2];
  int nworkers;
  int chunk;                  // cells per reduction batch
  int tile;                   // tridiagonal tile edge (autotuned)
  bool tuned;
  // chunk workspace (chunk * nk matrices)
  zd* C64;
  zf* C32;
  zf* vec32;
  zf* part32;
  double* de;
  double* tau;
  zd* beta;
  unsigned* count;
  double* lamT;
  double* scr;
  double* Y;
  zd* phase;
  zf* X32;
  zd* X64;
  zd* CX;
  zd* G;
  zd* H;
  zd* W;
  double* theta;
  uint16_t* cxA;
  uint16_t* cxB;
  float* cxD;
  int* cxeA;
  int* cxeB;
  double* w;                  // chunk * nk * nbands
  int* st;                    // chunk * nk
  int* d_rowidx;              // cells.size() * nk target rows (cell * nk + k), chunk-major
  double* d_Gall;             // cells.size() * 2N plane-wave vectors G of each cell
  // LOBPCG workspace (chunk * nk problems), allocated when the solver is chosen
  int lb;                     // LOBPCG block size (0: not allocated)
  zf* lS;
  zf* lCS;
  zf* lA;
  zf* lpart;
  zf* lZ;
  zf* lY;
  zf* lX0;
  LobState* lst;
  int* lndone;
  int* liters;
  zd* lLinv;                  // chunk x N x N: L_R^-1 of the chunk's cells (eigenvector output)
  float* lsig;                // inertia check scratch
  float* lsc;
  int* liw;
  double* fbw;                // dense-mixed rescue of uncertified LOBPCG entries
  int* fbst;
  int* fbrow;
  zd* vec64;                  // FP64 solver: reduction vectors and partial sums
  zd* part64;
  BandWs* band;               // FP64 solver: two-stage reduction workspace (large n)
  // [0] tensor-core pipeline timeout of a main-stream product, [1] a Gram
  // Cholesky failed, [2] a tensor-core timeout during a cell's assembly
  // (the workers' own flags are reset by every assembly, so each assembly's
  // flags are OR-ed in here right after it)
  int* d_err;
};

struct bs_batch {
  int ncells, nk, nbands, P;
  std::vector<bs_cell_desc> desc;       // geometry kept on the host
  std::vector<int> nphase;
  uint16_t* d_phase;                    // ncells * P * P
  double* d_raw;                        // concatenated (lam, mu, rho) per cell
  std::vector<size_t> raw_off;
  double* d_Q;                          // ncells * nk * 2
  double* d_w;                          // ncells * nk * nbands
  int* d_st;                            // ncells * nk
  std::vector<BatchGroup> groups;
  bool use_graph;
  cudaGraphExec_t graph;
  cudaStream_t cap;       // non-blocking stream the graph is recorded and replayed on
  cudaEvent_t ev_in, ev_out;
  // profiling: event pairs per chunk and phase (assembly, reduction, shifts, refinement)
  bool prof;
  std::vector<cudaEvent_t> pev;
  size_t pev_used;
  // eigen solver and LOBPCG starting vectors
  int solver;
  float2* d_U;                          // ncells * nk * nvec * 2 (2Mp+1)^2 coefficients
  int Mp, nvec;
  int* d_iters;                         // ncells * nk LOBPCG iterations of the last solve
  bool capturing;                       // a graph is being recorded
  int vecMp;                            // eigenvector output: waves |alpha|,|beta| <= vecMp
  float2* d_vec;                        // ncells * nk * nbands * 2 (2 vecMp + 1)^2, or null
  std::vector<int> fb;                  // ncells * nk: 1 where the dense fallback ran
  std::vector<int> cell_group, cell_gi; // group and index within it of every cell
};

static void prof_mark(bs_batch* B, cudaStream_t s) {
  if (!B->prof) return;
  if (B->pev_used == B->pev.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    B->pev.push_back(e);
  }
  cudaEventRecord(B->pev[B->pev_used++], s);
}

static void free_group(BatchGroup& g) {
  if (g.band) {
    bs_band_ws_free(g.band);
    delete g.band;
    g.band = nullptr;
  }
  for (int w = 0; w < g.nworkers; ++w) {
    if (g.workers[w]) bs_destroy_cell(g.workers[w]);
    if (g.wstream[w]) cudaStreamDestroy(g.wstream[w]);
    if (g.wdone[w]) cudaEventDestroy(g.wdone[w]);
  }
  if (g.fork) cudaEventDestroy(g.fork);
  for (int w = 0; w < kWorkers; ++w)
    if (g.tdone[w]) cudaEventDestroy(g.tdone[w]);
  if (g.gdone) cudaEventDestroy(g.gdone);
  if (g.gstream) cudaStreamDestroy(g.gstream);
  for (int p = 0; p < 2; ++p) {
    for (int w = 0; w < kWorkers; ++w)
      if (g.adone[p][w]) cudaEventDestroy(g.adone[p][w]);
    if (g.rdone[p]) cudaEventDestroy(g.rdone[p]);
    cudaFree(g.C64b[p]);
    cudaFree(g.C32b[p]);
    cudaFree(g.lX0b[p]);
    cudaFree(g.lLinvb[p]);
  }
  void* ps[] = {g.vec32, g.part32, g.de, g.tau, g.beta, g.count, g.lamT, g.scr, g.Y,
                g.phase, g.X32, g.X64, g.CX, g.G, g.H, g.W, g.theta, g.cxA, g.cxB, g.cxD, g.cxeA,
                g.cxeB, g.w, g.st, g.d_rowidx, g.d_Gall, g.lS, g.lCS, g.lA, g.lpart, g.lZ, g.lY,
                g.lst, g.lndone, g.liters, g.lsig, g.lsc, g.liw, g.fbw,
                g.fbst, g.fbrow, g.vec64, g.part64, g.d_err, g.gT, g.gLinv};
  for (void* p : ps) cudaFree(p);
}

static int mixed_rescue(bs_batch* B, BatchGroup& g, int c0, const std::vector<int>& f,
                        double floor2, cudaStream_t s);

static int alloc_lob(BatchGroup& g, int nk, int nbands) {
  if (g.lb) return BS_OK;
  const int b = bs_lob_block(nbands, g.n);
  const size_t K = (size_t)g.chunk * nk, n = g.n, coef = (size_t)BS_LOB_MAX_BLOCK * 3 * BS_LOB_MAX_BLOCK;
  int r = BS_OK;
  if (!r) r = balloc(&g.lS, 2 * K * 3 * b * n, "batch LOBPCG basis");
  if (!r) r = balloc(&g.lCS, 2 * K * 3 * b * n, "batch LOBPCG C basis");
  if (!r) r = balloc(&g.lA, K * bs_lob_small_elems(), "batch LOBPCG Gram");
  if (!r) r = balloc(&g.lpart, K * bs_lob_part_elems(g.n), "batch LOBPCG partial Gram");
  if (!r) r = balloc(&g.lZ, K * coef, "batch LOBPCG Ritz coefficients");
  if (!r) r = balloc(&g.lY, K * coef, "batch LOBPCG P coefficients");
  for (int p = 0; p < 2; ++p)
    if (!r) r = balloc(&g.lX0b[p], K * b * n, "batch LOBPCG starting block");
  g.lX0 = g.lX0b[0];
  if (!r) r = balloc(&g.lst, K, "batch LOBPCG state");
  if (!r) r = balloc(&g.lndone, 1, "batch LOBPCG counter");
  if (!r) r = balloc(&g.liters, K, "batch LOBPCG iterations");
  if (!r) r = balloc(&g.lsig, K, "batch inertia shifts");
  if (!r) r = balloc(&g.lsc, K * n, "batch inertia scales");
  if (!r) r = balloc(&g.liw, 3 * K, "batch inertia counters");
  if (!r) r = balloc(&g.fbw, K * nbands, "batch rescue omega");
  if (!r) r = balloc(&g.fbst, K, "batch rescue status");
  if (!r) r = balloc(&g.fbrow, K, "batch rescue rows");
  if (!r) g.lb = b;
  return r;
}

static int alloc_group(BatchGroup& g, int nk, int nbands) {
  const int n = g.n, b = g.b;
  const size_t K = (size_t)g.chunk * nk;
  size_t ca = 0, cb = 0, cd = 0;
  bs_cx_tc_elems(n, b, (int)K, &ca, &cb, &cd);
  int r = BS_OK;
  for (int p = 0; p < 2; ++p) {
    if (!r) r = balloc(&g.C64b[p], K * n * n, "batch C64");
    if (!r) r = balloc(&g.C32b[p], K * n * n, "batch C32");
  }
  g.C64 = g.C64b[0];
  g.C32 = g.C32b[0];
  if (!r) r = balloc(&g.vec32, K * bs_tridiag_vec_elems(n), "batch vec");
  if (!r) r = balloc(&g.part32, K * bs_tridiag_part_elems(n), "batch partials");
  if (!r) r = balloc(&g.de, K * 2 * n, "batch tridiagonal");
  if (!r) r = balloc(&g.tau, K * n, "batch tau");
  if (!r) r = balloc(&g.beta, K * n, "batch beta");
  if (!r) r = balloc(&g.count, K, "batch counters");
  if (!r) r = balloc(&g.lamT, K * (b + 1), "batch shifts");
  if (!r) r = balloc(&g.scr, K * b * 5 * n, "batch inverse iteration");
  if (!r) r = balloc(&g.Y, K * b * n, "batch Y");
  if (!r) r = balloc(&g.phase, K * n, "batch phases");
  if (!r) r = balloc(&g.X32, K * b * n, "batch X32");
  if (!r) r = balloc(&g.X64, K * b * n, "batch X64");
  if (!r) r = balloc(&g.CX, K * b * n, "batch CX");
  if (!r) r = balloc(&g.G, K * b * b, "batch G");
  if (!r) r = balloc(&g.H, K * b * b, "batch H");
  if (!r) r = balloc(&g.W, K * b * b, "batch W");
  if (!r) r = balloc(&g.theta, K * b, "batch theta");
  if (!r) r = balloc(&g.cxA, ca, "batch C digit planes");
  if (!r) r = balloc(&g.cxB, cb, "batch X digit planes");
  if (!r) r = balloc(&g.cxD, cd, "batch digit products");
  if (!r) r = balloc(&g.cxeA, K * n, "batch C exponents");
  if (!r) r = balloc(&g.cxeB, K * b, "batch X exponents");
  if (!r) r = balloc(&g.w, K * nbands, "batch omega");
  if (!r) r = balloc(&g.st, K, "batch status");
  if (!r) r = balloc(&g.d_rowidx, g.cells.size() * (size_t)nk, "batch row index");
  if (!r) r = balloc(&g.d_Gall, g.cells.size() * 2 * (size_t)g.N, "batch G vectors");
  if (!r) r = balloc(&g.gT, (size_t)g.chunk * 3 * g.N * g.N, "batch Gram blocks");
  if (!r) r = balloc(&g.gLinv, (size_t)g.chunk * 3 * g.N * g.N, "batch Gram inverse factors");
  if (!r) r = balloc(&g.d_err, 3, "batch error flags");
  if (!r && cudaMemset(g.d_err, 0, 3 * sizeof(int)) != cudaSuccess)
    r = bs_cuda_status(cudaGetLastError(), "batch error flag");
  return r;
}

// point a worker cell at the group's gi-th cell (device-resident inputs)
static int load_cell(bs_batch* B, BatchGroup& g, bs_cell* c, int gi, cudaStream_t s) {
  const int ci = g.cells[gi];
  const bs_cell_desc& d = B->desc[ci];
  const int np = B->nphase[ci];
  c->nphase = np;
  for (int i = 0; i < 2; ++i) {
    c->h1[i] = d.h1[i];
    c->h2[i] = d.h2[i];
  }
  const double det = d.h1[0] * d.h2[1] - d.h1[1] * d.h2[0];
  c->V = fabs(det);
  c->q1[0] = 2.0 * M_PI * d.h2[1] / det;
  c->q1[1] = -2.0 * M_PI * d.h2[0] / det;
  c->q2[0] = -2.0 * M_PI * d.h1[1] / det;
  c->q2[1] = 2.0 * M_PI * d.h1[0] / det;
  const size_t PP = (size_t)B->P * B->P;
  CK(cudaMemcpyAsync(c->d_phase, B->d_phase + (size_t)ci * PP, PP * 2, cudaMemcpyDeviceToDevice, s),
     "batch phase");
  CK(cudaMemcpyAsync(c->d_table + 3 * np, B->d_raw + B->raw_off[ci], 3 * np * sizeof(double),
                     cudaMemcpyDeviceToDevice, s),
     "batch table");
  CK(cudaMemcpyAsync(c->d_G, g.d_Gall + (size_t)gi * 2 * g.N, 2 * (size_t)g.N * sizeof(double),
                     cudaMemcpyDeviceToDevice, s),
     "batch G");
  return BS_OK;
}

static double floor2_of(const bs_batch* B, int ci, std::vector<double>& raw) {
  const bs_cell_desc& d = B->desc[ci];
  const int np = B->nphase[ci];
  double ct2 = 1e300;
  for (int i = 0; i < np; ++i) ct2 = std::min(ct2, raw[B->raw_off[ci] + np + i] / raw[B->raw_off[ci] + 2 * np + i]);
  const double det = d.h1[0] * d.h2[1] - d.h1[1] * d.h2[0];
  const double q1x = 2 * M_PI * d.h2[1] / det, q1y = -2 * M_PI * d.h2[0] / det;
  const double q2x = -2 * M_PI * d.h1[1] / det, q2y = 2 * M_PI * d.h1[0] / det;
  return ct2 * std::min(q1x * q1x + q1y * q1y, q2x * q2x + q2y * q2y) / 4.0;
}

// one chunk of a group: assemble its cells, build C(k), reduce + refine as one batch
static void use_buffers(BatchGroup& g, int p) {
  g.C64 = g.C64b[p];
  g.C32 = g.C32b[p];
  if (g.lX0b[p]) g.lX0 = g.lX0b[p];
  if (g.lLinvb[p]) g.lLinv = g.lLinvb[p];
}

// the workers start after everything already queued on s
static int fork_workers(BatchGroup& g, cudaStream_t s) {
  CK(cudaEventRecord(g.fork, s), "batch fork");
  for (int w = 0; w < g.nworkers; ++w) CK(cudaStreamWaitEvent(g.wstream[w], g.fork, 0), "batch fork");
  g.used[0] = g.used[1] = false;
  return BS_OK;
}

// enqueue the assembly and C(k) build of chunk (c0, cn) into buffer set p on
// the worker streams (after the reduction that last read set p), in three
// passes: (1) each worker, for its cells, the material table, the form
// factors and the Toeplitz blocks, copied into the chunk's Gram buffer;
// (2) one stream factors the Gram blocks of the whole chunk (Cholesky and
// triangular inverse batched over cells x 3: full launches instead of the
// small per-cell ones, whose FP64 panels are latency-bound); (3) each worker,
// for its cells, takes the factors back, forms the k-monomials, builds C(k)
// and the starting vectors.
static int assemble_chunk(bs_batch* B, BatchGroup& g, int c0, int cn, int p) {
  const int nk = B->nk, n = g.n;
  const size_t nn = (size_t)n * n, NN3 = 3 * (size_t)g.N * g.N;
  use_buffers(g, p);
  if (g.used[p])
    for (int w = 0; w < g.nworkers; ++w)
      CK(cudaStreamWaitEvent(g.wstream[w], g.rdone[p], 0), "batch buffer reuse");
  // pass 1: form factors and Toeplitz blocks
  for (int i = 0; i < cn; ++i) {
    const int wi = i % g.nworkers;
    bs_cell* wk = g.workers[wi];
    cudaStream_t ws = g.wstream[wi];
    int r = load_cell(B, g, wk, c0 + i, ws);
    if (!r) r = cudaMemsetAsync(wk->d_info, 0, 2 * sizeof(int), ws) == cudaSuccess
                    ? BS_OK
                    : bs_cuda_status(cudaGetLastError(), "batch info");
    if (!r) r = bs_launch_assembly(wk, ws);
    if (!r) r = bs_launch_toeplitz(wk, ws);
    if (!r) {   // a tensor-core timeout of the form factors, before the next cell clears it
      or_flags_kernel<<<1, 32, 0, ws>>>(wk->d_info, g.d_err + 1);
      r = cudaGetLastError() == cudaSuccess ? BS_OK : BS_ECUDA;
      if (r) bs_set_error("or_flags_kernel launch failed");
    }
    if (!r)
      r = cudaMemcpyAsync(g.gT + (size_t)i * NN3, wk->d_T, NN3 * sizeof(zd),
                          cudaMemcpyDeviceToDevice, ws) == cudaSuccess
              ? BS_OK
              : bs_cuda_status(cudaGetLastError(), "batch Gram blocks");
    if (r) return r;
  }
  // pass 2: the chunk's Gram factors at once
  for (int w = 0; w < g.nworkers; ++w) {
    CK(cudaEventRecord(g.tdone[w], g.wstream[w]), "batch Toeplitz done");
    CK(cudaStreamWaitEvent(g.gstream, g.tdone[w], 0), "batch Toeplitz join");
  }
  TRY_LAUNCH(bs_launch_cholesky(g.gT, g.N, 3 * cn, (long)g.N * g.N, g.d_err + 1, g.gstream));
  TRY_LAUNCH(bs_launch_trinv(g.gT, g.gLinv, g.N, 3 * cn, (long)g.N * g.N, g.gstream));
  CK(cudaEventRecord(g.gdone, g.gstream), "batch Gram done");
  for (int w = 0; w < g.nworkers; ++w)
    CK(cudaStreamWaitEvent(g.wstream[w], g.gdone, 0), "batch Gram join");
  // pass 3: monomials, C(k), starting vectors
  for (int i = 0; i < cn; ++i) {
    const int ci = g.cells[c0 + i], wi = i % g.nworkers;
    bs_cell* wk = g.workers[wi];
    cudaStream_t ws = g.wstream[wi];
    const bool lob = B->solver == BS_SOLVER_LOBPCG;
    // the worker's own Linv slot is read by the monomials (and T's slot for
    // L_R by the starting vectors); its host fields still describe cell i
    // only if the worker has no later cell of this chunk, so reload them
    int r = load_cell(B, g, wk, c0 + i, ws);
    if (!r)
      r = cudaMemcpyAsync(wk->d_Linv, g.gLinv + (size_t)i * NN3, NN3 * sizeof(zd),
                          cudaMemcpyDeviceToDevice, ws) == cudaSuccess
              ? BS_OK
              : bs_cuda_status(cudaGetLastError(), "batch Gram factors");
    if (!r && lob && B->d_U)
      r = cudaMemcpyAsync(wk->d_T + 2 * (size_t)g.N * g.N, g.gT + (size_t)i * NN3 + 2 * (size_t)g.N * g.N,
                          (size_t)g.N * g.N * sizeof(zd), cudaMemcpyDeviceToDevice, ws) == cudaSuccess
              ? BS_OK
              : bs_cuda_status(cudaGetLastError(), "batch L_R");
    if (!r) r = cudaMemsetAsync(wk->d_info, 0, 2 * sizeof(int), ws) == cudaSuccess
                    ? BS_OK
                    : bs_cuda_status(cudaGetLastError(), "batch info");
    if (!r) r = bs_launch_monomials(wk, ws);
    if (!r) {
      or_flags_kernel<<<1, 32, 0, ws>>>(wk->d_info, g.d_err + 1);
      r = cudaGetLastError() == cudaSuccess ? BS_OK : BS_ECUDA;
      if (r) bs_set_error("or_flags_kernel launch failed");
    }
    if (!r && B->d_vec)
      r = cudaMemcpyAsync(g.lLinv + (size_t)i * g.N * g.N, g.gLinv + (size_t)i * NN3 + 2 * (size_t)g.N * g.N,
                          (size_t)g.N * g.N * sizeof(zd), cudaMemcpyDeviceToDevice, ws) == cudaSuccess
              ? BS_OK
              : bs_cuda_status(cudaGetLastError(), "batch L_R stash");
    if (!r && B->solver == BS_SOLVER_FP64)
      r = bs_launch_builder(wk->d_Cm, n, B->d_Q + (size_t)ci * nk * 2, nk, wk->q1[0], wk->q1[1],
                            wk->q2[0], wk->q2[1], g.C64 + (size_t)i * nk * nn, ws);
    else if (!r)
      r = bs_launch_builder_mixed(wk->d_Cm, n, B->d_Q + (size_t)ci * nk * 2, nk, wk->q1[0],
                                  wk->q1[1], wk->q2[0], wk->q2[1], g.C64 + (size_t)i * nk * nn,
                                  g.C32 + (size_t)i * nk * nn, ws, lob);
    // starting vectors of this cell in the reduced basis (needs its L_R)
    if (!r && lob && B->d_U) {
      const size_t nl = 2 * (size_t)(2 * B->Mp + 1) * (2 * B->Mp + 1);
      r = bs_launch_lob_to_reduced(B->d_U + (size_t)ci * nk * B->nvec * nl,
                                   wk->d_T + 2 * (size_t)g.N * g.N, g.N, g.M, B->Mp, nk, B->nvec,
                                   g.lX0 + (size_t)i * nk * B->nvec * n, ws);
    }
    if (r) return r;
  }
  for (int w = 0; w < g.nworkers; ++w)
    CK(cudaEventRecord(g.adone[p][w], g.wstream[w]), "batch join");
  return BS_OK;
}

static int reduce_chunk(bs_batch* B, BatchGroup& g, int c0, int cn, int p, double floor2,
                        cudaStream_t s, int tile);
static int reduce_chunk_body(bs_batch* B, BatchGroup& g, int c0, int cn, int p, double floor2,
                             cudaStream_t s, int tile);

// one chunk start to finish (tile autotuning)
static int run_chunk(bs_batch* B, BatchGroup& g, int c0, int cn, double floor2, cudaStream_t s,
                     int tile) {
  TRY_LAUNCH(fork_workers(g, s));
  TRY_LAUNCH(assemble_chunk(B, g, c0, cn, 0));
  return reduce_chunk(B, g, c0, cn, 0, floor2, s, tile);
}

// reduce and refine chunk (c0, cn) from buffer set p on the main stream; marks
// set p free for reuse once done
static int reduce_chunk(bs_batch* B, BatchGroup& g, int c0, int cn, int p, double floor2,
                        cudaStream_t s, int tile) {
  const int r = reduce_chunk_body(B, g, c0, cn, p, floor2, s, tile);
  if (r) return r;
  CK(cudaEventRecord(g.rdone[p], s), "batch buffer done");
  g.used[p] = true;
  return BS_OK;
}

static int reduce_chunk_body(bs_batch* B, BatchGroup& g, int c0, int cn, int p, double floor2,
                             cudaStream_t s, int tile) {
  const int nk = B->nk, n = g.n, b = g.b;
  use_buffers(g, p);
  prof_mark(B, s);   // exposed assembly begins (the main stream waits for the workers)
  for (int w = 0; w < g.nworkers; ++w) CK(cudaStreamWaitEvent(s, g.adone[p][w], 0), "batch join");
  const int K = cn * nk;
  const int* rows = g.d_rowidx + (size_t)c0 * nk;
  prof_mark(B, s);   // assembly ends, reduction begins
  if (B->solver == BS_SOLVER_FP64) {
    // the plain FP64 dense path: Householder reduction and Sturm multisection
    if (g.band) {
      BandBisect bis{B->nbands, g.w, g.st};
      TRY_LAUNCH(bs_launch_eig_band(g.C64, n, K, *g.band, g.de, g.d_err, s, &bis));
      prof_mark(B, s);
    } else {
      TRY_LAUNCH(bs_launch_tridiag<double>(g.C64, n, K, g.vec64, g.part64, g.de, g.tau, g.beta,
                                           g.count, s));
      prof_mark(B, s);
      TRY_LAUNCH(bs_launch_bisect(g.de, n, K, B->nbands, g.w, g.st, s));
    }
    prof_mark(B, s);
    prof_mark(B, s);
  } else if (B->solver == BS_SOLVER_LOBPCG) {
    const int lb = g.lb;
    LobWs lw;
    lw.C32 = g.C32;
    lw.S = g.lS;
    lw.CS = g.lCS;
    lw.Axp = g.lA;
    lw.part = g.lpart;
    lw.Z = g.lZ;
    lw.Y = g.lY;
    lw.st = g.lst;
    lw.X0 = B->d_U ? g.lX0 : nullptr;
    lw.nvec = B->d_U ? B->nvec : 0;
    lw.ndone = g.lndone;
    // a graph replays a fixed sequence: no early exit there (finished k
    // return at once from every later launch)
    TRY_LAUNCH(bs_launch_lobpcg(lw, n, K, lb, B->nbands, bs_lob_maxit(), 1e-3f, 1e-6f, (float)floor2,
                                B->capturing ? 0 : 4, s));
    TRY_LAUNCH(bs_launch_lob_export(lw, n, K, lb, g.X64, g.liters, s));
    prof_mark(B, s);
    prof_mark(B, s);
    MixedWs w;
    memset(&w, 0, sizeof(w));
    w.C64 = g.C64; w.X64 = g.X64; w.CX = g.CX; w.G = g.G; w.H = g.H; w.W = g.W;
    w.theta = g.theta; w.lamT = nullptr; w.cxA = g.cxA; w.cxB = g.cxB; w.cxD = g.cxD;
    w.cxeA = g.cxeA; w.cxeB = g.cxeB; w.err = g.d_err;
    w.csig = g.lsig; w.cexp = g.liw + K;   // the count check's shift and expected count
    CK(cudaMemsetAsync(g.st, 0, K * sizeof(int), s), "batch status");
    TRY_LAUNCH(bs_launch_rr_tail(w, n, K, B->nbands, lb, 1e-6, floor2, g.w, g.st, s));
    TRY_LAUNCH(bs_launch_inertia_check(g.C32, n, K, g.theta, lb, B->nbands, floor2, g.lsig, g.lsc,
                                       g.liw, g.st, nullptr, s, true));
    if (B->d_vec)
      TRY_LAUNCH(bs_launch_lob_vectors(g.X64, g.W, g.lLinv, (long)g.N * g.N, nk, g.N, g.M, B->vecMp,
                                       lb, B->nbands, K, rows, B->d_vec, s));
    prof_mark(B, s);
    scatter_int_kernel<<<(K + 255) / 256, 256, 0, s>>>(g.liters, rows, K, 1, B->d_iters);
    BS_CHECK_LAUNCH("scatter_int_kernel");
    scatter_rows_kernel<<<(K * B->nbands + 255) / 256, 256, 0, s>>>(g.w, rows, K, B->nbands,
                                                                    B->d_w);
    BS_CHECK_LAUNCH("scatter_rows_kernel");
    scatter_int_kernel<<<(K + 255) / 256, 256, 0, s>>>(g.st, rows, K, 1, B->d_st);
    BS_CHECK_LAUNCH("scatter_int_kernel");
    // outside a graph: the uncertified entries of this chunk go through the
    // dense mixed path at once (their FP64 C(k) are still here)
    if (!B->capturing) {
      std::vector<int> sth(K);
      CK(cudaMemcpyAsync(sth.data(), g.st, K * sizeof(int), cudaMemcpyDeviceToHost, s),
         "batch rescue status");
      CK(cudaStreamSynchronize(s), "batch rescue sync");
      std::vector<int> f;
      for (int k = 0; k < K; ++k)
        if (sth[k]) f.push_back(k);
      if (!f.empty()) TRY_LAUNCH(mixed_rescue(B, g, c0, f, floor2, s));
    }
    return BS_OK;
  } else {
  TRY_LAUNCH(bs_launch_tridiag<float>(g.C32, n, K, g.vec32, g.part32, g.de, g.tau, g.beta, g.count,
                                      s, tile));
  prof_mark(B, s);
  TRY_LAUNCH(bs_launch_bisect(g.de, n, K, b + 1, g.lamT, nullptr, s, false, 1e-9));
  prof_mark(B, s);
  MixedWs w;
  w.C64 = g.C64; w.C32 = g.C32; w.de = g.de; w.tau = g.tau; w.beta = g.beta; w.lamT = g.lamT;
  w.scratch = g.scr; w.Y = g.Y; w.phase = g.phase; w.X32 = g.X32; w.X64 = g.X64; w.CX = g.CX;
  w.G = g.G; w.H = g.H; w.W = g.W; w.theta = g.theta; w.cxA = g.cxA; w.cxB = g.cxB;
  w.cxD = g.cxD; w.cxeA = g.cxeA; w.cxeB = g.cxeB; w.err = g.d_err;
  TRY_LAUNCH(bs_launch_mixed_refine(w, n, K, B->nbands, b, 1e-6, floor2, g.w, g.st, s));
  if (B->d_vec)
    TRY_LAUNCH(bs_launch_lob_vectors(g.X64, g.W, g.lLinv, (long)g.N * g.N, nk, g.N, g.M, B->vecMp, b,
                                     B->nbands, K, rows, B->d_vec, s));
  prof_mark(B, s);   // refinement ends
  }
  // scatter (cell, k) rows into caller order
  scatter_rows_kernel<<<(K * B->nbands + 255) / 256, 256, 0, s>>>(g.w, rows, K, B->nbands,
                                                                  B->d_w);
  BS_CHECK_LAUNCH("scatter_rows_kernel");
  scatter_int_kernel<<<(K + 255) / 256, 256, 0, s>>>(g.st, rows, K, 1, B->d_st);
  BS_CHECK_LAUNCH("scatter_int_kernel");
  return BS_OK;
}

// the single-cell checks of bs_create_cell, on host copies
static int validate(const bs_cell_desc& d, int i, const std::vector<double>& lmr,
                    const std::vector<uint16_t>& ph) {
  const int np = d.nphase;
  const double det = d.h1[0] * d.h2[1] - d.h1[1] * d.h2[0];
  if (d.M < 0 || d.M > 15 || 2 * d.M + 1 > d.P || np < 1 || np > 65536 || !(fabs(det) > 0.0) ||
      !isfinite(det)) {
    bs_set_error("bs_batch_create: cell %d: need 0 <= M <= 15, 2M+1 <= P, 1 <= nphase <= 65536 "
                 "and a lattice basis", i);
    return BS_EINVAL;
  }
  for (int k = 0; k < np; ++k) {
    const double lam = lmr[k], mu = lmr[np + k], rho = lmr[2 * np + k];
    if (!isfinite(lam) || !isfinite(mu) || !isfinite(rho) || !(mu > 0.0) || !(lam + mu > 0.0) ||
        !(rho > 0.0)) {
      bs_set_error("bs_batch_create: cell %d phase %d has lam=%g mu=%g rho=%g", i, k, lam, mu, rho);
      return BS_EINVAL;
    }
  }
  for (size_t k = 0; k < ph.size(); ++k)
    if (ph[k] >= np) {
      bs_set_error("bs_batch_create: cell %d pixel %zu has phase %u >= nphase %d", i, k, ph[k], np);
      return BS_EINVAL;
    }
  return BS_OK;
}

extern "C" int bs_batch_create(const bs_cell_desc* descs, int ncells, int nk, int nbands,
                               bs_batch** out) {
  if (!descs || !out || ncells < 1 || nk < 1 || nbands < 1 || nbands > BS_MIXED_MAX_BANDS) {
    bs_set_error("bs_batch_create: need descs, ncells >= 1, nk >= 1, 1 <= nbands <= %d",
                 BS_MIXED_MAX_BANDS);
    return BS_EINVAL;
  }
  *out = nullptr;
  const int P = descs[0].P;
  for (int i = 0; i < ncells; ++i) {
    const bs_cell_desc& d = descs[i];
    if (d.P != P || d.precision != BS_PREC_MIXED) {
      bs_set_error("bs_batch_create: cell %d: all cells need the same P and BS_PREC_MIXED", i);
      return BS_EINVAL;
    }
    const int n = 2 * (2 * d.M + 1) * (2 * d.M + 1);
    if (nbands + 2 > n || n > 2048) {
      bs_set_error("bs_batch_create: cell %d: need nbands + 2 <= n <= 2048 (n = %d)", i, n);
      return BS_EINVAL;
    }
  }
  bs_batch* B = new bs_batch();
  B->ncells = ncells;
  B->nk = nk;
  B->nbands = nbands;
  B->P = P;
  B->desc.assign(descs, descs + ncells);
  B->nphase.resize(ncells);
  B->raw_off.resize(ncells);
  size_t rawn = 0;
  for (int i = 0; i < ncells; ++i) {
    B->nphase[i] = descs[i].nphase;
    B->raw_off[i] = rawn;
    rawn += 3 * (size_t)descs[i].nphase;
  }
  int r = BS_OK;
  const size_t PP = (size_t)P * P;
  if (!r) r = balloc(&B->d_phase, ncells * PP, "batch phase maps");
  if (!r) r = balloc(&B->d_raw, rawn, "batch tables");
  if (!r) r = balloc(&B->d_Q, (size_t)ncells * nk * 2, "batch Q");
  if (!r) r = balloc(&B->d_w, (size_t)ncells * nk * nbands, "batch omega");
  if (!r) r = balloc(&B->d_st, (size_t)ncells * nk, "batch status");
  if (!r) r = balloc(&B->d_iters, (size_t)ncells * nk, "batch iterations");
  if (!r && cudaMemset(B->d_iters, 0, (size_t)ncells * nk * sizeof(int)) != cudaSuccess)
    r = bs_cuda_status(cudaGetLastError(), "bs_batch_create");
  B->cell_group.assign(ncells, 0);
  B->cell_gi.assign(ncells, 0);
  std::vector<double> raw(rawn);
  std::map<int, std::vector<int>> byM;
  std::vector<uint16_t> ph(PP);
  for (int i = 0; !r && i < ncells; ++i) {
    const int np = descs[i].nphase;
    if (np < 1 || !descs[i].phase || !descs[i].lam || !descs[i].mu || !descs[i].rho) {
      bs_set_error("bs_batch_create: cell %d: NULL array or nphase < 1", i);
      r = BS_EINVAL;
      break;
    }
    cudaError_t e = cudaMemcpy(ph.data(), descs[i].phase, PP * 2, cudaMemcpyDefault);
    if (e == cudaSuccess) e = cudaMemcpy(&raw[B->raw_off[i]], descs[i].lam, np * 8, cudaMemcpyDefault);
    if (e == cudaSuccess) e = cudaMemcpy(&raw[B->raw_off[i] + np], descs[i].mu, np * 8, cudaMemcpyDefault);
    if (e == cudaSuccess) e = cudaMemcpy(&raw[B->raw_off[i] + 2 * np], descs[i].rho, np * 8, cudaMemcpyDefault);
    if (e == cudaSuccess) e = cudaMemcpy(B->d_phase + i * PP, ph.data(), PP * 2, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      r = bs_cuda_status(e, "bs_batch_create copy");
      break;
    }
    std::vector<double> lmr(raw.begin() + B->raw_off[i], raw.begin() + B->raw_off[i] + 3 * np);
    r = validate(descs[i], i, lmr, ph);
    byM[descs[i].M].push_back(i);
  }
  if (!r) {
    cudaError_t e = cudaMemcpy(B->d_raw, raw.data(), rawn * 8, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) r = bs_cuda_status(e, "bs_batch_create tables");
  }
  // chunk budget: 60 % of the device memory free now, shared by the groups in
  // proportion to the workspace each would need to hold all of its cells
  // bytes per cell: C64 16 n^2, C32 8 n^2, C digit planes 24 n^2, C X
  // products 288 n b, vectors and inverse-iteration factors ~ 120 n b
  auto per_cell_bytes = [&](int M) {
    const double n = 2.0 * (2 * M + 1) * (2 * M + 1);
    return (double)nk * n * ((2 * (16.0 + 8.0) + 24.0) * n + 410.0 * bs_mixed_guard(nbands, (int)n));
  };
  double need = 0.0;
  for (auto& kv : byM) need += kv.second.size() * per_cell_bytes(kv.first);
  double budget = 12e9 * byM.size();
  {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) budget = 0.6 * (double)fr;
    else cudaGetLastError();
  }
  for (auto& kv : byM) {
    if (r) break;
    BatchGroup g{};
    g.cells = kv.second;
    g.M = kv.first;
    g.N = (2 * g.M + 1) * (2 * g.M + 1);
    g.n = 2 * g.N;
    g.b = bs_mixed_guard(nbands, g.n);
    int npmax = 1, ci0 = g.cells[0];
    for (int ci : g.cells) npmax = std::max(npmax, descs[ci].nphase);
    // worker cell: sized for the group's largest table
    bs_cell_desc wd = descs[ci0];
    std::vector<double> ones(npmax, 1.0);
    std::vector<uint16_t> zero(PP, 0);
    wd.nphase = npmax;
    wd.lam = ones.data();
    wd.mu = ones.data();
    wd.rho = ones.data();
    wd.phase = zero.data();
    g.nworkers = (int)std::min<size_t>(kWorkers, g.cells.size());
    for (int w = 0; !r && w < g.nworkers; ++w) {
      r = bs_create_cell(&wd, &g.workers[w]);
      if (!r) {
        cudaError_t e = cudaStreamCreateWithFlags(&g.wstream[w], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.wdone[w], cudaEventDisableTiming);
        if (e != cudaSuccess) r = bs_cuda_status(e, "bs_batch_create worker");
      }
    }
    if (!r) {
      cudaError_t e = cudaEventCreateWithFlags(&g.fork, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g.gstream, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.gdone, cudaEventDisableTiming);
      for (int w = 0; w < g.nworkers && e == cudaSuccess; ++w)
        e = cudaEventCreateWithFlags(&g.tdone[w], cudaEventDisableTiming);
      for (int p = 0; p < 2 && e == cudaSuccess; ++p) {
        e = cudaEventCreateWithFlags(&g.rdone[p], cudaEventDisableTiming);
        for (int w = 0; w < g.nworkers && e == cudaSuccess; ++w)
          e = cudaEventCreateWithFlags(&g.adone[p][w], cudaEventDisableTiming);
      }
      if (e != cudaSuccess) r = bs_cuda_status(e, "bs_batch_create events");
    }
    if (r) {
      B->groups.push_back(g);
      break;
    }
    for (size_t i = 0; i < g.cells.size(); ++i) {
      B->cell_group[g.cells[i]] = (int)B->groups.size();
      B->cell_gi[g.cells[i]] = (int)i;
    }
    const double per_cell = per_cell_bytes(g.M);
    const double share = budget * (g.cells.size() * per_cell) / std::max(need, 1.0);
    g.chunk = (int)std::max(1.0, std::min((double)g.cells.size(), share / per_cell));
    g.tile = 64;
    g.tuned = false;
    r = alloc_group(g, nk, nbands);
    if (!r) {
      // plane-wave vectors of every cell and the caller row of every (cell, k)
      std::vector<double> Gall(g.cells.size() * 2 * (size_t)g.N);
      std::vector<int> rows(g.cells.size() * (size_t)nk);
      for (size_t i = 0; i < g.cells.size(); ++i) {
        const bs_cell_desc& d = descs[g.cells[i]];
        const double det = d.h1[0] * d.h2[1] - d.h1[1] * d.h2[0];
        const double q1x = 2 * M_PI * d.h2[1] / det, q1y = -2 * M_PI * d.h2[0] / det;
        const double q2x = -2 * M_PI * d.h1[1] / det, q2y = 2 * M_PI * d.h1[0] / det;
        for (int a = 0; a < g.N; ++a) {
          const int al = a / (2 * g.M + 1) - g.M, be = a % (2 * g.M + 1) - g.M;
          Gall[i * 2 * g.N + a] = al * q1x + be * q2x;
          Gall[i * 2 * g.N + g.N + a] = al * q1y + be * q2y;
        }
        for (int k = 0; k < nk; ++k) rows[i * nk + k] = g.cells[i] * nk + k;
      }
      cudaError_t e = cudaMemcpy(g.d_Gall, Gall.data(), Gall.size() * 8, cudaMemcpyHostToDevice);
      if (e == cudaSuccess)
        e = cudaMemcpy(g.d_rowidx, rows.data(), rows.size() * 4, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) r = bs_cuda_status(e, "bs_batch_create group tables");
    }
    B->groups.push_back(g);
  }
  if (r) {
    bs_batch_destroy(B);
    return r;
  }
  *out = B;
  return BS_OK;
}

extern "C" int bs_batch_destroy(bs_batch* B) {
  if (!B) return BS_OK;
  for (auto& g : B->groups) free_group(g);
  for (cudaEvent_t e : B->pev) cudaEventDestroy(e);
  if (B->graph) cudaGraphExecDestroy(B->graph);
  if (B->cap) cudaStreamDestroy(B->cap);
  if (B->ev_in) cudaEventDestroy(B->ev_in);
  if (B->ev_out) cudaEventDestroy(B->ev_out);
  cudaFree(B->d_phase);
  cudaFree(B->d_raw);
  cudaFree(B->d_Q);
  cudaFree(B->d_w);
  cudaFree(B->d_st);
  cudaFree(B->d_iters);
  cudaFree(B->d_U);
  cudaFree(B->d_vec);
  delete B;
  return BS_OK;
}

static void drop_graph(bs_batch* B) {
  if (B->graph) {
    cudaGraphExecDestroy(B->graph);
    B->graph = nullptr;
  }
}

extern "C" int bs_batch_set_solver(bs_batch* B, int solver) {
  if (!B || (solver != BS_SOLVER_DENSE && solver != BS_SOLVER_LOBPCG && solver != BS_SOLVER_FP64)) {
    bs_set_error("bs_batch_set_solver: NULL batch or unknown solver");
    return BS_EINVAL;
  }
  if (solver == BS_SOLVER_LOBPCG) {
    if (B->nbands > BS_LOB_MAX_BANDS) {
      bs_set_error("bs_batch_set_solver: LOBPCG needs nbands <= %d", BS_LOB_MAX_BANDS);
      return BS_EINVAL;
    }
    for (auto& g : B->groups)
      if (B->nbands + 5 > g.n) {
        bs_set_error("bs_batch_set_solver: LOBPCG needs nbands + 5 <= n (n = %d)", g.n);
        return BS_EINVAL;
      }
    for (auto& g : B->groups) TRY_LAUNCH(alloc_lob(g, B->nk, B->nbands));
  }
  if (solver == BS_SOLVER_FP64) {
    for (auto& g : B->groups) {
      const size_t K = (size_t)g.chunk * B->nk;
      if (!g.vec64) TRY_LAUNCH(balloc(&g.vec64, K * bs_tridiag_vec_elems(g.n), "batch FP64 vectors"));
      if (!g.part64)
        TRY_LAUNCH(balloc(&g.part64, K * bs_tridiag_part_elems(g.n), "batch FP64 partials"));
      if (bs_use_band(g.n)) {
        if (!g.band) g.band = new BandWs();
        TRY_LAUNCH(bs_band_ws_alloc(g.band, g.n, (int)K, BS_SLICES_BAND));
      } else if (g.band) {
        bs_band_ws_free(g.band);
        delete g.band;
        g.band = nullptr;
      }
    }
  }
  if (solver != B->solver) drop_graph(B);
  B->solver = solver;
  return BS_OK;
}

extern "C" int bs_batch_set_start(bs_batch* B, const float* U, int Mp, int nvec) {
  if (!B) {
    bs_set_error("bs_batch_set_start: NULL batch");
    return BS_EINVAL;
  }
  if (!U) {
    if (B->d_U) drop_graph(B);
    cudaFree(B->d_U);
    B->d_U = nullptr;
    B->nvec = 0;
    return BS_OK;
  }
  int mmin = 1 << 30;
  for (auto& g : B->groups) mmin = std::min(mmin, g.M);
  int bmin = 1 << 30;
  for (auto& g : B->groups) bmin = std::min(bmin, bs_lob_block(B->nbands, g.n));
  if (Mp < 0 || Mp > mmin || nvec < 1 || nvec > bmin) {
    bs_set_error("bs_batch_set_start: need 0 <= Mp <= %d (smallest M) and 1 <= nvec <= %d",
                 mmin, bmin);
    return BS_EINVAL;
  }
  const size_t count = (size_t)B->ncells * B->nk * nvec * 2 * (2 * Mp + 1) * (2 * Mp + 1);
  if (!B->d_U || Mp != B->Mp || nvec != B->nvec) {
    drop_graph(B);
    cudaFree(B->d_U);
    B->d_U = nullptr;
    TRY_LAUNCH(balloc(&B->d_U, count, "batch starting vectors"));
  }
  B->Mp = Mp;
  B->nvec = nvec;
  CK(cudaMemcpy(B->d_U, U, count * sizeof(float2), cudaMemcpyDefault), "bs_batch_set_start");
  return BS_OK;
}

extern "C" int bs_batch_set_vectors(bs_batch* B, int Mp) {
  if (!B) {
    bs_set_error("bs_batch_set_vectors: NULL batch");
    return BS_EINVAL;
  }
  drop_graph(B);
  cudaFree(B->d_vec);
  B->d_vec = nullptr;
  if (Mp < 0) return BS_OK;
  for (auto& g : B->groups)
    if (Mp > g.M) {
      bs_set_error("bs_batch_set_vectors: Mp = %d exceeds a cell's M = %d", Mp, g.M);
      return BS_EINVAL;
    }
  for (auto& g : B->groups)
    for (int q = 0; q < 2; ++q)
      if (!g.lLinvb[q])
        TRY_LAUNCH(balloc(&g.lLinvb[q], (size_t)g.chunk * g.N * g.N, "batch L_R stash"));
  for (auto& g : B->groups) g.lLinv = g.lLinvb[0];
  const size_t len = 2 * (size_t)(2 * Mp + 1) * (2 * Mp + 1);
  TRY_LAUNCH(balloc(&B->d_vec, (size_t)B->ncells * B->nk * B->nbands * len, "batch vectors"));
  B->vecMp = Mp;
  return BS_OK;
}

extern "C" int bs_batch_vectors(const bs_batch* B, float* U_out) {
  if (!B || !U_out || !B->d_vec) {
    bs_set_error("bs_batch_vectors: NULL argument or vectors not enabled");
    return BS_EINVAL;
  }
  const size_t len = 2 * (size_t)(2 * B->vecMp + 1) * (2 * B->vecMp + 1);
  CK(cudaMemcpy(U_out, B->d_vec, (size_t)B->ncells * B->nk * B->nbands * len * sizeof(float2),
                cudaMemcpyDefault), "bs_batch_vectors");
  return BS_OK;
}

extern "C" int bs_batch_stats(const bs_batch* B, int* iters_out, int* fallback_out) {
  if (!B) {
    bs_set_error("bs_batch_stats: NULL batch");
    return BS_EINVAL;
  }
  const size_t nq = (size_t)B->ncells * B->nk;
  if (iters_out) CK(cudaMemcpy(iters_out, B->d_iters, nq * sizeof(int), cudaMemcpyDefault), "bs_batch_stats");
  if (fallback_out) {
    std::vector<int> fb(nq, 0);
    if (B->fb.size() == nq) fb = B->fb;
    CK(cudaMemcpy(fallback_out, fb.data(), nq * sizeof(int), cudaMemcpyDefault), "bs_batch_stats");
  }
  return BS_OK;
}

extern "C" int bs_batch_set_graph(bs_batch* B, int on) {
  if (!B) {
    bs_set_error("bs_batch_set_graph: NULL batch");
    return BS_EINVAL;
  }
  B->use_graph = on != 0;
  if (B->graph) {
    cudaGraphExecDestroy(B->graph);
    B->graph = nullptr;
  }
  return BS_OK;
}

extern "C" int bs_batch_tiles(const bs_batch* B, int* tiles, int* ns, int ngroups_max,
                              int* ngroups) {
  if (!B || !ngroups) {
    bs_set_error("bs_batch_tiles: NULL argument");
    return BS_EINVAL;
  }
  *ngroups = (int)B->groups.size();
  for (int i = 0; i < *ngroups && i < ngroups_max; ++i) {
    if (tiles) tiles[i] = B->groups[i].tile;
    if (ns) ns[i] = B->groups[i].n;
  }
  return BS_OK;
}

// tile autotuning: time both tile edges on the group's first chunk (once)
static int tune_group(bs_batch* B, BatchGroup& g, double floor2, cudaStream_t s) {
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0), "tune");
  CK(cudaEventCreate(&e1), "tune");
  const int cn = std::min(g.chunk, (int)g.cells.size());
  float best = 1e30f;
  int best_tile = 64;
  for (int tile : {64, 32}) {
    CK(cudaEventRecord(e0, s), "tune");
    TRY_LAUNCH(run_chunk(B, g, 0, cn, floor2, s, tile));
    CK(cudaEventRecord(e1, s), "tune");
    CK(cudaEventSynchronize(e1), "tune");
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1), "tune");
    if (ms < best) {
      best = ms;
      best_tile = tile;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  g.tile = best_tile;
  g.tuned = true;
  return BS_OK;
}

// Tile choices of earlier batches in this process, per (device, eigen
// dimension n, log2 of the matrices per reduction launch): a later batch of
// the same shape reuses the choice instead of timing both tile edges again.
static std::mutex g_tile_mu;
static std::map<std::tuple<int, int, int>, int> g_tile_cache;

static std::tuple<int, int, int> tile_key(const bs_batch* B, const BatchGroup& g) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) cudaGetLastError();
  const long mats = (long)std::min(g.chunk, (int)g.cells.size()) * B->nk;
  int lg = 0;
  while ((1L << (lg + 1)) <= mats) ++lg;
  return std::make_tuple(dev, g.n, lg);
}

static void drop_graph(bs_batch* B);

extern "C" int bs_batch_set_tile(bs_batch* B, int tile) {
  if (!B || (tile != -1 && tile != 32 && tile != 64)) {
    bs_set_error("bs_batch_set_tile: NULL batch or tile not in {-1, 32, 64}");
    return BS_EINVAL;
  }
  drop_graph(B);
  for (auto& g : B->groups) {
    if (tile == -1) {
      g.tuned = false;
    } else {
      g.tile = tile;
      g.tuned = true;
    }
  }
  return BS_OK;
}

extern "C" int bs_batch_set_profiling(bs_batch* B, int on) {
  if (!B) {
    bs_set_error("bs_batch_set_profiling: NULL batch");
    return BS_EINVAL;
  }
  B->prof = on != 0;
  B->pev_used = 0;
  return BS_OK;
}

// ms[0] assembly, ms[1] reduction, ms[2] shifts, ms[3] refinement (sums over chunks of the
// last non-graph solve)
extern "C" int bs_batch_phase_times(bs_batch* B, double ms[4]) {
  if (!B || !ms) {
    bs_set_error("bs_batch_phase_times: NULL argument");
    return BS_EINVAL;
  }
  for (int i = 0; i < 4; ++i) ms[i] = 0.0;
  if (!B->prof) return BS_OK;
  for (size_t c = 0; c + 5 <= B->pev_used; c += 5) {   // 5 marks per chunk
    CK(cudaEventSynchronize(B->pev[c + 4]), "bs_batch_phase_times");
    for (int i = 0; i < 4; ++i) {
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, B->pev[c + i], B->pev[c + i + 1]), "bs_batch_phase_times");
      ms[i] += t;
    }
  }
  return BS_OK;
}

// Dense mixed path on the entries f (chunk indices) of the chunk starting at
// cell c0 whose LOBPCG solve was not certified: their FP64 C(k) are moved to
// the front of the chunk buffer (ascending, so no source is overwritten
// before it is read), reduced in FP32 and refined; results go to their rows.
static int mixed_rescue(bs_batch* B, BatchGroup& g, int c0, const std::vector<int>& f,
                        double floor2, cudaStream_t s) {
  const int nk = B->nk, n = g.n, nf = (int)f.size();
  const size_t nn = (size_t)n * n;
  std::vector<int> rows(nf);
  for (int i = 0; i < nf; ++i) {
    if (f[i] != i)
      CK(cudaMemcpyAsync(g.C64 + (size_t)i * nn, g.C64 + (size_t)f[i] * nn, nn * sizeof(zd),
                         cudaMemcpyDeviceToDevice, s), "batch rescue copy");
    rows[i] = g.cells[c0 + f[i] / nk] * nk + f[i] % nk;
    B->fb[rows[i]] = 2;
    if (B->d_vec) {   // no vectors for rescued entries (NaN)
      const size_t len = 2 * (size_t)(2 * B->vecMp + 1) * (2 * B->vecMp + 1) * B->nbands;
      CK(cudaMemsetAsync(B->d_vec + (size_t)rows[i] * len, 0xff, len * sizeof(float2), s),
         "batch rescue vectors");
    }
  }
  CK(cudaMemcpyAsync(g.fbrow, rows.data(), nf * sizeof(int), cudaMemcpyHostToDevice, s),
     "batch rescue rows");
  TRY_LAUNCH(bs_launch_c64_to_c32(g.C64, g.C32, n, nf, s));
  TRY_LAUNCH(bs_launch_tridiag<float>(g.C32, n, nf, g.vec32, g.part32, g.de, g.tau, g.beta,
                                      g.count, s, g.tile));
  TRY_LAUNCH(bs_launch_bisect(g.de, n, nf, g.b + 1, g.lamT, nullptr, s, false, 1e-9));
  MixedWs w;
  w.C64 = g.C64; w.C32 = g.C32; w.de = g.de; w.tau = g.tau; w.beta = g.beta; w.lamT = g.lamT;
  w.scratch = g.scr; w.Y = g.Y; w.phase = g.phase; w.X32 = g.X32; w.X64 = g.X64; w.CX = g.CX;
  w.G = g.G; w.H = g.H; w.W = g.W; w.theta = g.theta; w.cxA = g.cxA; w.cxB = g.cxB;
  w.cxD = g.cxD; w.cxeA = g.cxeA; w.cxeB = g.cxeB; w.err = g.d_err;
  TRY_LAUNCH(bs_launch_mixed_refine(w, n, nf, B->nbands, g.b, 1e-6, floor2, g.fbw, g.fbst, s));
  scatter_rows_kernel<<<(nf * B->nbands + 255) / 256, 256, 0, s>>>(g.fbw, g.fbrow, nf,
                                                                   B->nbands, B->d_w);
  BS_CHECK_LAUNCH("scatter_rows_kernel");
  scatter_int_kernel<<<(nf + 255) / 256, 256, 0, s>>>(g.fbst, g.fbrow, nf, 1, B->d_st);
  BS_CHECK_LAUNCH("scatter_int_kernel");
  return BS_OK;
}

// (cell, k) entries the residual bound did not certify: assemble the cell
// again on a worker and solve those wavevectors with the dense FP64 path
static int dense_fallback(bs_batch* B, cudaStream_t s) {
  const size_t nq = (size_t)B->ncells * B->nk;
  std::vector<int> st(nq);
  CK(cudaMemcpyAsync(st.data(), B->d_st, nq * sizeof(int), cudaMemcpyDeviceToHost, s),
     "bs_batch_solve status");
  CK(cudaStreamSynchronize(s), "bs_batch_solve sync");
  if (B->fb.size() != nq) B->fb.assign(nq, 0);
  std::vector<double> Qh;
  for (int ci = 0; ci < B->ncells; ++ci) {
    std::vector<int> ks;
    for (int k = 0; k < B->nk; ++k)
      if (st[(size_t)ci * B->nk + k]) ks.push_back(k);
    if (ks.empty()) continue;
    if (Qh.empty()) {
      Qh.resize(nq * 2);
      CK(cudaMemcpy(Qh.data(), B->d_Q, nq * 2 * sizeof(double), cudaMemcpyDeviceToHost),
         "bs_batch_solve Q");
    }
    BatchGroup& g = B->groups[B->cell_group[ci]];
    bs_cell* wk = g.workers[0];
    TRY_LAUNCH(load_cell(B, g, wk, B->cell_gi[ci], s));
    TRY_LAUNCH(bs_assemble(wk, s));
    std::vector<double> Qf, om(ks.size() * B->nbands);
    std::vector<int> sf(ks.size());
    for (int k : ks) {
      Qf.push_back(Qh[((size_t)ci * B->nk + k) * 2]);
      Qf.push_back(Qh[((size_t)ci * B->nk + k) * 2 + 1]);
    }
    TRY_LAUNCH(bs_cell_dense_fp64(wk, Qf.data(), (int)ks.size(), B->nbands, om.data(), sf.data(), s));
    for (size_t t = 0; t < ks.size(); ++t) {
      const size_t row = (size_t)ci * B->nk + ks[t];
      CK(cudaMemcpy(B->d_w + row * B->nbands, om.data() + t * B->nbands, B->nbands * sizeof(double),
                    cudaMemcpyHostToDevice), "bs_batch_solve fallback omega");
      CK(cudaMemcpy(B->d_st + row, &sf[t], sizeof(int), cudaMemcpyHostToDevice),
         "bs_batch_solve fallback status");
      if (B->d_vec) {
        const size_t len = 2 * (size_t)(2 * B->vecMp + 1) * (2 * B->vecMp + 1) * B->nbands;
        CK(cudaMemset(B->d_vec + row * len, 0xff, len * sizeof(float2)),
           "bs_batch_solve fallback vectors");   // NaN: no vectors for fallback entries
      }
      B->fb[row] = 1;
    }
  }
  return BS_OK;
}

static int solve_all(bs_batch* B, const std::vector<double>& floors, cudaStream_t s) {
  for (auto& g : B->groups) {
    double f2 = 1e300;
    for (int ci : g.cells) f2 = std::min(f2, floors[ci]);
    CK(cudaMemsetAsync(g.d_err, 0, 3 * sizeof(int), s), "batch error flags");
    // chunk c + 1 is enqueued for assembly before chunk c is reduced, so the
    // workers build it while the main stream reduces (also when the
    // reduction waits on the host, as the LOBPCG progress checks do)
    const int ncells = (int)g.cells.size();
    TRY_LAUNCH(fork_workers(g, s));
    TRY_LAUNCH(assemble_chunk(B, g, 0, std::min(g.chunk, ncells), 0));
    for (int c = 0, c0 = 0; c0 < ncells; ++c, c0 += g.chunk) {
      const int cn = std::min(g.chunk, ncells - c0);
      if (c0 + g.chunk < ncells)
        TRY_LAUNCH(assemble_chunk(B, g, c0 + g.chunk, std::min(g.chunk, ncells - c0 - g.chunk),
                                  (c + 1) & 1));
      TRY_LAUNCH(reduce_chunk(B, g, c0, cn, c & 1, f2, s, g.tile));
    }
  }
  return BS_OK;
}

extern "C" int bs_batch_solve(bs_batch* B, const double* Q, double* omega_out, int* status_out,
                              void* stream) {
  if (!B || !Q || !omega_out) {
    bs_set_error("bs_batch_solve: NULL argument");
    return BS_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nq = (size_t)B->ncells * B->nk;
  std::vector<double> raw;
  std::vector<double> floors(B->ncells);
  {
    size_t rawn = 0;
    for (int i = 0; i < B->ncells; ++i) rawn += 3 * (size_t)B->nphase[i];
    raw.resize(rawn);
    CK(cudaMemcpy(raw.data(), B->d_raw, rawn * 8, cudaMemcpyDeviceToHost), "bs_batch_solve");
    for (int i = 0; i < B->ncells; ++i) floors[i] = floor2_of(B, i, raw);
  }
  CK(cudaMemcpyAsync(B->d_Q, Q, nq * 2 * sizeof(double), cudaMemcpyDefault, s), "bs_batch_solve Q");
  B->fb.assign(nq, 0);
  const bool prof = B->prof;
  B->prof = false;   // not while tuning or recording a graph
  for (auto& g : B->groups) {
    if (g.tuned || B->solver != BS_SOLVER_DENSE) continue;
    const auto key = tile_key(B, g);
    {
      std::lock_guard<std::mutex> lk(g_tile_mu);
      auto it = g_tile_cache.find(key);
      if (it != g_tile_cache.end()) {
        g.tile = it->second;
        g.tuned = true;
        continue;
      }
    }
    double f2 = 1e300;
    for (int ci : g.cells) f2 = std::min(f2, floors[ci]);
    TRY_LAUNCH(tune_group(B, g, f2, s));
    std::lock_guard<std::mutex> lk(g_tile_mu);
    g_tile_cache[key] = g.tile;
  }
  if (B->use_graph) {
    // the caller's stream may be the legacy default stream, which cannot be
    // captured: record and replay on the batch's own stream, ordered after
    // and before the caller's stream with events
    if (!B->cap) {
      CK(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking), "bs_batch_solve stream");
      CK(cudaEventCreateWithFlags(&B->ev_in, cudaEventDisableTiming), "bs_batch_solve event");
      CK(cudaEventCreateWithFlags(&B->ev_out, cudaEventDisableTiming), "bs_batch_solve event");
    }
    CK(cudaEventRecord(B->ev_in, s), "bs_batch_solve order");
    CK(cudaStreamWaitEvent(B->cap, B->ev_in, 0), "bs_batch_solve order");
    if (!B->graph) {
      cudaGraph_t graph;
      CK(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal), "bs_batch_solve capture");
      B->capturing = true;
      const int r = solve_all(B, floors, B->cap);
      B->capturing = false;
      cudaError_t ce = cudaStreamEndCapture(B->cap, &graph);
      if (r) return r;
      if (ce != cudaSuccess) return bs_cuda_status(ce, "bs_batch_solve end capture");
      ce = cudaGraphInstantiate(&B->graph, graph, 0);
      cudaGraphDestroy(graph);
      if (ce != cudaSuccess) return bs_cuda_status(ce, "bs_batch_solve instantiate");
    }
    CK(cudaGraphLaunch(B->graph, B->cap), "bs_batch_solve graph launch");
    CK(cudaEventRecord(B->ev_out, B->cap), "bs_batch_solve order");
    CK(cudaStreamWaitEvent(s, B->ev_out, 0), "bs_batch_solve order");
  } else {
    B->prof = prof;
    B->pev_used = 0;
    TRY_LAUNCH(solve_all(B, floors, s));
  }
  B->prof = prof;
  TRY_LAUNCH(dense_fallback(B, s));
  CK(cudaMemcpyAsync(omega_out, B->d_w, nq * B->nbands * sizeof(double), cudaMemcpyDefault, s),
     "bs_batch_solve omega");
  if (status_out)
    CK(cudaMemcpyAsync(status_out, B->d_st, nq * sizeof(int), cudaMemcpyDefault, s),
       "bs_batch_solve status");
  if (!dev_ptr(omega_out) || (status_out && !dev_ptr(status_out))) {
    CK(cudaStreamSynchronize(s), "bs_batch_solve sync");
    for (auto& g : B->groups) {
      int err[3] = {0, 0, 0};
      CK(cudaMemcpy(err, g.d_err, 3 * sizeof(int), cudaMemcpyDeviceToHost), "info");
      if (err[1]) {
        bs_set_error("bs_batch_solve: a Gram matrix was not positive definite");
        return BS_ENOTPD;
      }
      if (err[0] || err[2]) {
        bs_set_error("bs_batch_solve: a tensor-core pipeline wait reached its limit");
        return BS_ECUDA;
      }
    }
  }
  return BS_OK;
}
