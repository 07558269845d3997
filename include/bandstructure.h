/*
 * bandstructure.h - C ABI of the GB300 mixed-variational band-structure
 * library (libbs.so).
 *
 * The library computes phononic band structures of 2-D pixelated
 * multi-phase unit cells with the mixed-variational (Nemat-Nasser)
 * formulation of Srivastava, "Fast phononic band-structure calculations
 * through a GPU accelerated mixed-variational formulation":
 *
 *   assembly  : density and compliance form factors of the cell
 *               (Eqs. (eo), (ep); centroid quadrature of Sec. III),
 *   per-k     : H(k) of Eq. (eh), the Cholesky factors of the compliance
 *               Gram matrix Phi and of Omega, and the reduced Hermitian
 *               matrix C(k) = L_Omega^-1 H Phi^-1 H^* L_Omega^-dagger,
 *   eigensolve: lowest eigenvalues lambda = omega^2 of
 *               H Phi^-1 H^* U = lambda Omega U (Eq. (eigenvalueproblem)).
 *
 * Conventions shared by every call
 *   - Every function returns an int status: BS_OK (0) or a negative
 *     BS_E* code.  No C++ exception crosses this boundary.  After an
 *     error, bs_last_error() returns a message for the calling thread.
 *   - Pointers may be host or device pointers unless stated otherwise;
 *     the library finds out with cudaPointerGetAttributes.  The caller
 *     keeps ownership of every array it passes in.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls that return results into host memory synchronise
 *     the stream before returning; calls whose outputs are all device
 *     pointers are asynchronous on `stream`.
 *   - A bs_cell handle is not thread-safe: one thread (and one stream)
 *     at a time per handle.  Different handles are independent.
 *   - Wavevectors are fractional: k = Q1 q^1 + Q2 q^2, with the
 *     reciprocal vectors q^i of Eq. (1).
 */
#ifndef BANDSTRUCTURE_H
#define BANDSTRUCTURE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define BS_OK        0
#define BS_EINVAL   -1   /* bad argument: mu <= 0, lam + mu <= 0, rho <= 0, NaN,
                            P < 2M+1, nbands > 2(2M+1)^2, nk < 0, ...          */
#define BS_ENOTPD   -2   /* a Gram matrix (Phi or Omega block) is not positive
                            definite: Cholesky failed                          */
#define BS_ENOCONV  -3   /* an iteration reached its cap; per-k status is set  */
#define BS_ENOMEM   -4   /* device allocation failed                           */
#define BS_ECUDA    -5   /* any other CUDA runtime error                       */
#define BS_ESTATE   -6   /* call out of order (e.g. solve before assemble)     */

/* arithmetic of the eigen path */
#define BS_PREC_FP64   0  /* every step in float64                             */
#define BS_PREC_MIXED  1  /* FP32 reduction + FP64 Rayleigh-Ritz refinement    */

/* IBZ boundary paths for bs_bands (fractional corner points) */
#define BS_PATH_SQUARE_GXMG 0  /* G(0,0) - X(1/2,0) - M(1/2,1/2) - G              */
#define BS_PATH_HEX_GMKG    1  /* G(0,0) - M(1/2,0) - K(2/3,1/3) - G (h2 at 60 deg) */

typedef struct bs_cell bs_cell;

/*
 * Description of one unit cell.
 *   h1, h2  : unit-cell vectors h^1, h^2 in Cartesian coordinates (Sec. II).
 *   P       : pixels per side; pixel (p, q) covers fractional coordinates
 *             [p/P,(p+1)/P) x [q/P,(q+1)/P) and its centroid
 *             ((p+1/2)/P) h^1 + ((q+1/2)/P) h^2 is the quadrature point of
 *             Sec. III, with weight V/P^2, V = |h^1 x h^2|.
 *   phase   : P*P uint16 phase indices, p-major (phase[p*P + q]).
 *   nphase  : number of phases; every phase index must be < nphase.
 *   lam, mu, rho : per-phase Lame constants and density (isotropic plane
 *             strain, Sec. IV); need mu > 0, lam + mu > 0, rho > 0.
 *   M       : plane-wave truncation, alpha, beta in [-M, M]
 *             (Eq. (approximation2d)); N = (2M+1)^2 waves, eigen dimension
 *             n = 2N; requires 2M+1 <= P and M <= 15.
 *   precision : BS_PREC_FP64 or BS_PREC_MIXED.
 */
typedef struct bs_cell_desc {
    double h1[2];
    double h2[2];
    int32_t P;
    const uint16_t* phase;
    int32_t nphase;
    const double* lam;
    const double* mu;
    const double* rho;
    int32_t M;
    int32_t precision;
} bs_cell_desc;

/*
 * bs_create_cell - validate a cell description and copy it into
 * device-owned storage.  Allocates the cell's device workspace.
 * Errors: BS_EINVAL (any constraint above), BS_ENOMEM, BS_ECUDA.
 * On success *out owns the cell until bs_destroy_cell.
 * Synchronous.
 */
int bs_create_cell(const bs_cell_desc* desc, bs_cell** out);

/*
 * bs_mesh_desc - a unit cell given as a mesh of subdomains (the paper's
 * triangle meshes, Sec. III and the hexagonal example of Sec. V), each
 * integrated by the centroid rule int F = sum_e F(c_e) A_e.
 *   h1, h2    : as bs_cell_desc.
 *   nel       : elements; (2M+1)^2 <= nel <= 2^26.
 *   centroid  : nel x 2 doubles, fractional centroid (s, t) of each
 *               element, c_e = s h1 + t h2 (any periodic image); host or
 *               device.
 *   area      : nel doubles, Cartesian areas (> 0); host or device.
 *   phase     : nel uint16 phase indices (< nphase); host or device.
 *   nphase, lam, mu, rho, M, precision : as bs_cell_desc.
 * The caller keeps ownership of every array.
 */
typedef struct bs_mesh_desc {
    double h1[2];
    double h2[2];
    int32_t nel;
    const double* centroid;
    const double* area;
    const uint16_t* phase;
    int32_t nphase;
    const double* lam;
    const double* mu;
    const double* rho;
    int32_t M;
    int32_t precision;
} bs_mesh_desc;

/*
 * bs_create_cell_mesh - bs_create_cell for a mesh.  The form factors are
 * the centroid sums of Eqs. (eo), (ep) over the elements, and H of Eq. (eh)
 * keeps its integral I1 = int conj(f_a) f_b (the plane waves are orthogonal
 * under the pixel rule, not under a general mesh), so C(k) uses L_R^-1 I1
 * where the pixel path uses V L_R^-1.  Every other call takes the cell as
 * it takes a pixel cell (bs_assemble, bs_solve_k, bs_bands,
 * bs_solve_k_lobpcg, bs_stress_coefficients, bs_mode_field); the ragged
 * batch (bs_batch_*) takes pixel cells only.  Errors: BS_EINVAL (any
 * constraint above), BS_ENOMEM, BS_ECUDA; a mesh too coarse for M makes a
 * Gram matrix singular, reported as BS_ENOTPD after bs_assemble.
 * Synchronous.
 */
int bs_create_cell_mesh(const bs_mesh_desc* desc, bs_cell** out);

/*
 * bs_set_stiffness - give every phase a general in-plane stiffness instead of
 * the isotropic (lam, mu) of the cell's description (pixel or mesh cell).
 *   C6 : nphase x 6 doubles per phase, the Voigt entries C11, C22, C12, C16,
 *        C26, C66 of sigma = C (e11, e22, 2 e12) (plane strain); host or
 *        device.  Each C must be symmetric positive definite (BS_EINVAL).
 * The compliance Gram matrix of Eq. (ep) then has all its blocks, Phi =
 * [T[S_rc]] with S = C^-1 (the paper's factors 2 and 4 are those of the
 * Voigt compliance), and bs_assemble factors it as one 3N x 3N matrix.  The
 * densities stay those of the description.  Call before bs_assemble (the
 * cell needs a new bs_assemble afterwards); bs_form_factors then returns 7
 * fields (S11, S22, rho, S12, S13, S23, S33) instead of 3.  Every
 * single-cell call takes the cell; the ragged batch does not.  Synchronous.
 */
int bs_set_stiffness(bs_cell* cell, const double* C6);

/*
 * bs_assemble - everything that does not depend on k, on `stream`:
 *   material fields 1/(lam+mu), 1/mu, rho per pixel (Sec. IV, the
 *   compliance D_jkmn), their form factors ghat(d) = sum_i g_i V_i
 *   exp(-i G_d . x_i) for d in [-2M, 2M]^2 (Eqs. (eo), (ep) with the
 *   centroid rule of Sec. III), the plane-wave (Toeplitz) Gram blocks,
 *   their Cholesky factors, and the six k-monomial coefficient matrices
 *   of C(k).  Asynchronous; a failed Cholesky is reported by the next
 *   call that synchronises (bs_solve_k / bs_bands with host output, or
 *   bs_sync) as BS_ENOTPD.
 */
int bs_assemble(bs_cell* cell, void* stream);

/*
 * bs_solve_k - lowest `nbands` angular frequencies at `nk` wavevectors.
 *   Q        : nk*2 doubles (Q1, Q2) per wavevector, host or device.
 *   omega_out: nk*nbands doubles, ascending per k, omega = sqrt(max(lambda,0))
 *              (Eq. (eigenvalueproblem)); host or device.
 *   status_out: nk ints (0 = converged) or NULL; host or device.
 * Requires bs_assemble first (BS_ESTATE otherwise); 1 <= nbands <= 2N.
 * Asynchronous when every output is a device pointer.  Otherwise it
 * synchronises `stream` and returns BS_ENOCONV when a wavevector did not
 * converge (its status entry, if status_out is given, says which).
 */
int bs_solve_k(bs_cell* cell, const double* Q, int nk, int nbands,
               double* omega_out, int* status_out, void* stream);

/*
 * bs_bands - generate `nk` wavevectors uniform in Cartesian arc length
 * along the closed IBZ boundary `path` (first and last are Gamma), write
 * them to Q_out (nk*2, host or device, may be NULL) and solve them as
 * bs_solve_k does.  Requires nk >= 2.
 */
int bs_bands(bs_cell* cell, int path, int nk, int nbands,
             double* Q_out, double* omega_out, void* stream);

/*
 * bs_solve_k_lobpcg - the lowest `nbands` angular frequencies of the same
 * eigenproblem (Eq. (eigenvalueproblem)) by block LOBPCG instead of a dense
 * reduction.  The paper solves the dense problem; this iterative path is an
 * addition whose cost depends on the starting block, so a good guess of the
 * eigen-subspace (the previous wavevector's vectors, or a learned
 * prediction) saves iterations.
 *   Iterations run in FP32 on C(k) (block of 16 vectors, fewer when n is
 *   small; diagonal preconditioner; soft locking; at most BS_LOB_MAXIT;
 *   the wanted columns stop once their FP32 residual meets the bound below
 *   with a margin); an FP64 Rayleigh-Ritz projection then gives the
 *   frequencies, certified by the same residual bound as the mixed path
 *   (|theta - lambda| <= ||r||^2 / gap <= 2 tol max(theta, omega_floor^2)).
 *   Wavevectors the bound does not certify are solved again by the dense
 *   FP64 path (the fallback); their status is that solve's.
 *   Q, omega_out, status_out : as bs_solve_k (host or device).
 *   X0       : optional starting vectors, nk x nvec x n complex64
 *              (interleaved re, im) of plane-wave displacement coefficients
 *              u (index I*N + a, component I in {x, y}, wave a in the order
 *              of bs_cell_desc's M), host or device; NULL for the cold
 *              start (unit vectors at the smallest diagonal entries of
 *              C(k), with 1e-3 deterministic noise).  Columns beyond nvec
 *              come from the cold start.  0 <= nvec <= b.
 *   iters_out : nk ints, FP32 iterations taken (-1: the starting block
 *              could not be made full rank), or NULL; host or device.
 *   fallback_out : nk ints, 1 where the dense fallback was used, or NULL.
 *   vec_out  : optional nk x nbands x n complex64 eigenvectors u (Ritz
 *              vectors of the FP64 projection, u^dagger Omega u = 1), NaN
 *              for wavevectors that fell back; host or device.
 * Requires a BS_PREC_MIXED cell, 1 <= nbands <= BS_LOB_MAX_BANDS,
 * nbands + 5 <= n and n <= 2048 (BS_EINVAL otherwise).  Synchronises
 * `stream`.  Returns BS_ENOCONV when status_out is NULL and a fallback
 * solve failed.
 */
#define BS_LOB_MAX_BANDS 12
#define BS_LOB_MAXIT 80
int bs_solve_k_lobpcg(bs_cell* cell, const double* Q, int nk, int nbands,
                      const float* X0, int nvec, double* omega_out, int* status_out,
                      int* iters_out, int* fallback_out, float* vec_out, void* stream);

/*
 * bs_set_iteration_limits - the iteration caps of the iterative steps, for
 * tests and diagnostics (the paper has no counterpart; its eigensolve is a
 * direct one).  lobpcg_maxit: LOBPCG iterations per wavevector (default
 * BS_LOB_MAXIT, at most 1000); bisect_sweeps: FP64 multisection sweeps per
 * eigenvalue of the Sturm bisection (default 128, at most 128; the FP32
 * pre-sweeps are capped at min(64, bisect_sweeps)).  A value <= 0 restores
 * the default.  Process-wide; takes effect at the next solve (a CUDA graph
 * recorded earlier keeps the limits it was recorded with).  When the LOBPCG
 * cap runs out the wavevector goes to the certificate as it is and, if not
 * certified, to the dense fallbacks; when the sweep cap runs out before an
 * eigenvalue's bracket reaches FP64 accuracy, that wavevector's status is
 * BS_ENOCONV.  Errors: BS_EINVAL above the maxima.
 */
int bs_set_iteration_limits(int lobpcg_maxit, int bisect_sweeps);

/*
 * bs_set_reduction - how the FP64 path (BS_PREC_FP64 cells, the batch's
 * BS_SOLVER_FP64 and its FP64 fallback) reduces C(k) to real tridiagonal
 * form before the Sturm multisection of Eq. (eigenvalueproblem)'s lowest
 * eigenvalues.  The paper leaves the eigensolve to a host library; both
 * modes are unitary similarity transformations, so the eigenvalues agree
 * to rounding:
 *   BS_REDUCE_ONESTAGE: Householder reflectors column by column, on the
 *     FP64 pipe ((16/3) n^3 flops per k);
 *   BS_REDUCE_TWOSTAGE: dense -> band of half-width 8 by blocked Householder
 *     QR, the trailing two-sided updates as FP64-exact digit-plane products
 *     on the tensor cores (8 digits of 7 bits per operand), then band ->
 *     tridiagonal by bulge chasing in FP64 (O(n^2) work per k);
 *   BS_REDUCE_AUTO (default): two-stage for n >= 400, one-stage below.
 * Process-wide; takes effect at the next solve.  The two-stage reduction
 * needs an n x 8 complex panel in shared memory (n up to about 1800 on
 * GB300); larger n use the one-stage reduction in every mode.
 * Errors: BS_EINVAL for any other mode.
 */
/*
 * bs_reduction_times - with profiling on (bs_set_profiling), the device time
 * in ms of each kernel group of the last two-stage reduction of this cell's
 * FP64 solve, summed over its panel steps: [0] panel Householder QR,
 * [1] A22 V (digit planes of the trailing block and the tensor-core
 * product), [2] the W formation, [3] the trailing rank-2nb update (tensor
 * cores, FP64 epilogue), [4] the bulge chase to tridiagonal form; [5] the
 * number of matrices those launches processed.  The reduction runs the
 * batch in parts on concurrent streams (per part, the chain of panel steps
 * on a high-priority stream and the bulk of each rank-2nb update on a
 * low-priority one); the times are event pairs around the first part's
 * launches, which run beside the others', so every group but the bulge
 * chase also counts time its launches waited for SMs.  All zeros when profiling
 * is off or the last solve took the one-stage reduction.  A measurement aid
 * (the paper has no counterpart).
 */
int bs_reduction_times(bs_cell* cell, double ms[6]);

#define BS_REDUCE_AUTO     0
#define BS_REDUCE_ONESTAGE 1
#define BS_REDUCE_TWOSTAGE 2
int bs_set_reduction(int mode);

/*
 * bs_form_factors - copy the assembled form factors to `out`
 * (host or device): 3 fields (1/(lam+mu), 1/mu, rho), or the 7 of a cell
 * given bs_set_stiffness (S11, S22, rho, S12, S13, S23, S33), x D x D complex
 * (interleaved re, im), D = 4M+1, index [f][da+2M][db+2M].
 * Synchronises `stream` when `out` is a host pointer.
 */
int bs_form_factors(bs_cell* cell, double* out, void* stream);

/*
 * bs_reduced_matrix - the reduced Hermitian matrix
 * C(k) = L^-1 H(k) Phi^-1 H(k)^* L^-dagger (L = Cholesky factor of
 * Omega) at one wavevector Q (2 doubles), written to `out` as an n x n
 * complex column-major matrix (interleaved re, im; n = 2N).  Only the
 * lower triangle is defined.  Host or device pointers.
 */
int bs_reduced_matrix(bs_cell* cell, const double* Q, double* out, void* stream);

/*
 * bs_tridiag_eigenvalues - the eigen step on its own: the lowest `nbands`
 * eigenvalues lambda (ascending) of `batch` real symmetric tridiagonal
 * matrices, by the same Sturm-sequence multisection that finishes
 * bs_solve_k (the matrices Householder reduction leaves behind when the
 * reduced Hermitian matrix of Eq. (eigenvalueproblem) is tridiagonalised).
 *   d       : batch x n diagonals (row-major), host or device.
 *   e       : batch x (n-1) off-diagonals (row-major), host or device;
 *             only |e| matters.  May be NULL when n == 1.
 *   lam_out : batch x nbands eigenvalues, host or device.
 * Accuracy: absolute error <= 4 eps max(||T||, |lambda|).  Allocates and
 * frees its own device scratch; synchronises `stream` before returning.
 */
int bs_tridiag_eigenvalues(const double* d, const double* e, int n, int batch, int nbands,
                           double* lam_out, void* stream);

/*
 * bs_gemm_bf16 - the tensor-core contraction primitive on its own:
 * D[z][n][m] = sum_k A[z][m][k] B[z][n][k] for z < batch, with BF16
 * operands (raw 16-bit patterns) and FP32 results accumulated in tensor
 * memory.  The library uses it on "digit planes" (small-integer BF16
 * values) for which every product and every partial sum is exact, to
 * evaluate the form-factor sums (Eqs. (eo), (ep)) and the Rayleigh-Ritz
 * products of the mixed path at FP64 accuracy.
 *   A : batch x M x K, row-major (K contiguous); host or device.
 *   B : batch x N x K, row-major; host or device.
 *   D : batch x N x M, n-major (D[z][n][m] at (z N + n) M + m); host or device.
 * Requires 8 <= K <= 4096 with K % 8 == 0 and 16-byte aligned device
 * operands.  Synchronises `stream`.  BS_ECUDA if a pipeline wait reached
 * its iteration limit (the kernel then returns without results).
 */
int bs_gemm_bf16(const uint16_t* A, const uint16_t* B, float* D, int M, int N, int K, int batch,
                 void* stream);

/*
 * bs_tridiag_eigenvalues_static - bs_tridiag_eigenvalues without any
 * device allocation.  The paper has no counterpart: this entry point exists
 * for callers that cannot call cudaMalloc/cudaFree, such as code whose
 * device memory is owned by another allocator that reserved it up front,
 * or pipelined code that cannot let cudaFree wait for the whole device.
 *   d, e, lam_out : DEVICE pointers on the current device, with the layout
 *                   of bs_tridiag_eigenvalues (host pointers or memory of
 *                   another GPU: BS_EINVAL).
 *   Limits: batch * 2n <= 1048576 (the scratch is a fixed 8 MiB array in the
 *   library's device image, held by every GPU that loads the library until
 *   the process exits); larger batches return BS_EINVAL - split them.
 *   n <= (the device's opt-in shared memory per block) / 24 bytes, since
 *   one matrix's tridiagonal is staged in shared memory: n <= 9685 on a
 *   GB300 (227 KB); larger n returns BS_EINVAL.
 * The first call on a device looks up the array's device address with the
 * runtime (cudaGetSymbolAddress); make that first call before any stream
 * capture.  First calls from several host threads at once are safe (the
 * per-device address cache is atomic).  All calls share the one array and it keeps the last call's
 * contents, so calls that overlap on the GPU (different streams, or
 * different host threads) race: serialise them.  Asynchronous on `stream`.
 */
int bs_tridiag_eigenvalues_static(const double* d, const double* e, int n, int batch, int nbands,
                                  double* lam_out, void* stream);

/*
 * A batch of independent cells solved together on the mixed path (the
 * regime of many-cell band-structure optimisation the paper's conclusions
 * point to).  Cells may differ in lattice, materials, number of phases and
 * truncation M, but share the pixel count P and use BS_PREC_MIXED.
 *
 * bs_batch_create - copy `ncells` descriptions (host or device arrays; the
 *   caller keeps ownership) into device storage and size the workspace for
 *   `nk` wavevectors per cell and `nbands` branches (nbands <= 24,
 *   nbands + 2 <= n <= 2048 for every cell).  Errors: BS_EINVAL (with the
 *   failing cell's index in the message), BS_ENOMEM, BS_ECUDA.  Synchronous.
 * bs_batch_solve - Q: ncells * nk * 2 fractional wavevectors (cell-major),
 *   omega_out: ncells * nk * nbands (cell-major, ascending per k),
 *   status_out: ncells * nk (0, or the failure status of the dense
 *   fallback below, which re-solves every entry the residual bound did not
 *   certify) or
 *   NULL; host or device pointers.  The first call times the two tile
 *   edges of the per-step reduction per truncation group and keeps the
 *   faster (autotuning); the choice is remembered for the process, per
 *   device, eigen dimension and batch-size class (powers of two of the
 *   matrices per reduction launch), and reused by later batches.
 * bs_batch_set_graph - on != 0: the next bs_batch_solve records the whole
 *   solve in a CUDA graph, later calls replay it (the Q and output pointers
 *   of the recording call must be reused); on == 0 drops the graph.
 * bs_batch_tiles - the reduction variant chosen for each truncation group
 *   and the group's eigen dimension n: 64 or 32 (tile edge of the
 *   per-step kernel).
 * bs_batch_set_tile - force that choice for every group (32 or 64) or,
 *   with -1, return to timing both on the next solve (BS_EINVAL for any
 *   other value).  Drops a recorded graph.
 * bs_batch_set_profiling / bs_batch_phase_times - with profiling on, a
 *   solve that does not replay a graph records CUDA events around each
 *   chunk's phases; phase_times returns milliseconds summed over chunks:
 *   ms[0] assembly (all cells' k-independent set-up and C(k) build),
 *   ms[1] FP32 Householder reduction, ms[2] eigenvalue shifts, ms[3] FP64
 *   refinement.
 * bs_batch_destroy - free everything (NULL is a no-op).
 * bs_batch_set_solver - BS_SOLVER_DENSE (default: the FP32 Householder
 *   reduction above), BS_SOLVER_FP64 (the plain FP64 path of bs_solve_k on
 *   FP64 C(k): Householder reduction and Sturm multisection, every (cell, k)
 *   of a chunk at once) or BS_SOLVER_LOBPCG (the block LOBPCG of
 *   bs_solve_k_lobpcg, its FP64 Rayleigh-Ritz tail and residual bound;
 *   needs nbands <= BS_LOB_MAX_BANDS and nbands + 5 <= n).  Drops a
 *   recorded graph when the solver changes.
 * bs_batch_set_start - LOBPCG starting vectors: U holds ncells * nk * nvec
 *   vectors (cell-major, then k, then vector) of 2 (2Mp+1)^2 complex64
 *   displacement coefficients each, of the plane waves |alpha|, |beta| <= Mp
 *   only (component-major, waves ordered as for a cell of truncation Mp);
 *   the other coefficients are zero.  Copied at the call (host or device
 *   U); NULL returns to the cold start.  Needs Mp <= every cell's M and
 *   1 <= nvec <= the LOBPCG block size.
 * bs_batch_stats - per (cell, k) of the last solve: LOBPCG iterations
 *   (0 on the dense solver) and the fallback taken: 0 none, 1 the dense FP64
 *   solve, 2 the dense mixed path (LOBPCG entries whose residual bound or
 *   eigenvalue count failed are re-solved there within their chunk when the
 *   solve is not replayed from a graph; what still fails takes the FP64 one).
 * bs_batch_set_vectors - Mp >= 0 (at most every cell's M): later solves
 *   also keep the eigenvectors of the nbands branches as the displacement
 *   coefficients u of the waves |alpha|, |beta| <= Mp (u^dagger Omega u = 1
 *   for the full vector); Mp < 0 stops.  Drops a recorded graph.
 * bs_batch_vectors - copy them out: ncells * nk * nbands * 2 (2Mp+1)^2
 *   complex64 (cell-major, then k, band, component, wave), NaN for entries
 *   of the dense fallback; host or device U_out.
 * Every bs_batch_solve ends with that fallback: the (cell, k) entries whose
 * residual bound failed are solved again by the dense FP64 path (the cell
 * is assembled again), so the call always synchronises `stream`.
 */
typedef struct bs_batch bs_batch;
int bs_batch_create(const bs_cell_desc* descs, int ncells, int nk, int nbands, bs_batch** out);
int bs_batch_solve(bs_batch* batch, const double* Q, double* omega_out, int* status_out,
                   void* stream);
int bs_batch_set_graph(bs_batch* batch, int on);
int bs_batch_tiles(const bs_batch* batch, int* tiles, int* ns, int ngroups_max, int* ngroups);
int bs_batch_set_tile(bs_batch* batch, int tile);
int bs_batch_set_profiling(bs_batch* batch, int on);
int bs_batch_phase_times(bs_batch* batch, double ms[4]);
int bs_batch_destroy(bs_batch* batch);
#define BS_SOLVER_DENSE  0
#define BS_SOLVER_LOBPCG 1
#define BS_SOLVER_FP64   2
int bs_batch_set_solver(bs_batch* batch, int solver);
int bs_batch_set_start(bs_batch* batch, const float* U, int Mp, int nvec);
int bs_batch_stats(const bs_batch* batch, int* iters_out, int* fallback_out);
int bs_batch_set_vectors(bs_batch* batch, int Mp);
int bs_batch_vectors(const bs_batch* batch, float* U_out);

/*
 * Learned warm start for bs_solve_k_lobpcg / BS_SOLVER_LOBPCG (not in the
 * paper): a small convolutional network that maps a 64 x 64 cell (its
 * per-pixel lam, mu, rho) and a wavevector to nvec starting vectors, given
 * as the displacement coefficients of the plane waves |alpha|, |beta| <= Mp
 * (the layout of bs_batch_set_start).  Architecture (FP32): three input
 * channels log(lam + 2 mu), log mu, log rho (standardised); four 3x3
 * convolutions with circular padding (3->16->32->32->32 channels), each
 * followed by ReLU and 2x2 mean pooling (64 -> 4 pixels per side, 512
 * features per cell); per (cell, k) the features and 7 wavevector features
 * (Q1, Q2, cos/sin 2 pi Q1, cos/sin 2 pi Q2, hexagonal flag) pass three dense
 * layers 519 -> 512 -> 512 -> nvec * 2 (2Mp+1)^2 complex (ReLU between).
 * Training minimises, per sample, the part of the true eigenvectors' low-order
 * coefficients V (nb vectors) outside the predicted span U:
 *   loss = (||V||^2 - tr(B^H (U^H U + 1e-4 I)^-1 B)) / ||V||^2, B = U^H V,
 * averaged over the batch, with Adam (beta 0.9, 0.999, eps 1e-8).
 *   bs_cnn_create - nvec <= 16, Mp <= 3; capacity max_cells per call and
 *     max_samples = cells * kper per call.
 *   bs_cnn_num_params / set_params / get_params - the flat FP32 parameter
 *     vector (conv weights [co][ci][3][3] and biases layer by layer, then the
 *     dense weights [out][in] and biases); set_params resets Adam; get_params
 *     also returns the gradients of the last train step (grad may be NULL).
 *   bs_cnn_forward - cells c < ncells: phase maps (ncells x 64 x 64 uint16),
 *     their (lam | mu | rho) tables at table + toff[c] with nph[c] phases,
 *     hex[c] != 0 for hexagonal lattices; Q: ncells * kper fractional
 *     wavevectors (kper per cell, cell-major); U_out: ncells * kper * nvec *
 *     2 (2Mp+1)^2 complex64.  Any pointer may be host or device.  Synchronous.
 *   bs_cnn_train_step - the same inputs plus targets V (ncells * kper * nb *
 *     2 (2Mp+1)^2 complex64, nb <= 16); one forward, backward and (lr > 0)
 *     Adam step; per-sample losses to loss_out (or NULL).  With lr = 0 only
 *     the gradients are computed.  Synchronous.
 */
typedef struct bs_cnn bs_cnn;
int bs_cnn_create(int nvec, int Mp, int max_cells, int max_samples, bs_cnn** out);
int bs_cnn_destroy(bs_cnn* net);
int bs_cnn_num_params(const bs_cnn* net, long long* n);
int bs_cnn_set_params(bs_cnn* net, const float* params);
int bs_cnn_get_params(const bs_cnn* net, float* params, float* grad);
int bs_cnn_forward(bs_cnn* net, const uint16_t* phase, const double* table, const long* toff,
                   const int* nph, const int* hex, int ncells, const double* Q, int kper,
                   float* U_out, void* stream);
int bs_cnn_train_step(bs_cnn* net, const uint16_t* phase, const double* table, const long* toff,
                      const int* nph, const int* hex, int ncells, const double* Q, int kper,
                      const float* V, int nb, float lr, float* loss_out, void* stream);

/* bs_cell_dims - N (plane waves) and n = 2N (eigen dimension). */
int bs_cell_dims(const bs_cell* cell, int* N, int* n);

/*
 * bs_stress_coefficients - stress coefficients of Bloch modes (Sec. IV, the
 * second block row of Eq. (equationshomogeneousMatrix): Phi S + H^* U = 0,
 * so S = -Phi^-1 H^* U, as stated after Eq. (eigenvalueproblem)).
 *   Q     : nk*2 doubles (Q1, Q2), host or device.
 *   U     : nk x nvec x 2N complex128 (interleaved re, im) displacement
 *           coefficients, index I*N + a with component I in {u1, u2} and
 *           plane wave a in the alpha-major order of bs_cell_desc's M (the
 *           layout of bs_solve_k_lobpcg's vectors); host or device.
 *   S_out : nk x nvec x 3N complex128, index J*N + a with J in
 *           {S11, S22, S12}; host or device.
 * FP64 throughout, with the k-independent Gram factors of bs_assemble (any
 * precision); U need not be an eigenvector (the map is linear).  Requires
 * bs_assemble (BS_ESTATE otherwise); 1 <= nvec <= 16384.  Asynchronous when
 * U and S_out are both device pointers; nk = 0 does nothing.
 */
int bs_stress_coefficients(bs_cell* cell, const double* Q, int nk, int nvec,
                           const double* U, double* S_out, void* stream);

/*
 * bs_mode_field - fields of plane-wave expansions (Eq. (approximation2d)) on
 * a G x G grid of the unit cell: for every wavevector k and field f,
 *   out[k][f][p][q] = sum_a coef[k][f][a] exp(i K_a . x_pq),
 *   K_a = (Q1 + alpha_a) q^1 + (Q2 + beta_a) q^2  (Eq. (1)),
 *   x_pq = ((p + 1/2)/G) h1 + ((q + 1/2)/G) h2,  0 <= p, q < G
 * (the pixel centres when G = P; p runs along h1).  Displacement modes are
 * nfield = 2*nvec fields of U (u1, u2 of each mode), stress modes 3*nvec
 * fields of S from bs_stress_coefficients.
 *   Q     : nk*2 doubles, host or device.
 *   coef  : nk x nfield x N complex128 (interleaved), host or device.
 *   out   : nk x nfield x G x G complex64 (interleaved), host or device.
 * The phases are reduced exactly and evaluated in FP64, the two separable
 * contractions in FP32: |error| <= (2(2M+1) + 4) 2^-24 sum_a |coef_a| per
 * point.  1 <= G <= 8192, nfield >= 1.  Asynchronous when coef and out are
 * both device pointers; nk = 0 does nothing.
 */
int bs_mode_field(bs_cell* cell, const double* Q, int nk, int nfield,
                  const double* coef, int G, float* out, void* stream);

/*
 * 3-D cells (the paper's outlook: three displacement and six stress
 * components, 9 (2M+1)^3 unknowns), FP64 path.
 *
 * bs_cell3_desc - a voxelated cubic, tetragonal or any other 3-D cell:
 *   h1, h2, h3 : Cartesian cell vectors (a basis).
 *   P          : voxels per side, 1 <= P <= 128; phase is P x P x P uint16,
 *                phase[p][q][r] with p along h1, q along h2, r along h3
 *                (r fastest); voxel centres ((p+1/2)/P, (q+1/2)/P, (r+1/2)/P).
 *   nphase, lam, mu, rho : isotropic phases (mu > 0, 3 lam + 2 mu > 0, rho > 0).
 *   M          : plane waves |a|, |b|, |c| <= M, 0 <= M <= 5, 2M+1 <= P;
 *                N = (2M+1)^3, n = 3N, wave index (a+M)(2M+1)^2 + (b+M)(2M+1) + c+M.
 * All arrays host or device; the caller keeps ownership.
 */
typedef struct bs_cell3_desc {
    double h1[3];
    double h2[3];
    double h3[3];
    int32_t P;
    const uint16_t* phase;
    int32_t nphase;
    const double* lam;
    const double* mu;
    const double* rho;
    int32_t M;
} bs_cell3_desc;

typedef struct bs_cell3 bs_cell3;

/* bs_create_cell3 - validate and copy a 3-D cell (BS_EINVAL, BS_ENOMEM). Synchronous. */
int bs_create_cell3(const bs_cell3_desc* desc, bs_cell3** out);

/*
 * bs_assemble3 - the k-independent part on `stream`: form factors of
 * 1/(3 lam + 2 mu), 1/mu and rho over the voxels (Eqs. (eo), (ep) with the
 * centroid rule, three separable stages), their Toeplitz Gram blocks and
 * Cholesky factors (the isotropic Phi is block diagonal in the hydrostatic,
 * deviatoric and shear stress directions), and the ten k-monomial matrices
 * of C(k) (their twenty complex N^3 products as exact-slice tensor-core
 * contractions).  A failed Cholesky is reported as BS_ENOTPD by the next
 * synchronising call.
 */
int bs_assemble3(bs_cell3* cell, void* stream);

/*
 * bs_solve_k3 - lowest `nbands` angular frequencies at `nk` wavevectors
 * k = Q1 q^1 + Q2 q^2 + Q3 q^3 (Q: nk x 3 doubles), FP64 Householder
 * reduction and Sturm bisection of C(k) (n = 3N).  omega_out nk x nbands,
 * status_out nk or NULL; host or device.  Requires bs_assemble3
 * (BS_ESTATE); 1 <= nbands <= n.
 */
int bs_solve_k3(bs_cell3* cell, const double* Q, int nk, int nbands, double* omega_out,
                int* status_out, void* stream);

/* bs_form_factors3 - the 3 x D^3 form factors (1/(3 lam + 2 mu), 1/mu, rho),
 * complex, index [f][da+2M][db+2M][dc+2M], D = 4M+1. Synchronises `stream`. */
int bs_form_factors3(bs_cell3* cell, double* out, void* stream);

/* bs_reduced_matrix3 - C(k) (n x n complex, column-major, lower triangle
 * valid) for one wavevector Q (3 doubles). Synchronises `stream`. */
int bs_reduced_matrix3(bs_cell3* cell, const double* Q, double* out, void* stream);

/* bs_cell3_dims - N = (2M+1)^3 and n = 3N of a 3-D cell. */
int bs_cell3_dims(const bs_cell3* cell, int* N, int* n);

/* bs_destroy_cell3 - free a 3-D cell. NULL is a no-op. */
int bs_destroy_cell3(bs_cell3* cell);

/*
 * bs_set_profiling - when `on` is non-zero, bs_assemble and bs_solve_k
 * record CUDA events on their stream around each phase; bs_phase_times
 * then returns the elapsed milliseconds of the most recent call (the last
 * k batch of a multi-batch solve), synchronising on those events:
 *   ms[0] assembly (material table, exponential table, two contractions)
 *   ms[1] Gram blocks (Toeplitz expansion, Cholesky, triangular inverses)
 *   ms[2] k-monomial coefficient matrices
 *   ms[3] per-k builder of C(k)
 *   ms[4] Householder tridiagonalisation
 *   ms[5] bisection and omega
 *   ms[6] FP64 Rayleigh-Ritz refinement (mixed path)
 *   ms[7] the tensor-core contraction of the form factors alone (the
 *         first separable stage of Eqs. (eo), (ep), inside ms[0])
 * Phases that did not run in the last call report 0.
 */
int bs_set_profiling(bs_cell* cell, int on);
int bs_phase_times(bs_cell* cell, double ms[8]);

/*
 * bs_probe_fp64 - a measurement aid, not a step of the method (the paper
 * has no counterpart): the device's FP64 FMA throughput, from a kernel of
 * independent fused multiply-add chains on every SM (`blocks_per_sm` CTAs
 * of 256 threads per SM, `iters` iterations of 8 chains per thread), timed
 * with CUDA events on `stream`.  Writes TFLOP/s (2 flops per FMA) to
 * *tflops.  Synchronises `stream`.  BS_EINVAL for iters < 1 or
 * blocks_per_sm outside [1, 8].
 */
int bs_probe_fp64(int blocks_per_sm, int iters, double* tflops, void* stream);

/*
 * bs_launch_count - number of CUDA kernels this library has launched in
 * the process so far (all cells, all threads).
 */
int bs_launch_count(long long* out);

/* bs_sync - synchronise `stream` and report any deferred error. */
int bs_sync(bs_cell* cell, void* stream);

/* bs_destroy_cell - free the cell and its device storage.  NULL is a no-op. */
int bs_destroy_cell(bs_cell* cell);

/* bs_last_error - message of the last error on the calling thread ("" if none). */
const char* bs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* BANDSTRUCTURE_H */
