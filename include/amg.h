/*
 * libamg: GB300 (sm_103a) aggregation-based AMG-preconditioned flexible CG.
 *
 * The method is the solver of arXiv:2303.02352 ("BootCMatchGX"): the flexible
 * preconditioned CG of Alg. 1 driven by the V-cycle of Alg. 2 (operator B^k of
 * Sec. 3.1) with l1-Jacobi smoothing (Sec. 3.1), built by the coarsening of
 * Alg. 3 (pairwise aggregation from a half-approximate maximum-weight matching,
 * s pairwise steps composed into aggregates of at most 2^s rows, Galerkin
 * coarse operators).  Every step runs in this library's CUDA kernels on one GPU.
 *
 * Conventions for every entry point:
 *  - Matrices are square CSR with int32 row pointers and column indices,
 *    columns strictly ascending within a row, the diagonal stored, values
 *    float64; the matrix must be symmetric bit for bit (a_ij == a_ji) with a
 *    positive diagonal (SPD is required by the method and not checked beyond).
 *  - "device" pointers are CUDA global-memory pointers on the current device;
 *    "host" pointers are CPU memory (pinned memory makes copies faster).
 *  - All work is enqueued on the stream given to amg_setup (NULL = legacy
 *    default stream).  Every call returns only after that stream has finished
 *    the call's work, unless stated otherwise.
 *  - The caller owns all buffers it passes; the library copies what it keeps.
 *    The handle owns the hierarchy, work vectors and CUDA graphs until
 *    amg_destroy.  A handle must not be used by two threads at once.
 *  - Errors are returned as negative amg_status codes; no exception crosses the
 *    ABI.  amg_last_error gives a one-line description of the last failure.
 */
#ifndef AMG_H
#define AMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  AMG_OK = 0,
  AMG_NOT_CONVERGED = 1,     /* maxit reached; x and the history are still valid */
  AMG_ERR_INVALID_ARG = -1,  /* bad pointer, size, or matrix structure */
  AMG_ERR_NOT_SPD = -2,      /* non-positive diagonal */
  AMG_ERR_BREAKDOWN = -3,    /* rho <= 0 or not finite in Alg. 1; x holds the last good iterate */
  AMG_ERR_CUDA = -4,         /* a CUDA runtime call failed */
  AMG_ERR_OOM = -5,          /* device allocation failed */
  AMG_ERR_TIMEOUT = -6,      /* a bounded device loop hit its iteration cap */
  AMG_ERR_TOO_LARGE = -7     /* size beyond what an entry point supports */
} amg_status;

typedef enum { AMG_FP64 = 0, AMG_FP32 = 1, AMG_FP32_BF16FINE = 2 } amg_precision;

/* CSR matrix in device memory (see conventions above). */
typedef struct {
  int32_t n;
  int32_t nnz;
  const int32_t* row_ptr; /* device, n+1 */
  const int32_t* col_idx; /* device, nnz */
  const double* val;      /* device, nnz */
} amg_csr;

/* Parameters; amg_params_default gives the settings of Sec. 5 / Listing 1. */
typedef struct {
  int32_t aggr_steps;     /* s: pairwise matching steps composed per level (3 -> aggregates <= 8) */
  int32_t max_levels;     /* maximum number of hierarchy levels (39) */
  int32_t coarse_size;    /* stop coarsening once n <= coarse_size; 0 -> 40*round(cbrt(n)) */
  int32_t pre_sweeps;     /* l1-Jacobi pre-smoothing sweeps (4) */
  int32_t post_sweeps;    /* l1-Jacobi post-smoothing sweeps (4) */
  int32_t coarse_sweeps;  /* l1-Jacobi sweeps on the coarsest level (20) */
  int32_t precision;      /* amg_precision of the hierarchy inside the V-cycle (AMG_FP64) */
  int32_t true_res_every; /* low precision: r <- b - A u every k iterations (50); 0 = never */
  int32_t use_graph;      /* 1: replay the V-cycle and the FCG iteration as CUDA graphs (1) */
  int32_t graph_batch;    /* FCG iterations launched before the first convergence read (4); later reads
                             follow the observed convergence factor (1: a read after every iteration) */
  int32_t num_parts;      /* decoupled aggregation (Sec. 4.1): match only inside this many
                             contiguous row blocks, as np tasks would (1 = global matching) */
  int32_t cycle;          /* Listing 1 cycle_type: 0 V-cycle, 2 W-cycle (0) */
  int32_t relax_type;     /* Listing 1 relax_type: 4 l1-Jacobi, D = omega / sum_j |a_ij| (4);
                             0 Jacobi, D = omega / a_ii; every level including the coarsest */
  int32_t prolong_scale;  /* prolongator values (Sec. 3.1: they follow the smooth vector w,
                             w_next = P^T w): 0 unit entries, P 1 = 1 (0); 1 w-normalised
                             entries w_i / |w on the aggregate|, P^T P = I, with the level matrices
                             formed by the general sparse product amg_spgemm (Alg. 4's local
                             product); the aggregates are the same in both forms */
} amg_params;

typedef struct {
  int32_t num_levels;
  int32_t n[40];          /* rows per level */
  int64_t nnz[40];        /* nonzeros per level */
  double opc;             /* operator complexity: sum nnz / nnz of level 0 (Sec. 5) */
  int32_t num_pairwise;   /* pairwise matching steps performed in the setup */
  double setup_ms;        /* wall time of amg_setup */
  double vcycle_bytes;    /* algorithmic bytes one V-cycle moves (each kernel's reads and writes) */
  double iteration_bytes; /* algorithmic bytes of one FCG iteration (V-cycle + outer kernels) */
  int32_t vcycle_launches;    /* kernel launches of one V-cycle */
  int32_t iteration_launches; /* kernel launches of one FCG iteration */
  int32_t precision;          /* amg_precision of the hierarchy */
  double setup_match_ms;      /* setup time in the matching steps (weights, suitor, aggregation) */
  double setup_galerkin_ms;   /* setup time in the Galerkin products */
  int32_t bottom_level;       /* first level of the fused bottom (one cluster launch); num_levels: none */
  int32_t tile_rows[40];      /* rows per tile of the level's pipelined row kernels (0: non-pipelined) */
  int32_t stage_scale[40];    /* pipeline stage size of those kernels in units of the standard stage */
  double setup_spgemm_ms;     /* setup time in the general sparse products (prolong_scale = 1) */
  int32_t last_solve_launches; /* kernel launches of the last solve on the handle (0 before any) */
  int32_t consumer_groups[40];  /* groups of consumer warps taking a level's tiles in turn (0: non-pipelined) */
  int32_t column_patterns[40];  /* distinct column-offset tuples of a level whose V-cycle row kernels read
                                   pattern-coded columns (a one-byte tuple id per row instead of a 4-byte
                                   column index per entry; same entries and arithmetic); 0: CSR columns */
  int32_t outer_patterns;       /* the same for the FP64 outer kernels on level 0 */
  int32_t column_form[40];      /* 0 CSR columns; 1 pattern ids, rows located by row pointers; 2 pattern
                                   ids, rows located from the tuple lengths and one row pointer per 32
                                   rows (kernel forms with one thread per row) */
  int32_t outer_column_form;    /* the same for the FP64 outer kernels on level 0 */
} amg_info_t;

typedef struct amg_handle amg_handle;

/* Fills *p with the defaults above (the settings of Sec. 5 and Listing 1). */
void amg_params_default(amg_params* p);

/*
 * Builds the hierarchy on the GPU (Alg. 3, Sec. 3.1): matching weights, suitor
 * matching with an index tie-break, pairwise aggregation, Galerkin products,
 * s-fold composition, l1-Jacobi diagonals, low-precision copies.  It also
 * stores, for each level of at least 32,768 rows whose rows fall into at most
 * 255 distinct tuples of column offsets, a one-byte tuple id per row that the
 * solve-phase row kernels read instead of the column indices (the same
 * matrix: entries, order and results unchanged; amg_info_t column_patterns).
 * A: device CSR, read during the call only (deep-copied).  p: NULL = defaults.
 * stream: a cudaStream_t (may be NULL).  *out receives the handle.
 * Errors: AMG_ERR_INVALID_ARG (structure, asymmetry, NaN), AMG_ERR_NOT_SPD
 * (diagonal <= 0), AMG_ERR_OOM, AMG_ERR_CUDA, AMG_ERR_TIMEOUT.
 */
amg_status amg_setup(const amg_csr* A, const amg_params* p, void* stream, amg_handle** out);

/*
 * Alg. 1 (flexible PCG, one V-cycle per iteration) on A u = b.
 * b: device, n.  x: device, n; in: initial guess u_0, out: solution.
 * Stops when |r|_2/|b|_2 < tol after an update (confirmed on the true residual
 * b - A u) or after maxit iterations.  iters (host, may be NULL): number of
 * updates of u.  res_hist (host, may be NULL, length maxit+1): |r_i|/|b| for
 * i = 0..iters.  true_rel_res (host, may be NULL): |b - A u|/|b| at exit.
 * Returns AMG_OK, AMG_NOT_CONVERGED, AMG_ERR_BREAKDOWN or an error.
 */
amg_status amg_pcg_solve(amg_handle* h, const double* b, double* x, double tol, int32_t maxit,
                         int32_t* iters, double* res_hist, double* true_rel_res);

/* Alg. 1 as amg_pcg_solve, with b and x in host memory: the host-to-device copy
 * of b and x and the device-to-host copy of x are part of the call. */
amg_status amg_pcg_solve_host(amg_handle* h, const double* b_host, double* x_host, double tol,
                              int32_t maxit, int32_t* iters, double* res_hist, double* true_rel_res);

/* Plain CG (Alg. 1 with B = I, the paper's precflag = 0); same arguments. */
amg_status amg_cg_solve(amg_handle* h, const double* b, double* x, double tol, int32_t maxit,
                        int32_t* iters, double* res_hist, double* true_rel_res);

/* One application of the preconditioner, z = B r (Alg. 2).  r, z: device, n,
 * distinct buffers. */
amg_status amg_vcycle(amg_handle* h, const double* r, double* z);

/* y = A^k x for hierarchy level k (A^0 = A; A^{k+1} the Galerkin operator of
 * Alg. 3 / Sec. 3.1).  x, y: device, n_k, distinct buffers. */
amg_status amg_spmv(amg_handle* h, int32_t level, const double* x, double* y);

/* Hierarchy summary (host struct): levels, sizes and the operator complexity
 * the paper reports (Sec. 5), setup timings, kernel forms. */
amg_status amg_info(const amg_handle* h, amg_info_t* info);

/* Copies of the hierarchy to host memory.  agg_host: n_k ints, the level-k row
 * -> level-(k+1) row map (level < num_levels-1): the aggregates of Alg. 3
 * composed over the s pairwise steps of a level (Sec. 3.1), i.e. the column
 * of the prolongator's single unit entry in each row.  CSR: n_k+1, nnz_k,
 * nnz_k (the level matrix A^k). */
amg_status amg_get_aggregates(amg_handle* h, int32_t level, int32_t* agg_host);
amg_status amg_get_level_csr(amg_handle* h, int32_t level, int32_t* row_ptr_host,
                             int32_t* col_idx_host, double* val_host);
/* l1 row norms M_ii = sum_j |a_ij| of level k, the l1-Jacobi diagonal of
 * Sec. 3.1 (host, n_k doubles). */
amg_status amg_get_l1(amg_handle* h, int32_t level, double* l1_host);

/*
 * Measurement helpers (for benchmarking; results in milliseconds).
 * amg_time_vcycle: average time of one V-cycle over reps replays.
 * amg_time_kernel: average duration of one launch of kernel `which` on `level`
 *   over reps launches, timed with CUDA events on the handle's stream:
 *   0 = l1-Jacobi sweep, 1 = residual, 2 = restriction, 3 = prolongation,
 *   4 = outer SpMV fused with the dot products, 5 = fused axpys,
 *   6 = restriction from `level` fused with the first sweep of level+1,
 *   7 = l1-Jacobi sweep of level+1 fused with the prolongation into `level`
 *   (6 and 7 are the forms the V-cycle launches; 2 and 3 the unfused ones),
 *   8 = two l1-Jacobi sweeps of `level` in one launch (the second pass reads
 *   the matrix tiles the first pass brought into L2).
 * amg_kernel_bytes of 8 counts the matrix once (the bytes that must move).
 */
amg_status amg_time_vcycle(amg_handle* h, int32_t reps, double* ms);
amg_status amg_time_kernel(amg_handle* h, int32_t which, int32_t level, int32_t reps, double* ms);
/* bytes: host double; the algorithmic bytes of one launch of `which` on `level`
 * (values, column indices, row pointers and vector entries each counted once). */
amg_status amg_kernel_bytes(const amg_handle* h, int32_t which, int32_t level, double* bytes);
/*
 * Learned l1-Jacobi damping (not in the paper; a network gives each row of
 * each level a damping omega_i in (0, 2) with D_i = omega_i / M_ii, where
 * M_ii = sum_j |a_ij| is the l1-Jacobi diagonal of Sec. 3.1).
 *
 * amg_features: the four features of every row of `level`, row-major n_k x 4
 *   float (device): a_ii / M_ii, ln M_ii minus the mean of ln M_jj over the
 *   row's columns, nnz_i / 27, level / 4.
 * amg_set_omega: sets omega on `level` (device, n_k doubles; NULL = 1, plain
 *   l1-Jacobi) and recomputes D.  Solves and V-cycles use it until changed.
 * amg_mlp_forward: omega (device, n doubles) = 2 sigmoid(W3 relu(W2 relu(W1 f
 *   + b1) + b2) + b3) from feats (device, n x 4 float) and the 1249 bf16
 *   weights w (device, layout [W1 32x4, b1 32, W2 32x32, b2 32, W3 32, b3]);
 *   float32 arithmetic.  Enqueued on `stream`, not synchronised.
 * amg_mlp_backward: grad (device, 1249 floats) = d(sum_i domega_i omega_i)/dw
 *   for the same inputs; deterministic.  workspace: device memory of
 *   amg_mlp_workspace_bytes(n) bytes.  Enqueued on `stream`.
 * amg_adam_step: one Adam update of the float32 master weights theta (device)
 *   with moments m, v (device), step t >= 1; writes the bf16 copy w_bf16.
 * amg_apply_mlp: features + network + amg_set_omega on every level of the
 *   handle (w_bf16 NULL: back to omega = 1).
 * amg_vcycle_backward: adjoint of one FP64 V-cycle z = B(omega) r: given r and
 *   dz = dL/dz (device, n), writes dr = dL/dr (device, n) and, for every level
 *   k, domega[k] (device, n_k doubles) = dL/domega.  Recomputes each level's
 *   sweeps from the level's input instead of storing them (work buffers are
 *   allocated by the first call and kept by the handle).
 */
amg_status amg_features(amg_handle* h, int32_t level, float* feats);
amg_status amg_set_omega(amg_handle* h, int32_t level, const double* omega);
size_t amg_mlp_workspace_bytes(int32_t n);
amg_status amg_mlp_forward(int32_t n, const float* feats, const uint16_t* w_bf16, double* omega, void* stream);
amg_status amg_mlp_backward(int32_t n, const float* feats, const uint16_t* w_bf16, const double* domega,
                            float* grad, void* workspace, void* stream);
amg_status amg_adam_step(int32_t np, float* theta, const float* grad, float* m, float* v, uint16_t* w_bf16,
                         float lr, float beta1, float beta2, float eps, int32_t t, void* stream);
amg_status amg_apply_mlp(amg_handle* h, const uint16_t* w_bf16);
amg_status amg_vcycle_backward(amg_handle* h, const double* r, const double* dz, double* dr,
                               double* const* domega);
/* amg_vcycle_loss: the training loss of the damping, L = (1/m) ln(|r_m| / |r_0|)
 *   with r_{t+1} = r_t - A B(omega) r_t (m steps of the stationary iteration of
 *   the FP64 V-cycle on level 0), into *loss (host); with domega not NULL also
 *   dL/domega for every level k (device, n_k doubles each, overwritten), by the
 *   adjoint of the m steps (dL/dr_m = r_m / (m |r_m|^2); each step back takes
 *   dL/dz_t = -A dL/dr_{t+1} through amg_vcycle_backward's adjoint).  r0:
 *   device, n, not zero.  V-cycle, l1-Jacobi and unit prolongators only
 *   (AMG_ERR_INVALID_ARG otherwise).  Work buffers are kept by the handle. */
amg_status amg_vcycle_loss(amg_handle* h, const double* r0, int32_t m, double* loss, double* const* domega);

/*
 * Residual check that allocates nothing (the paper has no counterpart; this is
 * an addition of the library).  For callers that may not call cudaMalloc or
 * cudaFree themselves, such as a component whose host owns all device memory
 * through its own allocator, or a loop that cannot afford the synchronisation
 * an allocation may cause.  Computes norms[0] = |b - A x|_2 and
 * norms[1] = |b|_2, and r = b - A x when r is not NULL.
 * A: device CSR (as for amg_setup; symmetry is not needed).  b, x: device, n.
 * r: device, n, or NULL.  norms: device, 2 doubles.  stream: a cudaStream_t.
 * The work is only enqueued: results are ready once the stream reaches it.
 * Scratch space is a fixed device array inside the library (about 128 KB per
 * GPU, held until the process exits), which bounds n to 2,097,152 rows; larger
 * n returns AMG_ERR_TOO_LARGE.  The first call on a device looks up the array's
 * address; make that first call before any stream capture.  Every call reuses
 * the same array: calls whose work overlaps on the GPU race and give wrong
 * results.  Errors: AMG_ERR_INVALID_ARG, AMG_ERR_TOO_LARGE, AMG_ERR_CUDA;
 * amg_last_error(NULL) describes them.
 */
amg_status amg_residual_norm_noalloc(const amg_csr* A, const double* b, const double* x, double* r,
                                     double* norms, void* stream);

/*
 * General sparse matrix product C = A B (Sec. 4.2 / Alg. 4 form every coarse
 * matrix with such a product; this library uses it for the w-normalised
 * prolongators, prolong_scale = 1).  A: m x k, B: k x n, device CSR with int32
 * row pointers and column indices; the columns of every row of B strictly
 * ascending (A's rows may be in any order).  Two calls on the same inputs:
 *  1. c_col_idx = c_val = NULL: writes C's row pointers (device, m+1 ints) and
 *     *nnz_c (host) = the number of entries of C (symbolic phase);
 *  2. c_row_ptr from call 1, c_col_idx and c_val (device, nnz_c each): writes
 *     the columns (ascending in every row) and the values (numeric phase).
 * Every structurally present product is kept (an entry whose products cancel
 * is stored as 0).  Each entry sums its products in a fixed order (the
 * results are bitwise reproducible).  Scratch is taken from the stream-ordered
 * allocator for the call; the call synchronises `stream` before returning.
 * Errors: AMG_ERR_INVALID_ARG (sizes, NULL pointers; in call 1 also row
 * pointers not monotone, a column out of range or a row of B not strictly
 * ascending), AMG_ERR_OOM, AMG_ERR_CUDA; amg_last_error(NULL) describes them.
 */
amg_status amg_spgemm(int32_t m, int32_t k, int32_t n, const int32_t* a_row_ptr, const int32_t* a_col_idx,
                      const double* a_val, const int32_t* b_row_ptr, const int32_t* b_col_idx, const double* b_val,
                      int32_t* c_row_ptr, int32_t* c_col_idx, double* c_val, int64_t* nnz_c, void* stream);

/*
 * Problem generators on the device (the paper's library generates the
 * benchmark matrix on each process, Sec. 5 / App. A).  The N^3 grid's
 * unknowns are numbered x + N y + N^2 z, Dirichlet unknowns eliminated.
 * amg_stencil_size: *n = N^3 rows and *nnz entries of the points-point
 *   stencil (points 7 or 27; N >= 3; nnz below 2^31, else AMG_ERR_INVALID_ARG).
 * amg_generate_stencil: writes that CSR into caller-allocated device arrays
 *   (row_ptr n+1, col_idx nnz, val nnz; columns ascending).  kblock NULL (7
 *   points only): the integer Poisson stencil (6 on the diagonal, -1 off it).
 *   Otherwise kblock (host, ceil(N/block)^3 float32, x fastest) gives the
 *   coefficient of each block of block^3 cells; a link is
 *   2 k_i k_j / (k_i + k_j) divided by |d|^2 off the axes, negated off the
 *   diagonal, a link leaving the grid counts k_i, the diagonal sums the links
 *   of its row in column order; every operation rounded on its own.  The call
 *   synchronises stream (kblock is read during the call).
 * amg_random_vector: out (device, n) = 2 U_i - 1, U_i the top 53 bits of
 *   output i of SplitMix64 seeded with seed, times 2^-53.  Enqueued on stream.
 * amg_csr_times: y = A x (device; A as amg_csr, square), each row's products
 *   rounded and summed in column order from the first.  Enqueued on stream.
 * Errors: AMG_ERR_INVALID_ARG, AMG_ERR_OOM, AMG_ERR_CUDA; amg_last_error(NULL).
 */
amg_status amg_stencil_size(int32_t N, int32_t points, int64_t* n, int64_t* nnz);
amg_status amg_generate_stencil(int32_t N, int32_t points, const float* kblock, int32_t block, int32_t* row_ptr,
                                int32_t* col_idx, double* val, void* stream);
amg_status amg_random_vector(int64_t n, uint64_t seed, double* out, void* stream);
amg_status amg_csr_times(const amg_csr* A, const double* x, double* y, void* stream);

/* Self-check of the bounded device waits: launches one block that waits on a
 * barrier phase nothing completes, with a limit of limit_us microseconds
 * (1 .. 2,000,000).  Returns AMG_ERR_TIMEOUT when the wait gave up and
 * reported as designed (the expected result), AMG_OK if it did not. */
amg_status amg_check_bounded_wait(int32_t limit_us, void* stream);

/*
 * Saving a built hierarchy and loading it back (the paper keeps one setup for
 * many solves, Sec. 5.2; a file lets it outlive the process).
 * amg_save: writes the level matrices, aggregation maps, dampings (and for
 *   prolong_scale = 1 the smooth vectors and prolongator values) of h to the
 *   file at path (created or replaced).  Errors: AMG_ERR_INVALID_ARG (cannot
 *   open), AMG_ERR_CUDA (write or device copy failed).
 * amg_load: builds a handle from such a file without matching or Galerkin
 *   products; the rest (member lists, diagonals, low-precision copies, kernel
 *   forms, work vectors, graphs) is derived as in amg_setup, so the handle
 *   computes bit for bit what the saved one did.  p: NULL = the saved
 *   parameters; otherwise the solve-phase fields are taken from p (sweeps,
 *   precision, true_res_every, use_graph, graph_batch, cycle, relax_type) and
 *   aggr_steps, max_levels, coarse_size, num_parts, prolong_scale must equal
 *   the saved ones.  stream: as for amg_setup.  The file is checked like a
 *   caller's matrix (structure, diagonal, finite values, maps in range).
 *   Errors: AMG_ERR_INVALID_ARG (missing, foreign, truncated or corrupt file,
 *   mismatching parameters), AMG_ERR_NOT_SPD, AMG_ERR_OOM, AMG_ERR_CUDA;
 *   amg_last_error(NULL) describes them.
 */
amg_status amg_save(const amg_handle* h, const char* path);
amg_status amg_load(const char* path, const amg_params* p, void* stream, amg_handle** out);
/* The parameter block stored in a saved hierarchy (host, *out); the start of
 * a p for amg_load that changes only solve-phase fields.  AMG_ERR_INVALID_ARG
 * if the file cannot be read as a saved hierarchy. */
amg_status amg_saved_params(const char* path, amg_params* out);

/* Last error message of the handle (or of the last failed amg_setup if h is NULL). */
const char* amg_last_error(const amg_handle* h);

/* Frees everything the handle owns.  NULL is ignored. */
void amg_destroy(amg_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* AMG_H */
