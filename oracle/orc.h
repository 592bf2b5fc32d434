/*
 * CPU oracle for the aggregation-based AMG-preconditioned flexible CG of
 * arXiv:2303.02352 (BootCMatchGX).  TEST INFRASTRUCTURE ONLY: plain, serial,
 * slow FP64 C that the test-suite, the smoke check and the CPU-baseline leg of
 * the benchmark call to check the CUDA library.  Nothing in the product path
 * may link, load or call it.  It shares no code with the CUDA library.
 *
 * Follows: Alg. 1 (flexible PCG), Alg. 2 and the operator B^k of Sec. 3.1
 * (V-cycle), Alg. 3 (coarsening by maximum-weight matching) and the
 * composition of s pairwise prolongators (Sec. 3.1, "more aggressive
 * coarsening"), the l1-Jacobi smoother (Sec. 3.1) and the experimental
 * settings of Sec. 5 / Listing 1 (4+4 sweeps, 20 coarse sweeps, aggregates of
 * at most 8, coarsest size 40*nd, rtol 1e-6, 1000 iterations).
 *
 * The same source is built twice: serially (the checker the tests use; the
 * OpenMP pragmas are ignored) and with -fopenmp as the timed CPU baseline,
 * where the row loops of the SpMV, the sweeps, the residuals, the
 * prolongation, the dot products and the axpys of Alg. 1 are split statically
 * over the host's cores (the dot products then sum in another order; the
 * setup and the restriction stay serial).
 */
#ifndef ORC_H
#define ORC_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_NOT_CONVERGED = 1, ORC_ERR_ARG = -1, ORC_ERR_BREAKDOWN = -3 };
enum { ORC_COARSE_L1JACOBI = 0, ORC_COARSE_DENSE_CHOL = 1 };
enum { ORC_FP64 = 0, ORC_FP32 = 1, ORC_FP32_BF16FINE = 2 };
enum { ORC_PROLONG_UNIT = 0, ORC_PROLONG_W_NORMALIZED = 1 };

typedef struct orc_params {
  int aggr_steps;      /* s: pairwise steps merged per level (3 -> aggregates <= 8) */
  int max_levels;      /* cap on hierarchy levels (39) */
  int coarse_size;     /* stop coarsening at n <= coarse_size; 0 -> 40*round(cbrt(n)) */
  int pre_sweeps;      /* l1-Jacobi pre-smoothing sweeps (4) */
  int post_sweeps;     /* l1-Jacobi post-smoothing sweeps (4) */
  int coarse_sweeps;   /* l1-Jacobi sweeps on the coarsest level (20) */
  int coarse_solver;   /* ORC_COARSE_L1JACOBI or ORC_COARSE_DENSE_CHOL (exact, pins only) */
  int precision;       /* ORC_FP64 / ORC_FP32 / ORC_FP32_BF16FINE hierarchy emulation */
  int true_res_every;  /* mixed precision: replace r by b - A u every k iterations (50) */
  int num_parts;       /* decoupled aggregation (Sec. 4.1): matching inside np row blocks (1) */
  int cycle;           /* Listing 1 cycle_type: 0 V-cycle, 2 W-cycle (0) */
  int relax_type;      /* Listing 1 relax_type: 4 l1-Jacobi M_ii = sum_j |a_ij| (4), 0 Jacobi M_ii = a_ii;
                          the same relaxation on the coarsest level */
  int prolong_scale;   /* ORC_PROLONG_UNIT (P 1 = 1, the default) or ORC_PROLONG_W_NORMALIZED
                          (entries w_i / |w_aggregate|, P^T P = I; ablation of the prolongator
                          values of Sec. 3.1, oracle only) */
} orc_params;

typedef struct orc_hier orc_hier;

void orc_params_default(orc_params* p);

/* single steps (exposed for pins) */
int orc_weights(int n, const int32_t* rp, const int32_t* ci, const double* v, double* wgt);
/* weights restricted to the row blocks [bnd[p], bnd[p+1]) (edges across blocks get 0) */
int orc_weights_parts(int n, const int32_t* rp, const int32_t* ci, const double* v, int np, const int32_t* bnd,
                      double* wgt);
int orc_match_greedy(int n, const int32_t* rp, const int32_t* ci, const double* wgt, int32_t* mate);
int orc_aggregate(int n, const int32_t* mate, int32_t* agg);
/* Galerkin: first call with out arrays NULL returns nnz_c; second fills them */
int64_t orc_galerkin(int n, const int32_t* rp, const int32_t* ci, const double* v,
                     const int32_t* agg, int nc, int32_t* rp_c, int32_t* ci_c, double* v_c);

/* hierarchy */
orc_hier* orc_setup(int n, const int32_t* rp, const int32_t* ci, const double* v, const orc_params* p);
void orc_free(orc_hier* h);
int orc_num_levels(const orc_hier* h);
int orc_level_n(const orc_hier* h, int k);
int64_t orc_level_nnz(const orc_hier* h, int k);
void orc_level_csr(const orc_hier* h, int k, int32_t* rp, int32_t* ci, double* v);
void orc_level_agg(const orc_hier* h, int k, int32_t* agg);
void orc_level_l1(const orc_hier* h, int k, double* l1);
int orc_num_pairwise(const orc_hier* h);
int orc_pairwise_n(const orc_hier* h, int t);
int orc_set_omega(orc_hier* h, int k, const double* omega);

/* solve phase */
void orc_vcycle(orc_hier* h, const double* r, double* z);
int orc_fcg(orc_hier* h, const double* b, double* u, double tol, int maxit, int precflag,
            int* iters, double* hist, double* true_rel);
void orc_spmv(const orc_hier* h, int k, const double* x, double* y);

/* learned smoother: loss (1/m) ln(|r_m|/|r_0|), r_{t+1} = r_t - A B r_t, and its
 * gradient with respect to every per-row damping omega of every level (l1-Jacobi
 * V-cycle only: NaN for another relaxation or cycle) */
double orc_vcycle_loss(orc_hier* h, const double* r0, int m);
double orc_vcycle_loss_grad(orc_hier* h, const double* r0, int m, double* const* domega);

/* threads the row loops use: 1 in the serial build */
int orc_threads(void);

/* plain helpers for bf16 emulation (used by tests) */
float orc_round_bf16(float x);

#ifdef __cplusplus
}
#endif
#endif
