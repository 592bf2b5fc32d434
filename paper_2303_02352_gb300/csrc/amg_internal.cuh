// Internal declarations of libamg (GB300, sm_103a).  Not part of the C ABI.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <utility>
#include <cstdio>
#include <string>
#include <vector>

#include "amg.h"

#define AMG_MAXL 40
#define AMG_BLOCK 256

using bf16 = __nv_bfloat16;

// ---------------------------------------------------------------------------
// device buffers: every allocation is rounded up and padded by 256 bytes so
// that vector loads that run past the logical end stay inside the allocation

struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

enum { ST_TIMEOUT = 1, ST_BADPTR = 2, ST_BADCOL = 4, ST_NODIAG = 8, ST_NOTPOS = 16, ST_NAN = 32,
       ST_ASYM = 64 };

// Bounds-checked builds (AMG_CHECKED): every gather index of the solve-phase
// kernels goes through amg_chk, which raises g_amg_bounds and substitutes
// index 0 for an index outside [0, n); the host reports it as AMG_ERR_CUDA.
// In normal builds amg_chk is the identity.
#ifdef AMG_CHECKED
static __device__ int g_amg_bounds = 0;  // one per translation unit; the solve-phase kernels live in solve.cu
#endif
__device__ __forceinline__ int amg_chk(int j, int n) {
#ifdef AMG_CHECKED
  if ((unsigned)j >= (unsigned)n) {
    atomicOr(&g_amg_bounds, 1);
    return 0;
  }
#endif
  return j;
}

// FCG state kept on the device (Alg. 1 scalars and the stop logic)
struct FcgState {
  int it;         // number of updates of u so far
  int done;       // 1: stop launching work (every solve-phase kernel checks it)
  int status;     // amg_status of the solve
  int need_true;  // 1: the next check kernel recomputes r = b - A u
  int maxit;
  int mixed;      // low-precision hierarchy: periodic true residual
  int true_every;
  int precflag;   // 0: B = I (plain CG)
  int timing;     // 1: kernels timed in isolation; no stop bookkeeping, no history writes
  int hist_len;   // entries of hist (maxit + 1)
  double* hist;   // residual history (read through the state so that captured graphs stay valid)
  double tol;
  double nb;      // |b|_2
  double res;     // current |r|/|b|
  double true_res;
  double rho;     // rho_{i-1}
  double a;       // alpha_i / rho_i
  double g;       // gamma_i / rho_{i-1}
};

struct PairCtl;  // paired-pass kernel control word (pair.cuh)

struct Level {
  int n = 0;
  int64_t nnz = 0;
  int maxrow = 0;            // longest row (nonzeros)
  int bw = 0;                // bandwidth: max |i - j| over the stored entries
  int R = 256;               // tile height of the row kernels with this level's V-cycle value type
  int Rd = 256;              // tile height with FP64 values (outer kernels, amg_spmv)
  bool pipe = false;         // every tile fits a pipeline stage (V-cycle value type)
  bool piped = false;        // same with FP64 values
  int sb = 1;                // stage form of the pipelined kernels (1 standard; 2, 4, 5 FP64 long-row forms; 6 two consumer groups)
  int sbd = 1;               // same for the FP64 outer kernels
  int32_t* rp = nullptr;     // CSR (FP64 values)
  int32_t* ci = nullptr;
  double* v = nullptr;
  float* vf = nullptr;       // low-precision copies of the values
  bf16* vb = nullptr;
  double* l1 = nullptr;      // sum_j |a_ij|
  double* omega = nullptr;   // per-row damping (nullptr: 1)
  double* dinv = nullptr;    // omega / l1
  float* dinvf = nullptr;
  int32_t* agg = nullptr;    // row -> row of the next level
  int32_t* mptr = nullptr;   // members of each next-level row (ascending)
  int32_t* mem = nullptr;
  // w-normalised prolongator (prolong_scale = 1): P_{i,agg(i)} = w_i / w^{next}_{agg(i)};
  // nullptr for the unit prolongator
  double* wsv = nullptr;     // smooth vector w of this level (w = 1 on level 0)
  double* pw = nullptr;      // P value of each row (prolongation), n
  double* pwm = nullptr;     // the same values in member order (restriction), n
  float* pwf = nullptr;      // float copies for a low-precision level
  float* pwmf = nullptr;
  // pattern-coded columns (pattern.cu): the column indices of row i are
  // i + ptab[pid[i] * pk + j] for its entries j = 0, 1, ...; rows with the same
  // tuple of column offsets share one table row.  nullptr: CSR columns only.
  uint8_t* pid = nullptr;
  int32_t* ptab = nullptr;
  int32_t* plen = nullptr;   // entries of each tuple
  int32_t* pcb = nullptr;    // row_ptr at every 32nd row, and nnz: ceil(n / 32) + 1 entries
  int npat = 0;              // table rows (distinct offset tuples), at most 255
  int pk = 0;                // entries per table row (the longest row)
  // column form of the pipelined V-cycle row kernels of this level: 0 CSR; 1
  // pattern ids, rows located by row_ptr; 2 pattern ids, rows located from the
  // tuple lengths (forms with one thread per row: a warp's 32 rows start at
  // pcb and follow each other)
  int pat = 0;
  int patd = 0;              // the same for the FP64 outer kernels
  bool stage_rows = true;    // small-stage pattern kernels move row pointers and row vectors by bulk copy
  bool lowp = false;         // this level runs in float inside the V-cycle
  PairCtl* pctl = nullptr;   // paired-pass kernel state (pair.cuh): control word and per-tile counters
  unsigned* pcnt = nullptr;
  // work vectors (double or float according to lowp)
  void* r = nullptr;         // level input (restricted residual), levels > 0
  void* za = nullptr;
  void* zb = nullptr;
  void* t = nullptr;         // residual
  float* r0f = nullptr;      // level 0 low precision: float copy of the FCG residual
  void* e = nullptr;         // W-cycle: first coarse correction of this level (levels > 0)
  void* r2 = nullptr;        // W-cycle: input of the second visit (levels > 0)
};

struct AdjState;  // adjoint work buffers (learned.cu)
struct BotPlan;   // fused-bottom launch arguments (solve.cu)

struct amg_handle {
  amg_params p{};
  cudaStream_t stream = nullptr;  // caller's stream
  cudaStream_t cap = nullptr;     // internal stream used for graph capture
  int nl = 0;
  Level L[AMG_MAXL];
  int npair = 0;
  double setup_ms = 0.0;
  double match_ms = 0.0;      // setup time in the matching steps
  double galerkin_ms = 0.0;   // setup time in the Galerkin products
  double spgemm_ms = 0.0;     // setup time in the general sparse products (w-normalised prolongator)
  // FCG vectors
  double *b = nullptr, *u = nullptr, *r = nullptr, *w = nullptr, *d = nullptr, *v = nullptr,
         *q = nullptr;
  double* partial = nullptr;   // per-block partial sums of the reductions
  unsigned* counter = nullptr; // last-block ticket
  FcgState* st = nullptr;      // device state
  FcgState* st_host = nullptr; // pinned host mirror
  double* hist = nullptr;      // device residual history
  int hist_cap = 0;
  int* dev_flags = nullptr;    // error bits written by kernels
  int* zero_flag = nullptr;    // a device int that stays 0 (skip flag of standalone V-cycles)
  int red_grid = 0;            // persistent grid of the outer row kernels
  int ax_grid = 0;             // grid of the fused axpys
  int use_pipe = 1;            // 0: non-pipelined tiled row kernels
  int use_bottom = 2;          // bottom levels in one cluster launch: 0 never, 1 always (if they fit), 2 where the owner spread says it pays
  int small_rows = 0;          // levels with fewer rows use the non-pipelined tiled kernels
  int min_tpr = 1;             // tuning hook: least threads per row of the pipelined kernels
  int fuse = 1;                // restriction and prolongation fused into the coarse level's first / last sweep
  int use_big = 0;             // long-row form of the FP64 row kernels: 0 (off; measured best), 4 (4x stages, one thread per row), 2, 5
  int use_ng = 1;              // levels with tiles of 32-128 rows in two consumer groups with half the threads per row (sb = 6): 0 none, 1 all kernels (measured best with staged row data and the wait hint), 2 the FP64 outer kernels and pattern-coded float levels only
  int use_stage = 1;           // row data of the small-stage pattern kernels by bulk copy (0: the consumers load it)
  int use_pat = 1;             // pattern-coded columns on levels whose rows fall into at most 255 offset tuples: 0 never, 1 with row pointers (measured best), 2 with rows located from the tuple lengths where one thread takes a row
  int use_pair = 0;            // consecutive row passes in one launch (0 never: measured slower; 1 on levels with room for the lag; 2 always)
  int pair_slack = -1;         // tiles of lag beyond the halo (-1: two rounds of the grid)
  int kb = AMG_MAXL;           // first level of the fused bottom (nl: none)
  BotPlan* bot = nullptr;      // launch arguments of the fused bottom (solve.cu)
  long long suitor_cap = -1;   // test hook: step cap of the matching loop (-1: proof-level bound)
  int fail_alloc_after = -1;   // test hook: the allocation with this index fails (-1: never)
  int n_allocs = 0;
  cudaGraphExec_t g_vcycle = nullptr;
  cudaGraphExec_t g_iter = nullptr;
  cudaGraphExec_t g_iter_cg = nullptr;
  int launches_vcycle = 0;
  int launches_iter = 0;
  int launches_iter_cg = 0;    // kernel launches of one unpreconditioned CG iteration
  int launches_last_solve = 0; // kernel launches of the last solve
  double bytes_vcycle = 0.0;   // algorithmic bytes of one V-cycle
  double bytes_iter = 0.0;     // algorithmic bytes of one FCG iteration
  AdjState* adj = nullptr;     // allocated by the first amg_vcycle_backward
  std::string err;
  std::vector<DBuf> bufs;
};

// ---------------------------------------------------------------------------
// helpers shared by the translation units of the library

amg_status amg_fail(amg_handle* h, amg_status s, const char* fmt, ...);
void* amg_alloc(amg_handle* h, size_t bytes);  // zeroed, padded; nullptr on failure
void amg_free_all(amg_handle* h);
void amg_release(amg_handle* h, void* p);     // frees one allocation of the handle

#define AMG_CK(h, call)                                                                     \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return amg_fail((h), AMG_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));   \
  } while (0)

#define AMG_ALLOC(h, ptr, type, count)                                                      \
  do {                                                                                      \
    (ptr) = (type*)amg_alloc((h), sizeof(type) * (size_t)(count));                          \
    if (!(ptr)) return amg_fail((h), AMG_ERR_OOM, "device allocation of %zu bytes failed",  \
                                sizeof(type) * (size_t)(count));                           \
  } while (0)

static inline int amg_blocks(int64_t threads) { return (int)((threads + AMG_BLOCK - 1) / AMG_BLOCK); }

// consumer threads of the pipelined row kernels and the bytes of one pipeline
// stage (values + column indices), sized per value type so that a tile of a
// 7-point stencil fits with little slack
#ifndef PIPE_CONSUMERS
#define PIPE_CONSUMERS 256
#endif
// largest offset table of a pattern-coded level (entries, pattern.cu): the
// row kernels keep it in shared memory, and 4 KB per block keeps four FP64
// blocks per multiprocessor
#define PAT_TAB_MAX 1024
// suspend-time hint of the row kernels' mbarrier waits (ns): a waiting warp
// sleeps until the phase completes or the hint runs out instead of polling
// through issue slots the working warps need (7-point Poisson 320^3: FP32
// solve 51.3 -> 49.7 ms, BF16 50.8 -> 48.7 ms, FP64 81.5 -> 80.5 ms; 300 ns to
// 10 us measured alike)
#ifndef CSR_STAGE_ROWS
#define CSR_STAGE_ROWS 128  // CSR sweeps and residuals with tiles of at most this many rows stage their row data
#endif
#ifndef MBAR_SUSPEND_NS
#define MBAR_SUSPEND_NS 1000
#endif
#ifndef PIPE_STAGE_SCALE
#define PIPE_STAGE_SCALE 1  // stages are 24/16/12 KB divided by this (FP64/FP32/BF16 values)
#endif
__host__ __device__ constexpr int amg_pipe_tile_bytes(int value_bytes) {
  return (value_bytes >= 8 ? 24576 : (value_bytes >= 4 ? 16384 : 12288)) / PIPE_STAGE_SCALE;
}

// tile height of the row kernels: the largest power of two R <= 256 rows
// (at least rmin) whose longest-row bound fits one pipeline stage
static inline int amg_tile_rows(int maxrow, int value_bytes, int rmin = 32) {
  const int cap = amg_pipe_tile_bytes(value_bytes) / (value_bytes + 4);
  int R = PIPE_CONSUMERS;
  while (R > rmin && (int64_t)R * maxrow > cap) R /= 2;
  return R;
}

void amg_set_setup_error(const std::string& msg);
void amg_adj_destroy(amg_handle* h);             // frees the adjoint bookkeeping (learned.cu)  // message for amg_last_error(NULL)
amg_status amg_level_diag(amg_handle* h, int k);   // l1 norms and D = omega / l1 of level k
// w-normalised prolongators (spgemm.cu): smooth vectors, P values and the
// level matrices P^T A P by the general sparse product, from level 0 down
amg_status amg_normalise_hierarchy(amg_handle* h);
amg_status amg_build_members(amg_handle* h, int k);  // member lists of level k's aggregates (setup.cu)
amg_status amg_member_values(amg_handle* h, int k);  // pwm of level k from pw and the member lists (spgemm.cu)
amg_status amg_finish_setup(amg_handle* h);          // derived data, plan, work vectors, graphs (setup.cu)
amg_status amg_build_patterns(amg_handle* h, int k); // pattern-coded columns of level k where they exist (pattern.cu)
amg_status amg_check_level(amg_handle* h, int k, int nc);  // structure of a level read from a file (setup.cu)
void amg_read_hooks(amg_handle* h);                  // test and tuning hooks from the environment (setup.cu)

int amg_num_sms();  // multiprocessors of the current device

// solve-phase internals (solve.cu)
amg_status amg_prepare_solve(amg_handle* h);
amg_status amg_plan_bottom(amg_handle* h);        // chooses kb and lays out the fused bottom (solve.cu)
void amg_free_bottom(amg_handle* h);
amg_status amg_capture_graphs(amg_handle* h);

// ---------------------------------------------------------------------------
// device-side helpers

// Programmatic dependent launch: a kernel lets the next kernel in the stream
// start early (launch_dependents) and, before it touches data written by the
// previous kernel, waits for that kernel's completion and memory (wait).  Both
// are no-ops for kernels launched without the programmatic attribute.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// launch with the programmatic-serialization attribute when enabled
bool amg_pdl_enabled();
template <typename... KArgs, typename... Args>
static inline cudaError_t amg_launch(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                     Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = amg_pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

__device__ __forceinline__ double to_acc(double x) { return x; }
__device__ __forceinline__ float to_acc(float x) { return x; }
__device__ __forceinline__ float to_acc(bf16 x) { return __bfloat162float(x); }

template <typename T>
struct AccOf { using type = float; };
template <>
struct AccOf<double> { using type = double; };

// mask of the G-lane group that contains this lane (G divides 32)
template <int G>
__device__ __forceinline__ unsigned group_mask() {
  if (G == 32) return 0xffffffffu;
  unsigned lane = threadIdx.x & 31u;
  return ((1u << G) - 1u) << (lane & ~(unsigned)(G - 1));
}

template <int G, typename T>
__device__ __forceinline__ T group_sum(T s) {
  const unsigned m = group_mask<G>();
#pragma unroll
  for (int off = G / 2; off > 0; off >>= 1) s += __shfl_xor_sync(m, s, off);
  return s;
}

// Deterministic block reduction of NV doubles: every thread passes its values;
// on return thread 0 holds the block totals.  All threads of the block must
// call it.  sm must hold 32*NV doubles.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sm) {
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) sm[k * 32 + warp] = v[k];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double x = lane < nw ? sm[k * 32 + lane] : 0.0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
      v[k] = x;
    }
  }
  __syncthreads();
}

// Grid-wide deterministic reduction with the last-block pattern (no waiting):
// each block stores its totals, takes a ticket; the block that takes the last
// ticket sums all partials in a fixed order and returns true with the grid
// totals in v (thread 0).  The counter is reset for the next kernel.
template <int NV>
__device__ __forceinline__ bool grid_sum(double (&v)[NV], double* partial, unsigned* counter, double* sm) {
  __shared__ bool is_last;
  block_sum<NV>(v, sm);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) partial[(size_t)blockIdx.x * NV + k] = v[k];
    __threadfence();
    unsigned t = atomicAdd(counter, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
      x += __ldcg(&partial[(size_t)b * NV + k]);
    v[k] = x;
  }
  block_sum<NV>(v, sm);
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}
