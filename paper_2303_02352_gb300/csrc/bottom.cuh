// The bottom of the V-cycle in one launch (included by solve.cu).
//
// Levels with few rows (at most BOT_MAX_ROWS) do so little work per pass that a
// kernel launch per pass costs more than the pass.  One thread-block cluster
// runs all of them: the down-sweep (pre-smoothing, residual, restriction) of
// each bottom level, the coarsest level's sweeps, and the up-sweep
// (prolongation, post-smoothing), with a hardware cluster barrier between
// passes (barrier.cluster with release/acquire ordering, so one pass's global
// writes are visible to the next pass in every block of the cluster; no
// spinning).  The matrices stay in L2.  Vectors written inside the kernel are
// read with coherent loads, never through the read-only path.
#pragma once

#include <cooperative_groups.h>

#include "amg_internal.cuh"

#define BOT_MAXL 8
#define BOT_THREADS 1024
#define BOT_MAX_ROWS 16384

struct BotLevel {
  int n;
  const int32_t* rp;
  const int32_t* ci;
  const void* v;      // level value type (double on the coarsest level)
  const void* dinv;
  const int32_t* agg;  // to the next bottom level
  const int32_t* mptr;
  const int32_t* mem;
  void* r;             // level input
  void* za;            // result ends here
  void* zb;
  void* t;
};

struct BotArgs {
  int nb;  // number of bottom levels; the last one is the coarsest
  BotLevel L[BOT_MAXL];
  int pre, post, csweeps;
  const int* skip;
};

__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

template <typename MT, typename VT>
__device__ __forceinline__ VT bot_row_dot(const BotLevel& L, const VT* x, int i) {
  const MT* v = (const MT*)L.v;
  VT s = 0;
  for (int p = L.rp[i]; p < L.rp[i + 1]; ++p) s += (VT)to_acc(v[p]) * x[L.ci[p]];
  return s;
}

// one pass over the rows of a level, rows distributed over the whole cluster
#define BOT_ROWS(L, ...)                  \
  for (int i = g; i < (L).n; i += G) {    \
    __VA_ARGS__;                          \
  }                                       \
  cluster_barrier();

// smoothing from zero: `sweeps` l1-Jacobi sweeps; returns the buffer holding z
template <typename MT, typename VT>
__device__ VT* bot_smooth_zero(const BotLevel& L, const VT* r, int sweeps, int g, int G) {
  VT* za = (VT*)L.za;
  VT* zb = (VT*)L.zb;
  const VT* D = (const VT*)L.dinv;
  if (sweeps <= 0) {
    BOT_ROWS(L, za[i] = (VT)0);
    return za;
  }
  BOT_ROWS(L, za[i] = D[i] * r[i]);
  VT* cur = za;
  for (int s = 1; s < sweeps; ++s) {
    VT* nxt = cur == za ? zb : za;
    BOT_ROWS(L, nxt[i] = cur[i] + D[i] * (r[i] - bot_row_dot<MT, VT>(L, cur, i)));
    cur = nxt;
  }
  return cur;
}

template <typename MT, typename VT>
__device__ VT* bot_smooth_from(const BotLevel& L, const VT* r, VT* cur, int sweeps, int g, int G) {
  VT* za = (VT*)L.za;
  VT* zb = (VT*)L.zb;
  const VT* D = (const VT*)L.dinv;
  for (int s = 0; s < sweeps; ++s) {
    VT* nxt = cur == za ? zb : za;
    BOT_ROWS(L, nxt[i] = cur[i] + D[i] * (r[i] - bot_row_dot<MT, VT>(L, cur, i)));
    cur = nxt;
  }
  return cur;
}

// MT/VT: value and vector types of the bottom levels above the coarsest one;
// the coarsest level runs in FP64.  The result of bottom level 0 is left in
// its za buffer.
template <typename MT, typename VT>
__global__ void __launch_bounds__(BOT_THREADS) k_bottom(const __grid_constant__ BotArgs a) {
  if (*a.skip) return;
  namespace cg = cooperative_groups;
  const int g = (int)(cg::this_cluster().block_rank() * blockDim.x + threadIdx.x);
  const int G = (int)(cg::this_cluster().num_blocks() * blockDim.x);
  const int nb = a.nb;
  VT* res[BOT_MAXL];  // pre-smoothing results of the levels above the coarsest
  // down-sweep
  for (int k = 0; k < nb - 1; ++k) {
    const BotLevel& L = a.L[k];
    const VT* r = (const VT*)L.r;
    VT* z = bot_smooth_zero<MT, VT>(L, r, a.pre, g, G);
    VT* t = (VT*)L.t;
    BOT_ROWS(L, t[i] = r[i] - bot_row_dot<MT, VT>(L, z, i));
    const BotLevel& C = a.L[k + 1];
    if (k + 1 == nb - 1) {
      double* rc = (double*)C.r;
      BOT_ROWS(C, { VT s = 0; for (int m = L.mptr[i]; m < L.mptr[i + 1]; ++m) s += t[L.mem[m]]; rc[i] = (double)s; });
    } else {
      VT* rc = (VT*)C.r;
      BOT_ROWS(C, { VT s = 0; for (int m = L.mptr[i]; m < L.mptr[i + 1]; ++m) s += t[L.mem[m]]; rc[i] = s; });
    }
    res[k] = z;
  }
  // coarsest level (FP64)
  const BotLevel& Lc = a.L[nb - 1];
  double* zc = bot_smooth_zero<double, double>(Lc, (const double*)Lc.r, a.csweeps, g, G);
  // up-sweep
  for (int k = nb - 2; k >= 0; --k) {
    const BotLevel& L = a.L[k];
    VT* z = res[k];
    if (k + 1 == nb - 1) {
      const double* zcc = zc;
      BOT_ROWS(L, z[i] += (VT)zcc[L.agg[i]]);
    } else {
      const VT* zcc = (const VT*)a.L[k + 1].za;
      BOT_ROWS(L, z[i] += zcc[L.agg[i]]);
    }
    z = bot_smooth_from<MT, VT>(L, (const VT*)L.r, z, a.post, g, G);
    if (z != (VT*)L.za) {
      VT* za = (VT*)L.za;
      BOT_ROWS(L, za[i] = z[i]);
    }
  }
  if (nb == 1 && zc != (double*)Lc.za) {
    double* za = (double*)Lc.za;
    BOT_ROWS(Lc, za[i] = zc[i]);
  }
}

// cluster size of the bottom kernel: 16 blocks when the part allows it, else 8
template <typename MT, typename VT>
static int bottom_cluster_size() {
  static int cs = 0;
  if (cs) return cs;
  auto kern = k_bottom<MT, VT>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  for (int want : {16, 8}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(want);
    cfg.blockDim = dim3(BOT_THREADS);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = want;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) == cudaSuccess && clusters > 0) {
      cs = want;
      return cs;
    }
    cudaGetLastError();
  }
  cs = 8;
  return cs;
}

template <typename MT, typename VT>
static cudaError_t launch_bottom(cudaStream_t s, const BotArgs& a) {
  const int cs = bottom_cluster_size<MT, VT>();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(BOT_THREADS);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_bottom<MT, VT>, a);
}
