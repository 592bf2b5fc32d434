// The bottom of the V-cycle in one launch (included by solve.cu).
//
// Levels with few rows (at most BOT_MAX_ROWS) do so little work per pass that
// the dependent memory round trips of each pass, not bandwidth, set their
// time.  One thread-block cluster runs all of them: the down-sweep
// (pre-smoothing, residual, restriction) of each bottom level, the coarsest
// level's sweeps, and the up-sweep (prolongation, post-smoothing), with a
// hardware cluster barrier between passes (no spinning).
//
// Each block of the cluster owns a power-of-two chunk of every bottom level's
// rows and keeps that level's vectors (input r, iterates za/zb, residual t) in
// its own shared memory; a row reads its neighbours' entries from the owning
// block's shared memory (distributed shared memory).  The matrices, the l1
// diagonals and the aggregation maps do not change during a solve: they are
// read from global memory (L1/L2-resident after the first pass).  The level-0
// input of the bottom comes from global memory, its result goes back there.
#pragma once

#include <cooperative_groups.h>

#include "amg_internal.cuh"

#define BOT_MAXL 8
#define BOT_THREADS 1024
#define BOT_MAX_ROWS 16384

struct BotLevel {
  int n;
  int shift;           // chunk = 1 << shift rows per block
  const int32_t* rp;
  const int32_t* ci;
  const void* v;       // level value type (double on the coarsest level)
  const void* dinv;
  const int32_t* agg;  // to the next bottom level
  const int32_t* mptr; // members of the next level's rows
  const int32_t* mem;
  int off_r, off_za, off_zb, off_t;  // byte offsets of the level's vectors in shared memory
};

struct BotArgs {
  int nb;                 // number of bottom levels; the last one is the coarsest
  BotLevel L[BOT_MAXL];
  int pre, post, csweeps;
  const void* r_in;       // input of bottom level 0 (global, its vector type)
  void* z_out;            // result of bottom level 0 (global)
  const int* skip;
};

__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

namespace bot {

namespace cg = cooperative_groups;

// element j of the distributed vector whose local part starts at `local`
template <typename T>
__device__ __forceinline__ T dget(const T* local, int j, int shift, unsigned me) {
  const unsigned owner = (unsigned)j >> shift;
  const int off = j & ((1 << shift) - 1);
  if (owner == me) return local[off];
  const T* remote = cg::this_cluster().map_shared_rank(local, owner);
  return remote[off];
}

struct Ctx {
  unsigned me;        // block rank in the cluster
  unsigned char* sm;  // this block's shared memory
};

template <typename T>
__device__ __forceinline__ T* vec(const Ctx& c, int off) {
  return reinterpret_cast<T*>(c.sm + off);
}

// rows of level L owned by this block: [row0, row1)
__device__ __forceinline__ void rows(const BotLevel& L, const Ctx& c, int& row0, int& row1) {
  row0 = (int)(c.me << L.shift);
  row1 = min(L.n, row0 + (1 << L.shift));
}

// s = sum_j a_ij x_j with x distributed
template <typename MT, typename VT>
__device__ __forceinline__ VT row_dot(const BotLevel& L, const Ctx& c, const VT* xl, int i) {
  const MT* v = (const MT*)L.v;
  VT s = 0;
  for (int p = __ldg(&L.rp[i]); p < __ldg(&L.rp[i + 1]); ++p)
    s += (VT)to_acc(__ldg(&v[p])) * dget(xl, __ldg(&L.ci[p]), L.shift, c.me);
  return s;
}

// `sweeps` l1-Jacobi sweeps; from zero when from_zero.  Returns the offset of
// the buffer that holds the result.
template <typename MT, typename VT>
__device__ int smooth(const BotLevel& L, const Ctx& c, int cur, int sweeps, bool from_zero) {
  int row0, row1;
  rows(L, c, row0, row1);
  const VT* r = vec<VT>(c, L.off_r);
  const VT* D = (const VT*)L.dinv;
  for (int s = 0; s < sweeps; ++s) {
    const int nxt = (cur == L.off_za) ? L.off_zb : L.off_za;
    VT* zo = vec<VT>(c, nxt);
    if (s == 0 && from_zero) {
      for (int i = row0 + (int)threadIdx.x; i < row1; i += blockDim.x) zo[i - row0] = __ldg(&D[i]) * r[i - row0];
    } else {
      const VT* zi = vec<VT>(c, cur);
      for (int i = row0 + (int)threadIdx.x; i < row1; i += blockDim.x)
        zo[i - row0] = zi[i - row0] + __ldg(&D[i]) * (r[i - row0] - row_dot<MT, VT>(L, c, zi, i));
    }
    cluster_barrier();
    cur = nxt;
  }
  if (sweeps <= 0 && from_zero) {
    VT* z = vec<VT>(c, cur);
    for (int i = row0 + (int)threadIdx.x; i < row1; i += blockDim.x) z[i - row0] = 0;
    cluster_barrier();
  }
  return cur;
}

}  // namespace bot

// MT/VT: value and vector types of the bottom levels above the coarsest one;
// the coarsest level runs in FP64.
template <typename MT, typename VT>
__global__ void __launch_bounds__(BOT_THREADS) k_bottom(const __grid_constant__ BotArgs a) {
  using namespace bot;
  pdl_trigger();
  pdl_wait();
  if (*a.skip) return;  // uniform over the cluster: every block reads the same flag
  extern __shared__ __align__(16) unsigned char bot_smem[];
  Ctx c{cg::this_cluster().block_rank(), bot_smem};
  const int nb = a.nb;
  // input of bottom level 0
  {
    const BotLevel& L = a.L[0];
    int row0, row1;
    rows(L, c, row0, row1);
    if (nb == 1) {
      const double* rin = (const double*)a.r_in;
      double* r = vec<double>(c, L.off_r);
      for (int i = row0 + (int)threadIdx.x; i < row1; i += blockDim.x) r[i - row0] = rin[i];
    } else {
      const VT* rin = (const VT*)a.r_in;
      VT* r = vec<VT>(c, L.off_r);
      for (int i = row0 + (int)threadIdx.x; i < row1; i += blockDim.x) r[i - row0] = rin[i];
    }
  }
  cluster_barrier();
  int res[BOT_MAXL];
  // down-sweep
  for (int k = 0; k < nb - 1; ++k) {
    const BotLevel& L = a.L[k];
    const BotLevel& C = a.L[k + 1];
    const int zoff = smooth<MT, VT>(L, c, L.off_za, a.pre, true);
    int row0, row1;
    rows(L, c, row0, row1);
    {
      const VT* r = vec<VT>(c, L.off_r);
      const VT* z = vec<VT>(c, zoff);
      VT* t = vec<VT>(c, L.off_t);
      for (int i = row0 + (int)threadIdx.x; i < row1; i += blockDim.x)
        t[i - row0] = r[i - row0] - row_dot<MT, VT>(L, c, z, i);
    }
    cluster_barrier();
    int c0, c1;
    rows(C, c, c0, c1);
    const VT* t = vec<VT>(c, L.off_t);
    for (int J = c0 + (int)threadIdx.x; J < c1; J += blockDim.x) {
      VT s = 0;
      for (int m = __ldg(&L.mptr[J]); m < __ldg(&L.mptr[J + 1]); ++m) s += dget(t, __ldg(&L.mem[m]), L.shift, c.me);
      if (k + 1 == nb - 1) vec<double>(c, C.off_r)[J - c0] = (double)s;
      else vec<VT>(c, C.off_r)[J - c0] = s;
    }
    cluster_barrier();
    res[k] = zoff;
  }
  // coarsest level (FP64)
  const BotLevel& Lc = a.L[nb - 1];
  const int zc_off = smooth<double, double>(Lc, c, Lc.off_za, a.csweeps, true);
  // up-sweep
  int up = zc_off;  // result of the level below
  for (int k = nb - 2; k >= 0; --k) {
    const BotLevel& L = a.L[k];
    const BotLevel& C = a.L[k + 1];
    int row0, row1;
    rows(L, c, row0, row1);
    VT* z = vec<VT>(c, res[k]);
    for (int i = row0 + (int)threadIdx.x; i < row1; i += blockDim.x) {
      const int J = __ldg(&L.agg[i]);
      if (k + 1 == nb - 1) z[i - row0] += (VT)dget(vec<double>(c, up), J, C.shift, c.me);
      else z[i - row0] += dget(vec<VT>(c, up), J, C.shift, c.me);
    }
    cluster_barrier();
    up = smooth<MT, VT>(L, c, res[k], a.post, false);
  }
  // result of bottom level 0 to global memory
  {
    const BotLevel& L = a.L[0];
    int row0, row1;
    rows(L, c, row0, row1);
    if (nb == 1) {
      const double* z = vec<double>(c, up);
      double* out = (double*)a.z_out;
      for (int i = row0 + (int)threadIdx.x; i < row1; i += blockDim.x) out[i] = z[i - row0];
    } else {
      const VT* z = vec<VT>(c, up);
      VT* out = (VT*)a.z_out;
      for (int i = row0 + (int)threadIdx.x; i < row1; i += blockDim.x) out[i] = z[i - row0];
    }
  }
  cluster_barrier();  // no block leaves while others may still read its shared memory
}

// cluster size of the bottom kernel: 16 blocks when the part allows it, else 8
template <typename MT, typename VT>
static int bottom_cluster_size(int smem) {
  static int cs = 0;
  if (cs) return cs;
  auto kern = k_bottom<MT, VT>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
  for (int want : {16, 8}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(want);
    cfg.blockDim = dim3(BOT_THREADS);
    cfg.dynamicSmemBytes = smem;
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
static cudaError_t launch_bottom(cudaStream_t s, const BotArgs& a, int cs, int smem) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(BOT_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = amg_pdl_enabled() ? 2 : 1;
  return cudaLaunchKernelEx(&cfg, k_bottom<MT, VT>, a);
}
