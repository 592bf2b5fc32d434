// The bottom of the V-cycle in one launch (included by solve.cu).
//
// Levels with few rows do so little work per pass that a separate launch per
// pass costs more than the pass itself (about 2.4 us per dependent launch).
// One thread-block cluster runs all of them: the down-sweep (pre-smoothing,
// residual, restriction) of each bottom level, the coarsest level's sweeps,
// and the up-sweep (prolongation, post-smoothing), with a hardware cluster
// barrier between passes.
//
// Block c of the cluster owns the rows [c*chunk, (c+1)*chunk) of every bottom
// level, chunk = ceil(n / cluster size).  At launch it copies its slice of
// each level's CSR arrays, l1 diagonal, aggregation map and aggregate member
// lists into its own shared memory; these copies are made before waiting on
// the previous kernel (they do not change during a solve).  Each level's work
// vectors (input r, iterates za / zb, residual t) live in shared memory too,
// distributed the same way: a row reads its neighbours' entries from the
// owning block's shared memory (distributed shared memory).
//
// Measured on this part: a load from distributed shared memory costs a few
// hundred cycles when a warp's lanes all reach one block, but the lanes of one
// load that reach several blocks are served one block after another.  On the
// regular levels of a 7-point hierarchy neighbours sit in the same or the
// adjacent block and the kernel beats separate launches; on the irregular
// coarse levels of 27-point problems it does not.  The library times both forms
// once per hierarchy and keeps the faster (amg_prepare_solve).
//
// The row sums, the restriction sums and the prolongation use the operation
// order of the separate kernels (entries in CSR order, members ascending).
#pragma once

#include <cooperative_groups.h>

#include <vector>

#include "amg_internal.cuh"

#define BOT_MAXL 8
#define BOT_THREADS 1024
#define BOT_MAX_CS 16
#define BOT_MAX_ROWS 16384             // largest level taken into the bottom
#define BOT_SMEM_MAX (200 * 1024)      // shared memory budget per block

struct BotLevel {
  int n;                     // rows
  int chunk;                 // rows per block
  unsigned long long magic;  // ceil(2^32 / chunk): the owner of row j is (j * magic) >> 32
  const int32_t* rp;
  const int32_t* ci;
  const void* v;             // level value type (double on the coarsest level)
  const void* dinv;
  const int32_t* agg;        // to the next bottom level
  const int32_t* mptr;       // members of the next level's rows
  const int32_t* mem;
  int e0[BOT_MAX_CS + 1];    // first entry of each block's rows: row_ptr[min(c*chunk, n)]
  int m0[BOT_MAX_CS + 1];    // first member of each block's next-level rows
  // byte offsets of the level's shared-memory sections (the same in every block)
  int o_rp, o_ci, o_v, o_dinv, o_agg, o_mptr, o_mem, o_r, o_za, o_zb, o_t;
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

struct Ctx {
  int me;             // block rank in the cluster
  unsigned char* sm;  // this block's shared memory
};

template <typename T>
__device__ __forceinline__ T* sec(const Ctx& c, int off) {
  return reinterpret_cast<T*>(c.sm + off);
}

// rows of level L owned by this block: [r0, r0 + cnt)
__device__ __forceinline__ void rows(const BotLevel& L, const Ctx& c, int& r0, int& cnt) {
  r0 = min(c.me * L.chunk, L.n);
  cnt = min(L.n - r0, L.chunk);
}

// entry j of the distributed vector whose sections start at byte offset off
template <typename T>
__device__ __forceinline__ T dget(const BotLevel& L, const Ctx& c, int off, int j) {
  j = amg_chk(j, L.n);
  const int o = (int)(((unsigned long long)(unsigned)j * L.magic) >> 32);
  const int k = j - o * L.chunk;
  const T* local = sec<T>(c, off);
  if (o == c.me) return local[k];
  return cg::this_cluster().map_shared_rank(local, (unsigned)o)[k];
}

// address of entry j of a distributed vector (own block: the local section;
// another block: its section through the cluster window).  A select, not a
// branch, so that a row's loads can all be issued before the first returns.
template <typename T>
__device__ __forceinline__ const T* daddr(const BotLevel& L, const Ctx& c, int off, int j) {
  j = amg_chk(j, L.n);
  const int o = (int)(((unsigned long long)(unsigned)j * L.magic) >> 32);
  const T* local = sec<T>(c, off);
  const T* remote = cg::this_cluster().map_shared_rank(local, (unsigned)o);
  return (o == c.me ? local : remote) + (j - o * L.chunk);
}

// gathers of a row issued before its multiply-adds (within the 64 registers a
// thread of a 1024-thread block has)
template <typename T>
__host__ __device__ constexpr int bot_batch() {
  return sizeof(T) == 8 ? 4 : 8;
}

// copy this block's slice of level L (and of its maps to the next level C)
template <typename MT, typename VT>
__device__ void load_level(const BotLevel& L, const BotLevel* C, const Ctx& c) {
  int r0, cnt;
  rows(L, c, r0, cnt);
  const int e0 = L.e0[c.me], ne = L.e0[c.me + 1] - e0;
  int32_t* rp = sec<int32_t>(c, L.o_rp);
  for (int i = threadIdx.x; i <= cnt; i += blockDim.x) rp[i] = __ldg(&L.rp[r0 + i]) - e0;
  int32_t* ci = sec<int32_t>(c, L.o_ci);
  MT* v = sec<MT>(c, L.o_v);
  const MT* gv = static_cast<const MT*>(L.v);
  for (int p = threadIdx.x; p < ne; p += blockDim.x) {
    ci[p] = __ldg(&L.ci[e0 + p]);
    v[p] = __ldg(&gv[e0 + p]);
  }
  VT* d = sec<VT>(c, L.o_dinv);
  const VT* gd = static_cast<const VT*>(L.dinv);
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) d[i] = __ldg(&gd[r0 + i]);
  if (C) {
    int32_t* agg = sec<int32_t>(c, L.o_agg);
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) agg[i] = __ldg(&L.agg[r0 + i]);
    int R0, ccnt;
    rows(*C, c, R0, ccnt);
    const int m0 = L.m0[c.me], nm = L.m0[c.me + 1] - m0;
    int32_t* mp = sec<int32_t>(c, L.o_mptr);
    for (int i = threadIdx.x; i <= ccnt; i += blockDim.x) mp[i] = __ldg(&L.mptr[R0 + i]) - m0;
    int32_t* mm = sec<int32_t>(c, L.o_mem);
    for (int m = threadIdx.x; m < nm; m += blockDim.x) mm[m] = __ldg(&L.mem[m0 + m]);
  }
}

// r_i - sum_j a_ij x_j over row i (local index), accumulated from r_i like
// the row kernels; x distributed at byte offset xo
template <typename MT, typename VT>
__device__ __forceinline__ VT row_resid(const BotLevel& L, const Ctx& c, int xo, int i, VT ri) {
  const int32_t* rp = sec<int32_t>(c, L.o_rp);
  const int32_t* ci = sec<int32_t>(c, L.o_ci);
  const MT* v = sec<MT>(c, L.o_v);
  VT s = ri;
  const int p1 = rp[i + 1];
  // the row's gathers (shared or distributed shared memory) are independent:
  // issue a batch of them, then the multiply-adds in entry order
  constexpr int B = bot_batch<VT>();
  for (int p = rp[i]; p < p1; p += B) {
    VT xv[B];
#pragma unroll
    for (int u = 0; u < B; ++u)
      if (p + u < p1) xv[u] = *daddr<VT>(L, c, xo, ci[p + u]);
#pragma unroll
    for (int u = 0; u < B; ++u)
      if (p + u < p1) s -= (VT)v[p + u] * xv[u];
  }
  return s;
}

// `sweeps` l1-Jacobi sweeps starting from the iterate at offset cur (from zero
// when from_zero).  Returns the offset of the section that holds the result.
template <typename MT, typename VT>
__device__ int smooth(const BotLevel& L, const Ctx& c, int cur, int sweeps, bool from_zero) {
  int r0, cnt;
  rows(L, c, r0, cnt);
  const VT* r = sec<VT>(c, L.o_r);
  const VT* D = sec<VT>(c, L.o_dinv);
  for (int s = 0; s < sweeps; ++s) {
    const int nxt = (cur == L.o_za) ? L.o_zb : L.o_za;
    VT* zo = sec<VT>(c, nxt);
    if (s == 0 && from_zero) {
      for (int i = threadIdx.x; i < cnt; i += blockDim.x) zo[i] = D[i] * r[i];
    } else {
      const VT* zi = sec<VT>(c, cur);
      for (int i = threadIdx.x; i < cnt; i += blockDim.x)
        zo[i] = zi[i] + D[i] * row_resid<MT, VT>(L, c, cur, i, r[i]);
    }
    cluster_barrier();
    cur = nxt;
  }
  if (sweeps <= 0 && from_zero) {
    VT* z = sec<VT>(c, cur);
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) z[i] = 0;
    cluster_barrier();
  }
  return cur;
}

// r_C[J] = sum over the members i of J (ascending) of t_i for this block's
// rows J of the next level (its input: own rows only)
template <typename VT, typename CT>
__device__ __forceinline__ void restrict_to(const BotLevel& L, const BotLevel& C, const Ctx& c) {
  int R0, ccnt;
  rows(C, c, R0, ccnt);
  const int32_t* mp = sec<int32_t>(c, L.o_mptr);
  const int32_t* mm = sec<int32_t>(c, L.o_mem);
  CT* rc = sec<CT>(c, C.o_r);
  for (int J = threadIdx.x; J < ccnt; J += blockDim.x) {
    VT s = 0;
    const int m1 = mp[J + 1];
    constexpr int B = bot_batch<VT>();
    for (int m = mp[J]; m < m1; m += B) {  // members' loads first, then the sum in member order
      VT tv[B];
#pragma unroll
      for (int u = 0; u < B; ++u)
        if (m + u < m1) tv[u] = *daddr<VT>(L, c, L.o_t, mm[m + u]);
#pragma unroll
      for (int u = 0; u < B; ++u)
        if (m + u < m1) s += tv[u];
    }
    rc[J] = (CT)s;
  }
}

// z_i += z_C[agg(i)] on this block's rows of L (iterate at zoff, coarse at coff)
template <typename VT, typename CT>
__device__ __forceinline__ void prolong_from(const BotLevel& L, const BotLevel& C, const Ctx& c, int zoff, int coff) {
  int r0, cnt;
  rows(L, c, r0, cnt);
  VT* z = sec<VT>(c, zoff);
  const int32_t* agg = sec<int32_t>(c, L.o_agg);
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) z[i] = z[i] + (VT)dget<CT>(C, c, coff, agg[i]);
}

}  // namespace bot

// VT: vector and value type of the bottom levels above the coarsest one; the
// coarsest level runs in FP64.
template <typename VT>
__global__ void __launch_bounds__(BOT_THREADS) k_bottom(const __grid_constant__ BotArgs a) {
  using namespace bot;
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char bot_smem[];
  Ctx c{(int)cg::this_cluster().block_rank(), bot_smem};
  const int nb = a.nb;
  // the constant slices, before waiting for the previous kernel
  for (int k = 0; k < nb; ++k) {
    if (k == nb - 1) load_level<double, double>(a.L[k], nullptr, c);
    else load_level<VT, VT>(a.L[k], &a.L[k + 1], c);
  }
  pdl_wait();
  if (*a.skip) return;  // uniform over the cluster: every block reads the same flag
  // input of bottom level 0 (own rows)
  {
    const BotLevel& L = a.L[0];
    int r0, cnt;
    rows(L, c, r0, cnt);
    if (nb == 1) {
      const double* rin = (const double*)a.r_in;
      double* r = sec<double>(c, L.o_r);
      for (int i = threadIdx.x; i < cnt; i += blockDim.x) r[i] = rin[r0 + i];
    } else {
      const VT* rin = (const VT*)a.r_in;
      VT* r = sec<VT>(c, L.o_r);
      for (int i = threadIdx.x; i < cnt; i += blockDim.x) r[i] = rin[r0 + i];
    }
  }
  cluster_barrier();  // every block started; slices and input visible
  int res[BOT_MAXL];
  // down-sweep
  for (int k = 0; k < nb - 1; ++k) {
    const BotLevel& L = a.L[k];
    const BotLevel& C = a.L[k + 1];
    const int zoff = smooth<VT, VT>(L, c, L.o_za, a.pre, true);
    int r0, cnt;
    rows(L, c, r0, cnt);
    {
      const VT* r = sec<VT>(c, L.o_r);
      VT* t = sec<VT>(c, L.o_t);
      for (int i = threadIdx.x; i < cnt; i += blockDim.x) t[i] = row_resid<VT, VT>(L, c, zoff, i, r[i]);
    }
    cluster_barrier();
    if (k + 1 == nb - 1) restrict_to<VT, double>(L, C, c);
    else restrict_to<VT, VT>(L, C, c);
    __syncthreads();
    res[k] = zoff;
  }
  // coarsest level (FP64)
  const BotLevel& Lc = a.L[nb - 1];
  int up = smooth<double, double>(Lc, c, Lc.o_za, a.csweeps, true);  // result of the level below
  // up-sweep
  for (int k = nb - 2; k >= 0; --k) {
    const BotLevel& L = a.L[k];
    const BotLevel& C = a.L[k + 1];
    if (k + 1 == nb - 1) prolong_from<VT, double>(L, C, c, res[k], up);
    else prolong_from<VT, VT>(L, C, c, res[k], up);
    cluster_barrier();
    up = smooth<VT, VT>(L, c, res[k], a.post, false);
  }
  // result of bottom level 0 to global memory
  {
    const BotLevel& L = a.L[0];
    int r0, cnt;
    rows(L, c, r0, cnt);
    if (nb == 1) {
      const double* z = sec<double>(c, up);
      double* out = (double*)a.z_out;
      for (int i = threadIdx.x; i < cnt; i += blockDim.x) out[r0 + i] = z[i];
    } else {
      const VT* z = sec<VT>(c, up);
      VT* out = (VT*)a.z_out;
      for (int i = threadIdx.x; i < cnt; i += blockDim.x) out[r0 + i] = z[i];
    }
  }
}

// can a cluster of cs blocks with smem bytes each be resident?
template <typename VT>
static bool bottom_fits(int cs, int smem) {
  auto kern = k_bottom<VT>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, BOT_SMEM_MAX);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(BOT_THREADS);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int clusters = 0;
  const bool ok = cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) == cudaSuccess && clusters > 0;
  cudaGetLastError();
  return ok;
}

template <typename VT>
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
  return cudaLaunchKernelEx(&cfg, k_bottom<VT>, a);
}
