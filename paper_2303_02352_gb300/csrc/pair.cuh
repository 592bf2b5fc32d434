// Two consecutive row passes of one level in one persistent launch, sharing
// the matrix read through L2 (included by solve.cu after rows.cuh).
//
// On the large levels the V-cycle streams the whole matrix from HBM once per
// pass (an l1-Jacobi sweep or the residual), while the level's matrix is far
// larger than L2.  Passes come in runs (3 pre-smoothing sweeps and the
// residual, 4 post-smoothing sweeps), and pass B of a pair needs, for the rows
// of tile t, only the results of pass A on the tiles within the matrix
// bandwidth of t: tiles t-H .. t+H, H = ceil(bandwidth / R).  The paired
// kernel therefore runs pass A on tile t and pass B on tile t - lag in the same
// sweep over the matrix.  With lag = H + 1 + 2G (G resident blocks) tile t's
// values and column indices were read from HBM by pass A a few MB of traffic
// earlier and pass B finds them in L2: one HBM read of the matrix for two
// passes.  Every row is computed exactly as by the single-pass kernel.
//
// Measured on GB300 (7-point Poisson 160^3, level 0): the pair reads 372 MB
// from DRAM instead of 588 MB for two single passes (FP32), but it takes 197
// to 320 us against 2 x 50 us (FP32) and 2 x 81 us (FP64): per item it pays the
// hand-out from the shared counter, the dependency check, the release of its
// completion and second-pass gathers served by L2, none of which the single-
// pass kernel (static tiles, two stages of look-ahead) has.  The library
// therefore does not pair passes by default (use_pair = 0; AMG_PAIR=1 pairs
// where the level has room for the lag, AMG_PAIR=2 everywhere); the kernel is
// kept, tested for bitwise equality with the single passes.
//
// Order: work item q (q = 0 .. 2*ntiles-1) is the first pass of tiles
// 0 .. lag-1, then alternately the second pass of tile j and the first pass of
// tile j + lag, then the remaining second passes.  Items are handed out in
// this order: a block's producer takes the next item from a global counter
// whenever one of its stages is free.  The second pass of tile t waits
// until the first pass of every tile <= t + H is complete; those items come
// earlier in the order, so they were handed out earlier, to blocks that are
// running, and the smallest unfinished item can always proceed -- whether or
// not every block of the grid is resident (with programmatic dependent launch
// the previous kernel may still hold multiprocessors while this one starts).
//
// Completion tracking: tiles are grouped in chunks of PAIR_CHUNK; each
// consumer warp adds 1 to its tile's chunk counter with release semantics
// after writing its rows of the first pass.  Before it issues the copies of a
// second-pass item, the producer warp checks the chunk counters of tiles
// t-H .. t+H (one warp-wide load of relaxed reads, then an acquire fence);
// the consumers, a full pipeline stage behind, never wait on dependencies,
// and no serial chain links the tiles.  Counters are cumulative over launches
// (chunk c is complete at (epoch + 1) * consumer warps * tiles of c); the last
// block of a launch resets the hand-out counter and advances the epoch.  Every
// wait is bounded in time: on expiry ST_TIMEOUT is set, the warp leaves its
// loop, and the host resets the state.
#pragma once

#include "rows.cuh"

struct PairCtl {
  unsigned epoch;        // completed launches on this level
  unsigned done_blocks;  // blocks that finished the current launch
  int pad;
  int next;              // next item to hand out (current launch)
};

template <typename MT, typename VT, typename OT>
struct PairArgs {
  int n;
  const int32_t* rp;
  const int32_t* ci;
  const MT* v;
  const VT* dinv;
  const VT* r;
  const VT* z0;      // input of the first pass (a sweep)
  VT* z1;            // result of the first pass, input of the second
  OT* out;           // result of the second pass (sweep result or residual); may alias z0
  const int* skip;
  int* flags;
  PairCtl* ctl;
  unsigned* cnt;     // per chunk of PAIR_CHUNK tiles, cumulative over launches
  int halo;          // H
  int lag;           // >= H + PAIR_CHUNK + 1
};

#define PAIR_CHUNK 64
#define PAIR_BATCH 4   // items handed out per counter access
#ifndef PAIR_STAGES
#define PAIR_STAGES 2  // pipeline depth of the paired kernel
#endif

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned ld_acquire_u(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// are the first passes of tiles t-H .. t+H (inside [0, ntiles)) complete?
// Whole-warp call; lane l checks chunk lo/PAIR_CHUNK + l (+32, ...) with
// acquire loads (one per lane for halos up to 32 chunks).
__device__ __forceinline__ bool pair_deps_done(const unsigned* cnt, int t, int H, int ntiles, unsigned per_tile,
                                               int lane) {
  const int c0 = max(0, t - H) / PAIR_CHUNK, c1 = min(ntiles - 1, t + H) / PAIR_CHUNK;
  bool ok = true;
  for (int c = c0 + lane; c <= c1; c += 32) {
    const unsigned tiles = (unsigned)min(PAIR_CHUNK, ntiles - c * PAIR_CHUNK);
    ok = ok && ld_acquire_u(&cnt[c]) >= per_tile * tiles;
  }
  return __all_sync(0xffffffffu, ok);
}

// item q -> (phase, tile); phase 0 = first pass, 1 = second pass
__device__ __forceinline__ void pair_item(int q, int ntiles, int lag, int& phase, int& tile) {
  const int first = min(lag, ntiles);
  if (q < first) {
    phase = 0;
    tile = q;
    return;
  }
  const int E = ntiles - first;  // interleaved pairs
  const int m = q - first;
  if (m < 2 * E) {
    phase = (m & 1) ? 0 : 1;
    tile = (m & 1) ? first + (m >> 1) : (m >> 1);
    return;
  }
  phase = 1;
  tile = E + (m - 2 * E);
}

// MODE2: PM_SWEEP (out = z1 + D (r - A z1)) or PM_RESID (out = r - A z1)
template <int TPR, int S, int MODE2, typename MT, typename VT, typename OT>
__global__ void __launch_bounds__(PIPE_CONSUMERS + 32) k_rows_pair(const PairArgs<MT, VT, OT> a) {
  constexpr int R = PIPE_CONSUMERS / TPR;
  pdl_trigger();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  auto* P = reinterpret_cast<PipeSmem<MT, S>*>(smem_raw);
  constexpr int VE = PipeTile<MT, 1>::VE;
  constexpr int NCW = PIPE_CONSUMERS / 32;
  const int n = a.n;
  const int ntiles = (n + R - 1) / R;
  const int nitems = 2 * ntiles;
  const int G = gridDim.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&P->full[s], 1);
      mbar_init(&P->empty[s], NCW);
    }
    mbar_fence_init();
  }
  __syncthreads();

  __shared__ int item_of[S];  // the item in each stage (-1: no more items)
  auto issue = [&](int q, int stage) {
    int ph, tile;
    pair_item(q, ntiles, a.lag, ph, tile);
    item_of[stage] = q;
    const int row0 = tile * R, row1 = min(row0 + R, n);
    const int p0 = __ldg(&a.rp[row0]), p1 = __ldg(&a.rp[row1]);
    const int av = p0 & ~(VE - 1), ac = p0 & ~3;
    const uint32_t bv = (uint32_t)(((p1 - av) * (int)sizeof(MT) + 15) & ~15);
    const uint32_t bc = (uint32_t)(((p1 - ac) * 4 + 15) & ~15);
    mbar_expect_tx(&P->full[stage], bv + bc);
    tma_load_1d(P->st[stage].v, a.v + av, bv, &P->full[stage]);
    tma_load_1d(P->st[stage].c, a.ci + ac, bc, &P->full[stage]);
  };
  // every item is handed out after the wait: the counter belongs to the
  // previous launch on this level until that launch has completed
  pdl_wait();
  if (*a.skip) return;
  // the control word is read at gpu scope: with programmatic dependent launch
  // this block may have started while the previous launch on the level still
  // ran on this multiprocessor, and a plain load could return its L1 copy
  const unsigned epoch = (unsigned)ld_acquire((const int*)&a.ctl->epoch);
  const unsigned target = (epoch + 1u) * (unsigned)NCW;

  if (warp == NCW) {
    // ---------------- producer warp ----------------
    int k = 0;
    bool aborted = false;
    int qnext = 0, qend = 0;  // this block's current batch of items
    for (;; ++k) {
      const int stage = k % S;
      if (qnext == qend) {  // next batch (taken before the wait for a free stage)
        int q0 = 0;
        if (lane == 0) q0 = atomicAdd(&a.ctl->next, PAIR_BATCH);
        qnext = __shfl_sync(0xffffffffu, q0, 0);
        qend = qnext + PAIR_BATCH;
      }
      if (k >= S && !mbar_wait_warp(&P->empty[stage], (uint32_t)(((k / S) - 1) & 1))) {
        aborted = true;
        break;
      }
      const int q = qnext++;
      if (q >= nitems) {  // no more items: release the consumers
        if (lane == 0) {
          item_of[stage] = -1;
          mbar_arrive(&P->full[stage]);
        }
        break;
      }
      int phase, tile;
      pair_item(q, ntiles, a.lag, phase, tile);
      if (phase == 1) {  // the first pass on every tile this tile's rows reach
        if (!pair_deps_done(a.cnt, tile, a.halo, ntiles, target, lane)) {
          const uint64_t t0 = global_ns();
          for (;;) {
            __nanosleep(128);
            if (pair_deps_done(a.cnt, tile, a.halo, ntiles, target, lane)) break;
            if (global_ns() - t0 > PIPE_WAIT_NS) {
              aborted = true;
              break;
            }
          }
          if (aborted) break;
        }
      }
      if (lane == 0) issue(q, stage);
      __syncwarp();
    }
    if (aborted && lane == 0) {  // drain the copies in flight, bounded
      atomicOr(a.flags, ST_TIMEOUT);
      for (int j = 1; j <= S && k - j >= 0; ++j) {
        const int kk = k - j;
        mbar_wait(&P->full[kk % S], (uint32_t)((kk / S) & 1));
      }
    }
    __syncwarp();
  } else {
    // ---------------- consumer warps ----------------
    for (int k = 0;; ++k) {
      const int stage = k % S;
      if (!mbar_wait_warp(&P->full[stage], (uint32_t)((k / S) & 1))) {
        if (lane == 0) atomicOr(a.flags, ST_TIMEOUT);
        break;
      }
      const int q = item_of[stage];
      if (q < 0) break;
      int phase, tile;
      pair_item(q, ntiles, a.lag, phase, tile);
      const int row0 = tile * R, row1 = min(row0 + R, n);
      const int sub = (int)threadIdx.x % TPR;
      const int row = row0 + (int)threadIdx.x / TPR;
      const bool live = row < row1;
      const bool lead = live && sub == 0;
      const int p0 = __ldg(&a.rp[row0]);
      int q0 = 0, q1 = 0;
      VT own = 0, rr = 0, dd = 0;
      if (live) {
        q0 = __ldg(&a.rp[row]) + sub;
        q1 = __ldg(&a.rp[row + 1]);
      }
      if (lead) {
        rr = __ldg(&a.r[row]);
        if (phase == 0) {
          own = __ldg(&a.z0[row]);
          dd = __ldg(&a.dinv[row]);
        } else if constexpr (MODE2 == PM_SWEEP) {
          own = __ldcg(&a.z1[row]);
          dd = __ldg(&a.dinv[row]);
        }
      }
      const int av = p0 & ~(VE - 1), ac = p0 & ~3;
      const PipeTile<MT, 1>& T = P->st[stage];
      VT s = rr;  // r_i - sum_j a_ij x_j accumulated from r_i, as in the single-pass kernel
      if (phase == 0) {
#pragma unroll 8
        for (int qq = q0; qq < q1; qq += TPR) s -= (VT)to_acc(T.v[qq - av]) * __ldg(&a.z0[amg_chk(T.c[qq - ac], n)]);
      } else {
#pragma unroll 8
        for (int qq = q0; qq < q1; qq += TPR) s -= (VT)to_acc(T.v[qq - av]) * __ldcg(&a.z1[amg_chk(T.c[qq - ac], n)]);
      }
      if constexpr (TPR > 1) s = group_sum<TPR>(s);
      __syncwarp();
      if (lane == 0) mbar_arrive(&P->empty[stage]);
      if (phase == 0) {
        if (lead) a.z1[row] = own + dd * s;
        __syncwarp();
        if (lane == 0) red_release_add(&a.cnt[tile / PAIR_CHUNK], 1u);
      } else if (lead) {
        if constexpr (MODE2 == PM_SWEEP) a.out[row] = (OT)(own + dd * s);
        else a.out[row] = (OT)s;
      }
    }
  }
  // the last block of the launch resets the hand-out counter and advances the epoch
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&a.ctl->done_blocks, 1u) == (unsigned)G - 1u) {
      atomicExch(&a.ctl->done_blocks, 0u);
      atomicExch(&a.ctl->next, 0);
      atomicAdd(&a.ctl->epoch, 1u);
      __threadfence();
    }
  }
}

template <int TPR, int S, int MODE2, typename MT, typename VT, typename OT>
static int pair_grid(int n) {
  static int bps = -1;
  constexpr int smem = (int)sizeof(PipeSmem<MT, S>);
  auto kern = k_rows_pair<TPR, S, MODE2, MT, VT, OT>;
  if (bps < 0) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, PIPE_CONSUMERS + 32, smem);
    bps = b < 1 ? 1 : b;
  }
  constexpr int R = PIPE_CONSUMERS / TPR;
  const int items = 2 * ((n + R - 1) / R);
  const int g = amg_num_sms() * bps;
  return items < g ? items : g;
}

template <int TPR, int S, int MODE2, typename MT, typename VT, typename OT>
static void launch_pair_tpr(cudaStream_t s, const PairArgs<MT, VT, OT>& a) {
  const int grid = pair_grid<TPR, S, MODE2, MT, VT, OT>(a.n);
  constexpr int smem = (int)sizeof(PipeSmem<MT, S>);
  amg_launch(k_rows_pair<TPR, S, MODE2, MT, VT, OT>, dim3(grid), dim3(PIPE_CONSUMERS + 32), (size_t)smem, s, a);
}
