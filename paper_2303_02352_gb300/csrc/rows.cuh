// Persistent TMA-pipelined row kernels (included by solve.cu).
//
// A block owns tiles of R consecutive rows, round-robin over the grid.  The
// nonzeros of a tile are contiguous in CSR; a producer warp issues 1D bulk
// copies (cp.async.bulk, the TMA engine) that move the tile's values and column
// indices (or, on pattern-coded levels, its one-byte row ids), and where the
// stage has room its row pointers and row vectors, into a shared-memory stage
// and signal the stage's "full" mbarrier.
// S stages rotate: while the consumer warps compute tile k, the copies of the
// next tiles are in flight, so HBM sees a continuous stream.  Each consumer
// thread finishes one row (one multiply-add per nonzero, no shuffle reduction:
// the FP64 issue rate is a co-limit on this part) and gathers the vector
// through L1/L2.
//
// Every mbarrier wait is bounded in time (2 s); on expiry the kernel sets
// ST_TIMEOUT in the device flags, drains its copies with a bounded wait and
// ends its tile loop; the host maps the flag to AMG_ERR_TIMEOUT.
#pragma once

#include "amg_internal.cuh"

#define PIPE_WAIT_NS 2000000000ull  // 2 s: a copy of at most 24 KB never takes this long

// stage capacity (values + column indices): sized per value type so that a
// PIPE_CONSUMERS-row tile of a 7-point stencil fits with little slack (smaller
// stages mean more resident blocks per multiprocessor, which is what the row
// kernels need)
// SB scales the stage: SB = 4 (FP64 only) holds 256 rows of up to 32 entries,
// so long-row levels keep one thread per row (see launch_rows)
// PAT: the column area holds the tile's one-byte row ids (pattern-coded
// columns; the same value capacity).  STG: the stage also has a row-data area
// for the tile's row pointers and up to three row vectors of VB bytes per
// entry (iterate, right-hand side, D) of its RT rows, so that every stream of
// the row pass arrives by bulk copy ahead of the consumers.
template <typename MT, int SB = 1, bool PAT = false, int VB = 8, int RT = PIPE_CONSUMERS, bool STG = PAT>
struct PipeTile {
  static constexpr int VE = 16 / (int)sizeof(MT);
  static constexpr int CAP = amg_pipe_tile_bytes((int)sizeof(MT)) * SB / ((int)sizeof(MT) + 4);
  MT v[CAP + 2 * VE];
  int32_t c[PAT ? (PIPE_CONSUMERS + 16) / 4 : CAP + 8];
  int32_t rps[STG ? RT + 8 : 4];
  alignas(16) unsigned char ov[STG ? 3 * RT * VB : 16];
};

template <typename MT, int S, int SB = 1, bool PAT = false, int VB = 8, int RT = PIPE_CONSUMERS, bool STG = PAT>
struct PipeSmem {
  PipeTile<MT, SB, PAT, VB, RT, STG> st[S];
  unsigned long long full[S];   // producer -> consumers: the stage holds the tile
  unsigned long long empty[S];  // consumers -> producer: every consumer warp has read it
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
  uint32_t ok;
#if MBAR_SUSPEND_NS > 0
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity), "r"((uint32_t)MBAR_SUSPEND_NS)
      : "memory");
#else
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
#endif
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// bounded wait: true when the phase completed, false after limit_ns of
// polling (the clock is read every 64 polls, so the bound holds whatever the
// suspend time of a single try_wait)
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t parity,
                                          uint64_t limit_ns = PIPE_WAIT_NS) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63u) == 0u && global_ns() - t0 > limit_ns) return false;
  }
}

// PM_SWEEP_PROLONG: an l1-Jacobi sweep of a coarse level whose result is also
// added to the next finer level's iterate, z_f[i] += z_c[J] for every member i
// of aggregate J (the unit piecewise-constant prolongation of the V-cycle)
enum { PM_SWEEP = 0, PM_RESID = 1, PM_SPMV = 2, PM_DOTS = 3, PM_RINIT = 4, PM_RTRUE = 5, PM_RNORM = 6,
       PM_SWEEP_PROLONG = 7 };

// stage of a pattern-coded kernel: the small one (values and ids), except for
// the outer SpMV with dot products, which measured faster in four blocks of
// full stages per multiprocessor than in six of small ones (7-point Poisson
// 320^3: 615 vs 665 us).  The V-cycle kernels all take the small stage: taken
// alone the FP64 sweep is faster in full stages (553 vs 572 us) and the
// residual in small ones (446 vs 532 us), but a V-cycle that alternates the
// two footprints ran 6% slower than either uniform choice (5.83 vs 5.47-5.49
// ms): consecutive launches overlap (programmatic dependent launch) only where
// a finished block's slot fits a block of the next kernel.
template <typename MT, int MODE, int PAT>
__host__ __device__ constexpr bool pat_small() {
  return PAT > 0 && MODE != PM_DOTS;
}

// stages with the row-data area: the small pattern stages, and CSR sweeps and
// residuals in standard stages of at most CSR_STAGE_ROWS rows (there the area
// is small against the stage: 27-point levels, 64-row tiles)
template <typename MT, int MODE, int PAT, int SB, int R>
__host__ __device__ constexpr bool row_stage() {
  return pat_small<MT, MODE, PAT>() ||
         (PAT == 0 && SB == 1 && R <= CSR_STAGE_ROWS && (MODE == PM_SWEEP || MODE == PM_RESID));
}

template <typename MT, typename VT, typename OT>
struct RowArgs {
  int n;
  const int32_t* rp;
  const int32_t* ci;
  const MT* v;
  const VT* x;      // gathered vector (z, w or u)
  const VT* dinv;   // sweep
  const VT* r;      // sweep / residual: level right-hand side; dots: FCG r
  const VT* b;      // FCG right-hand side
  const VT* q;      // dots
  OT* out;          // sweep: z_out, resid: t, spmv: y, dots: v, rinit/rtrue: r
  const int* skip;  // V-cycle modes
  FcgState* st;     // FCG modes
  double* partial;
  unsigned* counter;
  int* flags;
  // PM_SWEEP_PROLONG: members of each row's aggregate and the finer iterate
  const int32_t* mptr;
  const int32_t* mem;
  void* zf;
  int zf64;  // the finer iterate is double (else float)
  int nf;    // rows of the finer level (bounds-checked builds)
  // pattern-coded columns (PAT forms): row i's columns are i + ptab[pid[i] * pk + j]
  const uint8_t* pid;
  const int32_t* ptab;
  int pk;
  int ptab_n;           // table entries
  const int32_t* plen;  // entries of each tuple (npat)
  int npat;
  const int32_t* pcb;   // PAT = 2: row_ptr at every 32nd row, and nnz
  int stage_rows;       // small-stage pattern forms: row pointers and row vectors by bulk copy (16-byte aligned)
};


// z_f[i] += z for the members i of aggregate `row`, in the finer level's
// vector type.  The TPR lanes of the row share the members (lane `sub` takes
// members sub, sub + TPR, ...); each lane loads up to 8 member ids, then their
// z_f entries, then stores, so one row costs three dependent round trips.
template <typename FT, typename OT>
__device__ __forceinline__ void prolong_chunk(FT* zf, const int32_t* mem, int base, int m1, int step, OT z, int nf) {
  int idx[8];
  FT v[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int m = base + u * step;
    idx[u] = m < m1 ? amg_chk(__ldg(&mem[m]), nf) : -1;
  }
#pragma unroll
  for (int u = 0; u < 8; ++u)
    if (idx[u] >= 0) v[u] = zf[idx[u]];
#pragma unroll
  for (int u = 0; u < 8; ++u)
    if (idx[u] >= 0) zf[idx[u]] = v[u] + (FT)z;
}

template <int TPR, typename MT, typename VT, typename OT>
__device__ __forceinline__ void prolong_members(const RowArgs<MT, VT, OT>& a, int row, int sub, OT z) {
  const int m1 = __ldg(&a.mptr[row + 1]);
  for (int base = __ldg(&a.mptr[row]) + sub; base < m1; base += 8 * TPR) {
    if (a.zf64) prolong_chunk(static_cast<double*>(a.zf), a.mem, base, m1, TPR, z, a.nf);
    else prolong_chunk(static_cast<float*>(a.zf), a.mem, base, m1, TPR, z, a.nf);
  }
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// warp-uniform bounded wait (lane 0 polls, the result is broadcast)
__device__ __forceinline__ bool mbar_wait_warp(unsigned long long* bar, uint32_t parity) {
  bool ok = false;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity);
  return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}


// Warp-specialised persistent row kernel: PIPE_CONSUMERS / 32 consumer warps
// (8 by default) and one producer warp.  A tile holds R = PIPE_CONSUMERS / TPR
// rows; TPR threads share a row (entries strided by TPR, summed with shuffles),
// so that long rows still keep every consumer busy per tile; TPR = 1 for short
// rows (one thread per row).  Per stage a "full" barrier (the producer's
// expect_tx plus the bytes of its bulk copies) and an "empty" barrier (one
// arrival per consumer warp once it has read the stage).  No block-wide
// barrier inside the tile loop: warps drift up to S tiles apart.
//
// NG > 1 splits the consumer warps into NG groups that take the block's tiles
// in turn (group g: tiles g, g + NG, ...): tiles of R = PIPE_CONSUMERS / NG /
// TPR rows, S stages in flight, each stage read by one group.  Long rows then
// keep one thread per row with more, smaller stages in flight.
//
// PAT > 0: the level's columns are pattern-coded (pattern.cu).  The second
// copy of a tile moves its rows' one-byte pattern ids instead of the entries'
// column indices, and entry j of row i gathers x[i + ptab[id * pk + j]]; the
// table and the tuple lengths (at most 4 KB) are copied into shared memory
// behind the stages when the block starts, so an offset costs what a staged
// column index cost (read through L1 instead, the offset load added a
// dependent round trip before every gather: 7-point FP64 sweep 0.610 -> 0.647
// ms at 320^3, measured).  PAT = 2 (one thread per row) also leaves row_ptr
// unread: a warp's 32 rows are consecutive, start at pcb[first row / 32], and
// each row starts where the previous one ends (a warp scan of the tuple
// lengths).  Same entries, same order, same arithmetic in every form.
template <int TPR, int S, int MODE, typename MT, typename VT, typename OT, int SB = 1, int NG = 1, int PAT = 0>
__global__ void __launch_bounds__(PIPE_CONSUMERS + 32) k_rows_pipe(const RowArgs<MT, VT, OT> a) {
  static_assert(S % NG == 0, "each stage is read by one group");
  static_assert(PAT != 2 || TPR == 1, "rows located from the tuple lengths: one thread per row");
  constexpr bool CB = PAT == 2;
  constexpr int CG = PIPE_CONSUMERS / NG;  // consumer threads per group
  constexpr int R = CG / TPR;
  pdl_trigger();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr bool SMALL = pat_small<MT, MODE, PAT>();
  constexpr bool STG = row_stage<MT, MODE, PAT, SB, R>();
  constexpr int VB = (int)sizeof(VT);
  // staged row data of the forms with a row-data area: the row pointers (CSR
  // and form 1) and the row vectors the mode reads per row (slot 0 iterate,
  // 1 right-hand side or b, 2 D)
  constexpr int NV = !STG ? 0
                     : MODE == PM_SWEEP ? 3
                     : (MODE == PM_RESID || MODE == PM_RINIT || MODE == PM_RTRUE || MODE == PM_RNORM) ? 1 : 0;
  constexpr bool SRP = STG && PAT != 2;
  const bool stg = (SRP || NV > 0) && a.stage_rows != 0;
  auto* P = reinterpret_cast<PipeSmem<MT, S, SB, SMALL, VB, R, STG>*>(smem_raw);
  int32_t* tab = reinterpret_cast<int32_t*>(smem_raw + sizeof(PipeSmem<MT, S, SB, SMALL, VB, R, STG>));  // PAT: offsets, lengths
  __shared__ double red[96];
  constexpr int VE = PipeTile<MT>::VE;
  constexpr int NCW = PIPE_CONSUMERS / 32;  // consumer warps
  const int n = a.n;
  const int ntiles = (n + R - 1) / R;
  const int G = gridDim.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&P->full[s], 1);
      mbar_init(&P->empty[s], NCW / NG);
    }
    mbar_fence_init();
  }
  if constexpr (PAT > 0) {  // setup data: valid before the previous kernel ends
    for (int j = threadIdx.x; j < a.ptab_n; j += blockDim.x) tab[j] = __ldg(&a.ptab[j]);
    for (int j = threadIdx.x; j < a.npat; j += blockDim.x) tab[a.ptab_n + j] = __ldg(&a.plen[j]);
  }
  __syncthreads();

  // copies of this block's k-th tile (producer lane only); the matrix does not
  // change during a solve, so the first S tiles are requested before waiting
  // for the previous kernel
  // the row vectors of this block's k-th tile (they change from kernel to
  // kernel: requested only after the wait on the previous kernel)
  auto issue_vectors = [&](int k, int stage) {
    if constexpr (NV > 0) {
      if (!stg) return;
      const int tile = blockIdx.x + k * G;
      const int row0 = tile * R, row1 = min(row0 + R, n);
      const uint32_t nb = (uint32_t)(((row1 - row0) * VB + 15) & ~15);
      unsigned char* ov = P->st[stage].ov;
      if constexpr (MODE == PM_SWEEP) {
        tma_load_1d(ov, a.x + row0, nb, &P->full[stage]);
        tma_load_1d(ov + R * VB, a.r + row0, nb, &P->full[stage]);
        tma_load_1d(ov + 2 * R * VB, a.dinv + row0, nb, &P->full[stage]);
      } else if constexpr (MODE == PM_RESID) {
        tma_load_1d(ov + R * VB, a.r + row0, nb, &P->full[stage]);
      } else {
        tma_load_1d(ov + R * VB, a.b + row0, nb, &P->full[stage]);
      }
    }
  };
  auto issue = [&](int k, int stage, bool with_vectors) {
    const int tile = blockIdx.x + k * G;
    const int row0 = tile * R, row1 = min(row0 + R, n);
    // row0 is a multiple of 32 and row1 one or n
    const int p0 = CB ? __ldg(&a.pcb[row0 >> 5]) : __ldg(&a.rp[row0]);
    const int p1 = CB ? __ldg(&a.pcb[(row1 + 31) >> 5]) : __ldg(&a.rp[row1]);
    const int av = p0 & ~(VE - 1), ac = p0 & ~3;
    const uint32_t bv = (uint32_t)(((p1 - av) * (int)sizeof(MT) + 15) & ~15);
    // PAT: the ids of rows row0 .. row1-1 (row0 is a multiple of R >= 32, so
    // the source is 16-byte aligned; the allocation is padded past n)
    const uint32_t bc = PAT > 0 ? (uint32_t)((row1 - row0 + 15) & ~15) : (uint32_t)(((p1 - ac) * 4 + 15) & ~15);
    // staged row data: row pointers row0 .. row1 and NV vectors (all sources
    // 16-byte aligned, allocations padded past their end)
    const uint32_t brp = (SRP && stg) ? (uint32_t)(((row1 - row0 + 1) * 4 + 15) & ~15) : 0u;
    const uint32_t bvec = (NV > 0 && stg) ? (uint32_t)NV * (uint32_t)(((row1 - row0) * VB + 15) & ~15) : 0u;
    mbar_expect_tx(&P->full[stage], bv + bc + brp + bvec);
    tma_load_1d(P->st[stage].v, a.v + av, bv, &P->full[stage]);
    if constexpr (PAT > 0) tma_load_1d(P->st[stage].c, a.pid + row0, bc, &P->full[stage]);
    else tma_load_1d(P->st[stage].c, a.ci + ac, bc, &P->full[stage]);
    if (brp) tma_load_1d(P->st[stage].rps, a.rp + row0, brp, &P->full[stage]);
    if (with_vectors) issue_vectors(k, stage);
  };
  const bool producer = warp == NCW && lane == 0;
  int issued = 0;
  // the true-residual check usually has nothing to do: read its flags first
  constexpr bool early = MODE != PM_RTRUE;
  if (!early) pdl_wait();
  if (early && producer)
    for (; issued < S && blockIdx.x + issued * G < ntiles; ++issued) issue(issued, issued, false);

  if (early) pdl_wait();  // the previous kernel's results (vectors, flags) are visible from here on
  if (early && producer)  // the row vectors of the tiles requested early
    for (int k = 0; k < issued; ++k) issue_vectors(k, k);
  bool skip = false;
  if constexpr (MODE == PM_SWEEP || MODE == PM_RESID || MODE == PM_SWEEP_PROLONG) skip = *a.skip != 0;
  else if constexpr (MODE == PM_DOTS) skip = a.st->done != 0;
  else if constexpr (MODE == PM_RTRUE) skip = a.st->done || !a.st->need_true;
  if (skip) {
    if (producer)  // drain the copies already requested, bounded
      for (int k = 0; k < issued; ++k) mbar_wait(&P->full[k % S], 0);
    return;
  }
  if (!early && producer)
    for (; issued < S && blockIdx.x + issued * G < ntiles; ++issued) issue(issued, issued, true);

  double acc[3] = {0.0, 0.0, 0.0};
  const bool first = (MODE == PM_DOTS) ? (a.st->it == 0) : false;

  if (warp == NCW) {
    // ---------------- producer warp ----------------
    if (lane == 0) {
      int k = issued;
      bool aborted = false;
      for (;; ++k) {
        const int tile = blockIdx.x + k * G;
        if (tile >= ntiles) break;
        const int stage = k % S;
        if (!mbar_wait(&P->empty[stage], (uint32_t)(((k / S) - 1) & 1))) {
          atomicOr(a.flags, ST_TIMEOUT);
          aborted = true;
          break;
        }
        issue(k, stage, true);
      }
      if (aborted) {  // drain: the last copy issued into each stage, bounded
        for (int j = 1; j <= S && k - j >= 0; ++j) {
          const int kk = k - j;
          mbar_wait(&P->full[kk % S], (uint32_t)((kk / S) & 1));
        }
      }
    }
    __syncwarp();  // reconverge before the block-wide reduction below
  } else {
    // ---------------- consumer warps ----------------
    const int grp = (int)threadIdx.x / CG, tg = (int)threadIdx.x % CG;  // group, thread in group
    for (int k = grp;; k += NG) {
      const int tile = blockIdx.x + k * G;
      if (tile >= ntiles) break;
      const int stage = k % S;
      const int row0 = tile * R, row1 = min(row0 + R, n);
      const int sub = tg % TPR;  // lane within the row's group
      const int row = row0 + tg / TPR;
      const bool live = row < row1;
      const bool lead = live && sub == 0;      // the lane that finishes the row
      const bool rows_staged = SRP && stg;  // row pointers from the stage (after the wait)
      const bool vecs_staged = NV > 0 && stg;  // row vectors from the stage
      int p0 = 0;
      if (!rows_staged) p0 = CB ? __ldg(&a.pcb[row0 >> 5]) : __ldg(&a.rp[row0]);
      int q0 = 0, q1 = 0, qs = 0;
      VT own = 0, rr = 0, dd = 0, qq = 0;
      OT zn = 0;  // PM_SWEEP_PROLONG: the row's new value
      int wbase = 0;  // CB: first entry of the warp's first row
      if constexpr (CB) {
        if (row - lane < n) wbase = __ldg(&a.pcb[(row - lane) >> 5]);
      } else if (live && !rows_staged) {
        qs = __ldg(&a.rp[row]);
        q0 = qs + sub;
        q1 = __ldg(&a.rp[row + 1]);
      }
      if (lead && !vecs_staged) {
        if constexpr (MODE == PM_SWEEP || MODE == PM_SWEEP_PROLONG) {
          own = __ldg(&a.x[row]);
          rr = __ldg(&a.r[row]);
          dd = __ldg(&a.dinv[row]);
        } else if constexpr (MODE == PM_RESID) {
          rr = __ldg(&a.r[row]);
        } else if constexpr (MODE == PM_DOTS) {
          own = __ldg(&a.x[row]);
          rr = __ldg(&a.r[row]);
          if (!first) qq = __ldg(&a.q[row]);
        } else if constexpr (MODE == PM_RINIT || MODE == PM_RTRUE || MODE == PM_RNORM) {
          rr = __ldg(&a.b[row]);
        }
      }
      if (!mbar_wait_warp(&P->full[stage], (uint32_t)((k / S) & 1))) {
        if (lane == 0) atomicOr(a.flags, ST_TIMEOUT);
        break;
      }
      const PipeTile<MT, SB, SMALL, VB, R, STG>& T = P->st[stage];
      if (rows_staged) {
        p0 = T.rps[0];
        if (live) {
          qs = T.rps[row - row0];
          q0 = qs + sub;
          q1 = T.rps[row - row0 + 1];
        }
      }
      if constexpr (NV > 0) {
        if (vecs_staged && lead) {
          const VT* ov = reinterpret_cast<const VT*>(T.ov);
          const int j = row - row0;
          if constexpr (MODE == PM_SWEEP) {
            own = ov[j];
            rr = ov[R + j];
            dd = ov[2 * R + j];
          } else {
            rr = ov[R + j];
          }
        }
      }
      const int av = p0 & ~(VE - 1), ac = p0 & ~3;
      // residuals, and sweeps in standard stages, accumulate
      // r_i - sum_j a_ij x_j from r_i (the lead lane holds r_i, the others 0):
      // one FP64 operation per row fewer than summing first and subtracting, on
      // a part whose FP64 issue rate is a co-limit of these kernels (7-point
      // FP64 level-0 sweep 81.2 -> 80.2 us, level 1 11.8 -> 11.0 us, 27-point
      // residual 185.6 -> 176.9 us).  Sweeps in the long-row forms (SB > 1: one
      // block per multiprocessor, 8 consumer warps) sum first: starting from
      // r_i made the 27-point FP64 sweep 166 -> 199 us there (measured).
      constexpr bool FROM_R =
          MODE == PM_RESID || ((MODE == PM_SWEEP || MODE == PM_SWEEP_PROLONG) && SB == 1 && NG == 1);
      VT s = 0;
      if constexpr (PAT > 0) {
        // the row's offsets, indexed by entry position within the row
        const int pr = live ? (int)reinterpret_cast<const uint8_t*>(T.c)[row - row0] : 0;
        const int32_t* po = tab + pr * a.pk;
        if constexpr (CB) {  // the row's entries: after those of the warp's earlier rows
          const int len = live ? tab[a.ptab_n + pr] : 0;
          int incl = len;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
          }
          qs = wbase + incl - len;
          q0 = qs;
          q1 = qs + len;
        }
        if constexpr (FROM_R) {
          s = rr;
#pragma unroll 8
          for (int q = q0; q < q1; q += TPR)
            s -= (VT)to_acc(T.v[q - av]) * __ldg(&a.x[amg_chk(row + po[q - qs], n)]);
        } else {
#pragma unroll 8
          for (int q = q0; q < q1; q += TPR)
            s += (VT)to_acc(T.v[q - av]) * __ldg(&a.x[amg_chk(row + po[q - qs], n)]);
        }
      } else if constexpr (FROM_R) {
        s = rr;
#pragma unroll 8
        for (int q = q0; q < q1; q += TPR) s -= (VT)to_acc(T.v[q - av]) * __ldg(&a.x[amg_chk(T.c[q - ac], n)]);
      } else {
#pragma unroll 8
        for (int q = q0; q < q1; q += TPR) s += (VT)to_acc(T.v[q - av]) * __ldg(&a.x[amg_chk(T.c[q - ac], n)]);
      }
      if constexpr (TPR > 1) s = group_sum<TPR>(s);
      __syncwarp();
      if (lane == 0) mbar_arrive(&P->empty[stage]);  // this warp is done with the stage
      if (lead) {
        if constexpr (MODE == PM_SWEEP) {
          a.out[row] = (OT)(own + dd * (FROM_R ? s : rr - s));
        } else if constexpr (MODE == PM_SWEEP_PROLONG) {
          zn = (OT)(own + dd * (FROM_R ? s : rr - s));
          a.out[row] = zn;
        } else if constexpr (MODE == PM_RESID) {
          a.out[row] = (OT)(FROM_R ? s : rr - s);
        } else if constexpr (MODE == PM_SPMV) {
          a.out[row] = (OT)s;
        } else if constexpr (MODE == PM_DOTS) {
          a.out[row] = (OT)s;
          acc[0] += (double)own * (double)rr;
          acc[1] += (double)own * (double)s;
          if (!first) acc[2] += (double)own * (double)qq;
        } else {
          const double ri = (double)rr - (double)s;
          if constexpr (MODE != PM_RNORM) a.out[row] = (OT)ri;
          acc[0] += ri * ri;
          if constexpr (MODE == PM_RINIT) acc[1] += (double)rr * (double)rr;
        }
      }
      if constexpr (MODE == PM_SWEEP_PROLONG) {
        if constexpr (TPR > 1) zn = __shfl_sync(0xffffffffu, zn, 0, TPR);  // from the row's lead lane
        if (live) prolong_members<TPR>(a, row, sub, zn);
      }
    }
  }

  if constexpr (MODE == PM_DOTS) {
    if (!grid_sum<3>(acc, a.partial, a.counter, red) || threadIdx.x != 0) return;
    FcgState* st = a.st;
    if (st->timing) return;
    const double alpha = acc[0], beta = acc[1], gamma = acc[2];
    double rho_new, g;
    if (first) {
      rho_new = beta;
      g = 0.0;
    } else {
      rho_new = beta - gamma * gamma / st->rho;
      g = gamma / st->rho;
    }
    if (!(rho_new > 0.0) || !isfinite(rho_new)) {
      st->status = AMG_ERR_BREAKDOWN;
      st->done = 1;
    } else {
      st->g = g;
      st->a = alpha / rho_new;
      st->rho = rho_new;
    }
  } else if constexpr (MODE == PM_RINIT || MODE == PM_RTRUE || MODE == PM_RNORM) {
    double acc2[2] = {acc[0], acc[1]};
    if (!grid_sum<2>(acc2, a.partial, a.counter, red) || threadIdx.x != 0) return;
    fcg_residual_epilogue<MODE == PM_RINIT ? RES_INIT : (MODE == PM_RTRUE ? RES_TRUE : RES_NORM)>(a.st, acc2);
  }
}

// dynamic shared memory of a pipelined row kernel: the stages and barriers,
// and for the pattern forms the offset table (16-byte granules)
template <typename MT, typename VT, int S, int SB, int MODE, int PAT, int R>
static constexpr int pipe_smem(int tab_n) {
  return (int)sizeof(PipeSmem<MT, S, SB, pat_small<MT, MODE, PAT>(), (int)sizeof(VT), R,
                              row_stage<MT, MODE, PAT, SB, R>()>) +
         (PAT > 0 ? ((tab_n * 4 + 15) & ~15) : 0);
}

// grid of a persistent pipelined kernel: one wave of resident blocks, at most
// one block per tile
template <int TPR, int S, int MODE, typename MT, typename VT, typename OT, int SB = 1, int NG = 1, int PAT = 0>
static int pipe_grid(int n, int tab_n = 0) {
  // resident blocks per multiprocessor, by table size in 256-byte steps
  static int bps_by[PAT_TAB_MAX * 4 / 256 + 1] = {0};
  static bool attr = false;
  constexpr int R = PIPE_CONSUMERS / NG / TPR;
  auto kern = k_rows_pipe<TPR, S, MODE, MT, VT, OT, SB, NG, PAT>;
  if (!attr) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, pipe_smem<MT, VT, S, SB, MODE, PAT, R>(PAT_TAB_MAX));
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    attr = true;
  }
  int& bps = bps_by[PAT > 0 ? (tab_n * 4 + 255) / 256 : 0];
  if (bps <= 0) {  // sized for the table rounded up to its 256-byte step
    int b = 0;
    const size_t occ = sizeof(PipeSmem<MT, S, SB, pat_small<MT, MODE, PAT>(), (int)sizeof(VT), R,
                                       row_stage<MT, MODE, PAT, SB, R>()>) +
                       (PAT > 0 ? (size_t)((tab_n * 4 + 255) & ~255) : 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, PIPE_CONSUMERS + 32, occ);
    bps = b < 1 ? 1 : b;
  }
  const int ntiles = (n + R - 1) / R;
  const int g = amg_num_sms() * bps;
  return ntiles < g ? ntiles : g;
}

template <int TPR, int S, int MODE, typename MT, typename VT, typename OT, int SB = 1, int NG = 1, int PAT = 0>
static void launch_pipe(cudaStream_t s, const RowArgs<MT, VT, OT>& a) {
  constexpr int R = PIPE_CONSUMERS / NG / TPR;
  const int tab_n = PAT > 0 ? a.ptab_n + a.npat : 0;  // offsets, then lengths
  const int grid = pipe_grid<TPR, S, MODE, MT, VT, OT, SB, NG, PAT>(a.n, tab_n);
  const int smem = pipe_smem<MT, VT, S, SB, MODE, PAT, R>(tab_n);
  amg_launch(k_rows_pipe<TPR, S, MODE, MT, VT, OT, SB, NG, PAT>, dim3(grid), dim3(PIPE_CONSUMERS + 32), (size_t)smem, s,
             a);
}
