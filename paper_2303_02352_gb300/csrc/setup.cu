// Hierarchy construction on the GPU: Alg. 3 of arXiv:2303.02352 (coarsening
// by maximum-weight matching) with the s-fold composition of pairwise
// prolongators of Sec. 3.1, the l1-Jacobi diagonal of Sec. 3.1, and the
// low-precision copies used by the mixed-precision V-cycle.
//
// Matching: the suitor algorithm (Sec. 4.1) under a strict total order on the
// edges (weight descending, ties broken by the smaller endpoint pair).  Under a
// strict order the suitor matching equals the greedy one, whatever the order in
// which proposals land, so the result is deterministic.  Each vertex keeps its
// eligible neighbours sorted by that order; the record of who currently courts
// vertex v is one 64-bit word (rank of the suitor in v's own order, suitor id)
// updated with atomicMin, so a better suitor always wins and the displaced one
// resumes its scan.
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <chrono>
#include <cstdlib>
#include <algorithm>
#include <vector>

#include "amg_internal.cuh"

// ---------------------------------------------------------------------------
// errors and allocation

amg_status amg_fail(amg_handle* h, amg_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (h) h->err = buf;
  return s;
}

void* amg_alloc(amg_handle* h, size_t bytes) {
  size_t sz = ((bytes + 255) / 256) * 256 + 256;
  void* p = nullptr;
  if (h->fail_alloc_after >= 0 && h->n_allocs++ >= h->fail_alloc_after) return nullptr;  // test hook
  if (cudaMalloc(&p, sz) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (cudaMemsetAsync(p, 0, sz, h->stream) != cudaSuccess) {
    cudaFree(p);
    return nullptr;
  }
  h->bufs.push_back({p, sz});
  return p;
}

void amg_release(amg_handle* h, void* p) {
  if (!p) return;
  for (size_t i = 0; i < h->bufs.size(); ++i)
    if (h->bufs[i].p == p) {
      cudaFree(p);
      h->bufs[i] = h->bufs.back();
      h->bufs.pop_back();
      return;
    }
}

void amg_free_all(amg_handle* h) {
  for (auto& b : h->bufs) cudaFree(b.p);
  h->bufs.clear();
}

// ---------------------------------------------------------------------------
// input validation (structure, then symmetry)

__global__ void k_validate(int n, int nnz, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const double* __restrict__ v, int32_t* __restrict__ diagpos, int* flags) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int p0 = rp[i], p1 = rp[i + 1];
  if (p0 < 0 || p1 < p0 || p1 > nnz) {
    atomicOr(flags, ST_BADPTR);
    diagpos[i] = -1;
    return;
  }
  int dp = -1, prev = -1;
  for (int p = p0; p < p1; ++p) {
    int j = ci[p];
    if (j < 0 || j >= n || j <= prev) atomicOr(flags, ST_BADCOL);
    prev = j;
    double a = v[p];
    if (!isfinite(a)) atomicOr(flags, ST_NAN);
    if (j == i) dp = p;
  }
  diagpos[i] = dp;
  if (dp < 0) atomicOr(flags, ST_NODIAG);
  else if (!(v[dp] > 0.0)) atomicOr(flags, ST_NOTPOS);
}

__device__ __forceinline__ int find_col(const int32_t* __restrict__ ci, int lo, int hi, int col) {
  hi -= 1;
  while (lo <= hi) {
    int mid = lo + ((hi - lo) >> 1);
    int c = ci[mid];
    if (c == col) return mid;
    if (c < col) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

__global__ void k_check_sym(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                            const double* __restrict__ v, int* flags) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    int j = ci[p];
    if (j == i) continue;
    int q = find_col(ci, rp[j], rp[j + 1], i);
    if (q < 0 || __double_as_longlong(v[q]) != __double_as_longlong(v[p])) {
      atomicOr(flags, ST_ASYM);
      return;
    }
  }
}

// ---------------------------------------------------------------------------
// matching weights: w_ij = 1 - 2 a_ij w_i w_j / (a_ii w_i^2 + a_jj w_j^2) with
// the unit smooth vector, every operation rounded separately (no fused
// multiply-add) so that the result is reproducible bit for bit

__global__ void k_diag(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                       const double* __restrict__ v, double* __restrict__ dg) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double d = 0.0;
  for (int p = rp[i]; p < rp[i + 1]; ++p)
    if (ci[p] == i) d = v[p];
  dg[i] = d;
}

// decoupled aggregation (Sec. 4.1): the row block of row i among the np
// contiguous blocks [bnd[q], bnd[q+1])
__device__ __forceinline__ int part_of(int i, int np, const int32_t* __restrict__ bnd) {
  int lo = 0, hi = np - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (i >= bnd[mid]) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void k_weights(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                          const double* __restrict__ v, const double* __restrict__ dg, int np,
                          const int32_t* __restrict__ bnd, double* __restrict__ wgt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double wi = 1.0, wj = 1.0;
  const double di = dg[i];
  const int pi = np > 1 ? part_of(i, np, bnd) : 0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    int j = ci[p];
    double a = v[p];
    if (j == i || a == 0.0 || (np > 1 && part_of(j, np, bnd) != pi)) {
      wgt[p] = 0.0;
      continue;
    }
    double t = __dmul_rn(2.0, a);
    t = __dmul_rn(t, wi);
    t = __dmul_rn(t, wj);
    double den = __dadd_rn(__dmul_rn(__dmul_rn(di, wi), wi), __dmul_rn(__dmul_rn(dg[j], wj), wj));
    wgt[p] = __dsub_rn(1.0, __ddiv_rn(t, den));
  }
}

// rank of every eligible entry of row v in v's strict order (weight desc, then
// column asc); sorted adjacency positions; eligible count per row
__global__ void k_rank(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                       const double* __restrict__ wgt, int32_t* __restrict__ rank_of, int32_t* __restrict__ srt_pos,
                       int32_t* __restrict__ cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int p0 = rp[i], p1 = rp[i + 1], c = 0;
  for (int p = p0; p < p1; ++p) {
    double w = wgt[p];
    int j = ci[p];
    if (j == i || !(w > 0.0)) {
      rank_of[p] = -1;
      continue;
    }
    ++c;
    int r = 0;
    for (int q = p0; q < p1; ++q) {
      if (q == p) continue;
      double w2 = wgt[q];
      int j2 = ci[q];
      if (j2 == i || !(w2 > 0.0)) continue;
      if (w2 > w || (w2 == w && j2 < j)) ++r;
    }
    rank_of[p] = r;
    srt_pos[p0 + r] = p;
  }
  cnt[i] = c;
}

// for row u's k-th best neighbour v: v's id, and u's rank in v's order
__global__ void k_other_rank(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                             const int32_t* __restrict__ rank_of, const int32_t* __restrict__ srt_pos,
                             const int32_t* __restrict__ cnt, int32_t* __restrict__ srt_col,
                             int32_t* __restrict__ key_rank, int* flags) {
  int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n) return;
  int base = rp[u];
  for (int k = 0; k < cnt[u]; ++k) {
    int p = srt_pos[base + k];
    int v = ci[p];
    int q = find_col(ci, rp[v], rp[v + 1], u);
    int rk = q >= 0 ? rank_of[q] : -1;
    if (rk < 0) {  // the matrix is bitwise symmetric, so this cannot happen
      atomicOr(flags, ST_ASYM);
      rk = 0x7fffffff;
    }
    srt_col[base + k] = v;
    key_rank[base + k] = rk;
  }
}

#define SUITOR_EMPTY 0xffffffffffffffffull

// One thread per vertex; a thread follows the chain of displaced suitors.
// Bounded: every successful atomicMin strictly improves a vertex's record and
// every failed attempt advances a scan pointer, so the total number of loop
// steps over all threads is at most 2*nnz + n; `cap` is set above that and the
// loop stops with ST_TIMEOUT if it is ever reached.
__global__ void k_suitor(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ cnt,
                         const int32_t* __restrict__ srt_col, const int32_t* __restrict__ key_rank,
                         unsigned long long* suitor, int32_t* next, long long cap, int* flags) {
  int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n) return;
  int cur = u;
  long long steps = 0;
  while (cur >= 0) {
    const int base = rp[cur], c = cnt[cur];
    int k = *((volatile int32_t*)&next[cur]);
    int partner = -1;
    unsigned long long key = 0;
    for (; k < c; ++k) {
      if (++steps > cap) {
        atomicOr(flags, ST_TIMEOUT);
        return;
      }
      int v = srt_col[base + k];
      unsigned long long kk = ((unsigned long long)(unsigned)key_rank[base + k] << 32) | (unsigned)cur;
      unsigned long long now = *((volatile unsigned long long*)&suitor[v]);
      if (kk < now) {
        partner = v;
        key = kk;
        break;
      }
    }
    if (partner < 0) {
      next[cur] = c;
      break;
    }
    next[cur] = k + 1;  // published before the proposal lands
    __threadfence();
    unsigned long long old = atomicMin(&suitor[partner], key);
    __threadfence();
    if (old > key) cur = (old == SUITOR_EMPTY) ? -1 : (int)(old & 0xffffffffull);
    // else: a better suitor got there first; cur rescans from k + 1
  }
}

__global__ void k_mate(int n, const unsigned long long* __restrict__ suitor, int32_t* __restrict__ mate,
                       int32_t* __restrict__ opener) {
  int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n) return;
  unsigned long long s = suitor[u];
  int m = -1;
  if (s != SUITOR_EMPTY) {
    int v = (int)(s & 0xffffffffull);
    unsigned long long sv = suitor[v];
    if (sv != SUITOR_EMPTY && (int)(sv & 0xffffffffull) == u) m = v;
  }
  mate[u] = m;
  opener[u] = (m < 0 || u < m) ? 1 : 0;
}

// ---------------------------------------------------------------------------
// exclusive scan of int32 (three phases: block scan, scan of block sums, add)

#define SCAN_ITEMS 4
#define SCAN_TILE (AMG_BLOCK * SCAN_ITEMS)

__global__ void k_scan_tiles(int n, const int32_t* __restrict__ in, int32_t* __restrict__ out,
                             int32_t* __restrict__ tile_sum) {
  __shared__ int32_t s[AMG_BLOCK];
  int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
  int32_t x[SCAN_ITEMS], tot = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    x[k] = (base + k < n) ? in[base + k] : 0;
    tot += x[k];
  }
  s[threadIdx.x] = tot;
  __syncthreads();
  for (int off = 1; off < AMG_BLOCK; off <<= 1) {
    int32_t y = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
    __syncthreads();
    s[threadIdx.x] += y;
    __syncthreads();
  }
  int32_t run = s[threadIdx.x] - tot;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    if (base + k < n) out[base + k] = run;
    run += x[k];
  }
  if (threadIdx.x == AMG_BLOCK - 1) tile_sum[blockIdx.x] = s[threadIdx.x];
}

// single block: exclusive scan of the tile sums in place, total to *total
__global__ void k_scan_sums(int m, int32_t* tile_sum, int32_t* total) {
  __shared__ int32_t s[AMG_BLOCK];
  int32_t carry = 0;
  for (int c0 = 0; c0 < m; c0 += AMG_BLOCK) {
    int i = c0 + threadIdx.x;
    int32_t x = i < m ? tile_sum[i] : 0;
    s[threadIdx.x] = x;
    __syncthreads();
    for (int off = 1; off < AMG_BLOCK; off <<= 1) {
      int32_t y = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
      __syncthreads();
      s[threadIdx.x] += y;
      __syncthreads();
    }
    if (i < m) tile_sum[i] = carry + s[threadIdx.x] - x;
    int32_t chunk = s[AMG_BLOCK - 1];
    __syncthreads();
    carry += chunk;
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_add(int n, int32_t* __restrict__ out, const int32_t* __restrict__ tile_sum) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] += tile_sum[i / SCAN_TILE];
}

// out[0..n-1] = exclusive scan of in, *total = sum (device).  scratch >= tiles ints.
static void scan_exclusive(cudaStream_t s, int n, const int32_t* in, int32_t* out, int32_t* scratch, int32_t* total) {
  int tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (tiles < 1) tiles = 1;
  k_scan_tiles<<<tiles, AMG_BLOCK, 0, s>>>(n, in, out, scratch);
  k_scan_sums<<<1, AMG_BLOCK, 0, s>>>(tiles, scratch, total);
  if (n > 0) k_scan_add<<<amg_blocks(n), AMG_BLOCK, 0, s>>>(n, out, scratch);
}

// the same scan for the other translation units (the general sparse product)
void amg_scan_exclusive(cudaStream_t s, int n, const int32_t* in, int32_t* out, int32_t* scratch, int32_t* total) {
  scan_exclusive(s, n, in, out, scratch, total);
}
int amg_scan_scratch_ints(int n) { return n / SCAN_TILE + 2; }

__global__ void k_number(int n, const int32_t* __restrict__ mate, const int32_t* __restrict__ opener,
                         const int32_t* __restrict__ pos, int32_t* __restrict__ agg, int32_t* __restrict__ open_idx) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (opener[i]) {
    agg[i] = pos[i];
    open_idx[pos[i]] = i;
  } else {
    agg[i] = pos[mate[i]];
  }
}

// ---------------------------------------------------------------------------
// pairwise Galerkin product A_c = P^T A P, canonical order: for each coarse
// pair (I, J) the entries a_ij with i in I (ascending) and agg(j) = J, in CSR
// order, summed one after the other starting from the first term.  Distinct J
// are emitted in ascending order by repeated minimum search.

template <bool NUMERIC>
__global__ void k_galerkin_pair(int nc, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                const double* __restrict__ v, const int32_t* __restrict__ agg,
                                const int32_t* __restrict__ open_idx, const int32_t* __restrict__ mate,
                                int32_t* __restrict__ cnt_or_rpc, int32_t* __restrict__ ci_c, double* __restrict__ v_c) {
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  int i0 = open_idx[I];
  int i1 = mate[i0];
  int a0 = rp[i0], a1 = rp[i0 + 1];
  int b0 = 0, b1 = 0;
  if (i1 >= 0) {
    b0 = rp[i1];
    b1 = rp[i1 + 1];
  }
  int out = NUMERIC ? cnt_or_rpc[I] : 0;
  int last = -1, count = 0;
  for (;;) {
    int J = 0x7fffffff;
    for (int p = a0; p < a1; ++p) {
      int k = agg[ci[p]];
      if (k > last && k < J) J = k;
    }
    for (int p = b0; p < b1; ++p) {
      int k = agg[ci[p]];
      if (k > last && k < J) J = k;
    }
    if (J == 0x7fffffff) break;
    if (NUMERIC) {
      double acc = 0.0;
      bool first = true;
      for (int p = a0; p < a1; ++p)
        if (agg[ci[p]] == J) {
          acc = first ? v[p] : acc + v[p];
          first = false;
        }
      for (int p = b0; p < b1; ++p)
        if (agg[ci[p]] == J) {
          acc = first ? v[p] : acc + v[p];
          first = false;
        }
      ci_c[out + count] = J;
      v_c[out + count] = acc;
    }
    ++count;
    last = J;
  }
  if (!NUMERIC) cnt_or_rpc[I] = count;
}

// A_c(I,J) := A_c(J,I) for J < I, so that A_c is symmetric bit for bit
__global__ void k_mirror(int nc, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, double* v) {
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  for (int p = rp[I]; p < rp[I + 1]; ++p) {
    int J = ci[p];
    if (J >= I) break;
    int q = find_col(ci, rp[J], rp[J + 1], I);
    if (q >= 0) v[p] = v[q];
  }
}

// block boundaries move to the aggregate ids of the blocks' first rows
__global__ void k_update_bnd(int np, int32_t* bnd, const int32_t* __restrict__ agg, int nfine, int nc) {
  for (int q = threadIdx.x; q < np; q += blockDim.x) bnd[q] = bnd[q] < nfine ? agg[bnd[q]] : nc;
  if (threadIdx.x == 0) bnd[np] = nc;
}

__global__ void k_compose(int n, int32_t* __restrict__ comp, const int32_t* __restrict__ agg) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) comp[i] = agg[comp[i]];
}

__global__ void k_iota(int n, int32_t* __restrict__ a) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = i;
}

// members of each aggregate, ascending: count, scan, place, sort each list
__global__ void k_count(int n, const int32_t* __restrict__ agg, int32_t* __restrict__ cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(&cnt[agg[i]], 1);
}

__global__ void k_place(int n, const int32_t* __restrict__ agg, const int32_t* __restrict__ mptr,
                        int32_t* __restrict__ fill, int32_t* __restrict__ mem) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int J = agg[i];
  int s = atomicAdd(&fill[J], 1);
  mem[mptr[J] + s] = i;
}

__global__ void k_sort_members(int nc, const int32_t* __restrict__ mptr, int32_t* __restrict__ mem) {
  int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= nc) return;
  int a = mptr[J], b = mptr[J + 1];
  for (int x = a + 1; x < b; ++x) {
    int key = mem[x], y = x - 1;
    while (y >= a && mem[y] > key) {
      mem[y + 1] = mem[y];
      --y;
    }
    mem[y + 1] = key;
  }
}

__global__ void k_maxrow(int n, const int32_t* __restrict__ rp, int* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicMax(out, rp[i + 1] - rp[i]);
}

// largest number of entries in a tile of R consecutive rows
__global__ void k_tile_max(int n, const int32_t* __restrict__ rp, int R, int* out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int r0 = t * R;
  if (r0 >= n) return;
  const int r1 = min(n, r0 + R);
  atomicMax(out, rp[r1] - rp[r0]);
}

// bandwidth max |i - j| (columns are sorted: the first and last entry decide)
__global__ void k_bandwidth(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || rp[i + 1] == rp[i]) return;
  atomicMax(out, max(i - ci[rp[i]], ci[rp[i + 1] - 1] - i));
}

// l1-Jacobi: M_ii = sum_j |a_ij| (CSR order), D_i = omega_i / M_ii
// (jacobi: D_i = omega_i / a_ii, Listing 1 relax_type 0; the l1 norms are kept)
__global__ void k_l1(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                     const double* __restrict__ v, const double* __restrict__ omega, double* __restrict__ l1,
                     double* __restrict__ dinv, float* __restrict__ dinvf, int jacobi) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0, a = 0.0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    s += fabs(v[p]);
    if (ci[p] == i) a = v[p];
  }
  l1[i] = s;
  double om = omega ? omega[i] : 1.0;
  double d = om / (jacobi ? a : s);
  dinv[i] = d;
  if (dinvf) dinvf[i] = __double2float_rn(d);
}

__global__ void k_round_vals(int64_t nnz, const double* __restrict__ v, float* __restrict__ vf, bf16* __restrict__ vb) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nnz) return;
  float f = __double2float_rn(v[p]);
  if (vf) vf[p] = f;
  if (vb) vb[p] = __float2bfloat16_rn(f);
}

// ---------------------------------------------------------------------------
// host side

struct PCsr {  // a pairwise-step matrix (device)
  int n = 0;
  int64_t nnz = 0;
  int32_t* rp = nullptr;
  int32_t* ci = nullptr;
  double* v = nullptr;
};

static amg_status sync_read(amg_handle* h, const int32_t* dev, int32_t* host_val) {
  AMG_CK(h, cudaMemcpyAsync(host_val, dev, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  AMG_CK(h, cudaStreamSynchronize(h->stream));
  return AMG_OK;
}

static amg_status check_flags(amg_handle* h, const char* where) {
  int f = 0;
  AMG_CK(h, cudaMemcpyAsync(&f, h->dev_flags, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  AMG_CK(h, cudaStreamSynchronize(h->stream));
  AMG_CK(h, cudaGetLastError());
  if (!f) return AMG_OK;
  AMG_CK(h, cudaMemsetAsync(h->dev_flags, 0, sizeof(int), h->stream));
  if (f & ST_TIMEOUT) return amg_fail(h, AMG_ERR_TIMEOUT, "%s: bounded device loop hit its cap", where);
  if (f & ST_BADPTR) return amg_fail(h, AMG_ERR_INVALID_ARG, "%s: row pointers not monotone or out of range", where);
  if (f & ST_BADCOL) return amg_fail(h, AMG_ERR_INVALID_ARG, "%s: column index out of range or not strictly ascending", where);
  if (f & ST_NODIAG) return amg_fail(h, AMG_ERR_INVALID_ARG, "%s: a row has no stored diagonal", where);
  if (f & ST_NAN) return amg_fail(h, AMG_ERR_INVALID_ARG, "%s: non-finite matrix value", where);
  if (f & ST_NOTPOS) return amg_fail(h, AMG_ERR_NOT_SPD, "%s: non-positive diagonal", where);
  if (f & ST_ASYM) return amg_fail(h, AMG_ERR_INVALID_ARG, "%s: matrix is not symmetric bit for bit", where);
  return amg_fail(h, AMG_ERR_CUDA, "%s: device error flags %d", where, f);
}

// one pairwise step: matching on `cur`, aggregation; returns nc and agg (device)
static amg_status pairwise_step(amg_handle* h, const PCsr& cur, int np, const int32_t* bnd, int32_t* agg,
                                int32_t* open_idx, int32_t* mate, int* nc_out) {
  cudaStream_t s = h->stream;
  const int n = cur.n;
  const int64_t nnz = cur.nnz;
  double *dg, *wgt;
  int32_t *rank_of, *srt_pos, *cnt, *srt_col, *key_rank, *next, *opener, *pos, *scratch, *total;
  unsigned long long* suitor;
  AMG_ALLOC(h, dg, double, n);
  AMG_ALLOC(h, wgt, double, nnz);
  AMG_ALLOC(h, rank_of, int32_t, nnz);
  AMG_ALLOC(h, srt_pos, int32_t, nnz);
  AMG_ALLOC(h, srt_col, int32_t, nnz);
  AMG_ALLOC(h, key_rank, int32_t, nnz);
  AMG_ALLOC(h, cnt, int32_t, n);
  AMG_ALLOC(h, next, int32_t, n);
  AMG_ALLOC(h, opener, int32_t, n);
  AMG_ALLOC(h, pos, int32_t, n);
  AMG_ALLOC(h, scratch, int32_t, n / SCAN_TILE + 2);
  AMG_ALLOC(h, total, int32_t, 1);
  AMG_ALLOC(h, suitor, unsigned long long, n);
  const int nb = amg_blocks(n);
  k_diag<<<nb, AMG_BLOCK, 0, s>>>(n, cur.rp, cur.ci, cur.v, dg);
  k_weights<<<nb, AMG_BLOCK, 0, s>>>(n, cur.rp, cur.ci, cur.v, dg, np, bnd, wgt);
  k_rank<<<nb, AMG_BLOCK, 0, s>>>(n, cur.rp, cur.ci, wgt, rank_of, srt_pos, cnt);
  k_other_rank<<<nb, AMG_BLOCK, 0, s>>>(n, cur.rp, cur.ci, rank_of, srt_pos, cnt, srt_col, key_rank, h->dev_flags);
  AMG_CK(h, cudaMemsetAsync(suitor, 0xff, sizeof(unsigned long long) * (size_t)n, s));
  long long cap = 2 * (long long)nnz + (long long)n + 1024;
  if (h->suitor_cap >= 0) cap = h->suitor_cap;  // test hook
  k_suitor<<<nb, AMG_BLOCK, 0, s>>>(n, cur.rp, cnt, srt_col, key_rank, suitor, next, cap, h->dev_flags);
  k_mate<<<nb, AMG_BLOCK, 0, s>>>(n, suitor, mate, opener);
  scan_exclusive(s, n, opener, pos, scratch, total);
  k_number<<<nb, AMG_BLOCK, 0, s>>>(n, mate, opener, pos, agg, open_idx);
  amg_status st = check_flags(h, "matching");
  if (st != AMG_OK) return st;
  int nc = 0;
  st = sync_read(h, total, &nc);
  if (st != AMG_OK) return st;
  for (void* p : {(void*)dg, (void*)wgt, (void*)rank_of, (void*)srt_pos, (void*)srt_col, (void*)key_rank,
                  (void*)cnt, (void*)next, (void*)opener, (void*)pos, (void*)scratch,
                  (void*)total, (void*)suitor})
    amg_release(h, p);
  *nc_out = nc;
  return AMG_OK;
}

static amg_status galerkin_step(amg_handle* h, const PCsr& cur, const int32_t* agg, const int32_t* open_idx,
                                const int32_t* mate, int nc, PCsr* out) {
  cudaStream_t s = h->stream;
  int32_t *cnt, *scratch, *total;
  AMG_ALLOC(h, cnt, int32_t, nc);
  AMG_ALLOC(h, scratch, int32_t, nc / SCAN_TILE + 2);
  AMG_ALLOC(h, total, int32_t, 1);
  const int nb = amg_blocks(nc);
  k_galerkin_pair<false><<<nb, AMG_BLOCK, 0, s>>>(nc, cur.rp, cur.ci, cur.v, agg, open_idx, mate, cnt, nullptr, nullptr);
  out->n = nc;
  AMG_ALLOC(h, out->rp, int32_t, nc + 1);
  scan_exclusive(s, nc, cnt, out->rp, scratch, total);
  AMG_CK(h, cudaMemcpyAsync(out->rp + nc, total, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  int nnz_c = 0;
  amg_status st = sync_read(h, total, &nnz_c);
  if (st != AMG_OK) return st;
  out->nnz = nnz_c;
  AMG_ALLOC(h, out->ci, int32_t, nnz_c);
  AMG_ALLOC(h, out->v, double, nnz_c);
  k_galerkin_pair<true><<<nb, AMG_BLOCK, 0, s>>>(nc, cur.rp, cur.ci, cur.v, agg, open_idx, mate, out->rp, out->ci, out->v);
  k_mirror<<<nb, AMG_BLOCK, 0, s>>>(nc, out->rp, out->ci, out->v);
  AMG_CK(h, cudaGetLastError());
  amg_release(h, cnt);
  amg_release(h, scratch);
  amg_release(h, total);
  return AMG_OK;
}

static amg_status build_members(amg_handle* h, Level& L, int nc) {
  cudaStream_t s = h->stream;
  int32_t *cnt, *fill, *scratch, *total;
  AMG_ALLOC(h, cnt, int32_t, nc);
  AMG_ALLOC(h, fill, int32_t, nc);
  AMG_ALLOC(h, scratch, int32_t, nc / SCAN_TILE + 2);
  AMG_ALLOC(h, total, int32_t, 1);
  AMG_ALLOC(h, L.mptr, int32_t, nc + 1);
  AMG_ALLOC(h, L.mem, int32_t, L.n);
  k_count<<<amg_blocks(L.n), AMG_BLOCK, 0, s>>>(L.n, L.agg, cnt);
  scan_exclusive(s, nc, cnt, L.mptr, scratch, total);
  AMG_CK(h, cudaMemcpyAsync(L.mptr + nc, total, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  k_place<<<amg_blocks(L.n), AMG_BLOCK, 0, s>>>(L.n, L.agg, L.mptr, fill, L.mem);
  k_sort_members<<<amg_blocks(nc), AMG_BLOCK, 0, s>>>(nc, L.mptr, L.mem);
  AMG_CK(h, cudaGetLastError());
  amg_release(h, cnt);
  amg_release(h, fill);
  amg_release(h, scratch);
  amg_release(h, total);
  return AMG_OK;
}

amg_status amg_build_members(amg_handle* h, int k) { return build_members(h, h->L[k], h->L[k + 1].n); }

// aggregation map entries in [0, nc)
__global__ void k_check_agg(int n, const int32_t* __restrict__ agg, int nc, int* flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && (agg[i] < 0 || agg[i] >= nc)) atomicOr(flags, ST_BADCOL);
}

// structure of level k as for a caller's matrix (row pointers, columns in
// range and ascending, diagonal stored and positive, finite values) and its
// aggregation map in range of the next level's nc rows (nc = 0: no map)
amg_status amg_check_level(amg_handle* h, int k, int nc) {
  Level& L = h->L[k];
  cudaStream_t s = h->stream;
  int32_t* diagpos;
  AMG_ALLOC(h, diagpos, int32_t, L.n);
  AMG_CK(h, cudaMemsetAsync(h->dev_flags, 0, sizeof(int), s));
  k_validate<<<amg_blocks(L.n), AMG_BLOCK, 0, s>>>(L.n, (int)L.nnz, L.rp, L.ci, L.v, diagpos, h->dev_flags);
  amg_status st = check_flags(h, "amg_load");
  amg_release(h, diagpos);
  if (st != AMG_OK || nc <= 0 || !L.agg) return st;
  k_check_agg<<<amg_blocks(L.n), AMG_BLOCK, 0, s>>>(L.n, L.agg, nc, h->dev_flags);
  return check_flags(h, "amg_load: aggregation map");
}

amg_status amg_level_diag(amg_handle* h, int k) {
  Level& L = h->L[k];
  k_l1<<<amg_blocks(L.n), AMG_BLOCK, 0, h->stream>>>(L.n, L.rp, L.ci, L.v, L.omega, L.l1, L.dinv, L.dinvf,
                                                      h->p.relax_type == 0 ? 1 : 0);
  AMG_CK(h, cudaGetLastError());
  return AMG_OK;
}

static amg_status setup_impl(amg_handle* h, const amg_csr* A) {
  cudaStream_t s = h->stream;
  const int n = A->n;
  const int64_t nnz = A->nnz;
  AMG_ALLOC(h, h->dev_flags, int, 1);
  AMG_ALLOC(h, h->zero_flag, int, 4);

  // level 0: deep copy of the caller's matrix, then validation
  Level& L0 = h->L[0];
  L0.n = n;
  L0.nnz = nnz;
  AMG_ALLOC(h, L0.rp, int32_t, n + 1);
  AMG_ALLOC(h, L0.ci, int32_t, nnz);
  AMG_ALLOC(h, L0.v, double, nnz);
  AMG_CK(h, cudaMemcpyAsync(L0.rp, A->row_ptr, sizeof(int32_t) * (size_t)(n + 1), cudaMemcpyDeviceToDevice, s));
  if (nnz) {
    AMG_CK(h, cudaMemcpyAsync(L0.ci, A->col_idx, sizeof(int32_t) * (size_t)nnz, cudaMemcpyDeviceToDevice, s));
    AMG_CK(h, cudaMemcpyAsync(L0.v, A->val, sizeof(double) * (size_t)nnz, cudaMemcpyDeviceToDevice, s));
  }
  int32_t ends[2] = {0, 0};
  AMG_CK(h, cudaMemcpyAsync(&ends[0], L0.rp, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  AMG_CK(h, cudaMemcpyAsync(&ends[1], L0.rp + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  AMG_CK(h, cudaStreamSynchronize(s));
  if (ends[0] != 0 || ends[1] != nnz)
    return amg_fail(h, AMG_ERR_INVALID_ARG, "row_ptr[0] must be 0 and row_ptr[n] must equal nnz");
  if (h->p.relax_type != 0 && h->p.relax_type != 4)
    return amg_fail(h, AMG_ERR_INVALID_ARG, "relax_type must be 4 (l1-Jacobi) or 0 (Jacobi)");
  if (h->p.prolong_scale != 0 && h->p.prolong_scale != 1)
    return amg_fail(h, AMG_ERR_INVALID_ARG, "prolong_scale must be 0 (unit) or 1 (w-normalised)");
  {
    int32_t* diagpos;
    AMG_ALLOC(h, diagpos, int32_t, n);
    k_validate<<<amg_blocks(n), AMG_BLOCK, 0, s>>>(n, (int)nnz, L0.rp, L0.ci, L0.v, diagpos, h->dev_flags);
    amg_status st = check_flags(h, "amg_setup");
    if (st != AMG_OK) return st;
    k_check_sym<<<amg_blocks(n), AMG_BLOCK, 0, s>>>(n, L0.rp, L0.ci, L0.v, h->dev_flags);
    st = check_flags(h, "amg_setup");
    if (st != AMG_OK) return st;
    amg_release(h, diagpos);
  }

  // coarsening loop (Alg. 3), s pairwise steps per level
  const int cs = h->p.coarse_size > 0 ? h->p.coarse_size : 40 * (int)std::lround(std::cbrt((double)n));
  const int ssteps = h->p.aggr_steps > 0 ? h->p.aggr_steps : 1;
  const int maxl = h->p.max_levels < AMG_MAXL ? h->p.max_levels : AMG_MAXL;
  h->nl = 1;
  PCsr cur{n, nnz, L0.rp, L0.ci, L0.v};
  bool cur_owned = false;  // cur's arrays belong to a level
  int32_t* comp;
  AMG_ALLOC(h, comp, int32_t, n);
  k_iota<<<amg_blocks(n), AMG_BLOCK, 0, s>>>(n, comp);
  int comp_n = n, group = 0;
  // row blocks of the decoupled aggregation
  const int np = std::max(1, std::min(h->p.num_parts, n));
  int32_t* bnd;
  {
    std::vector<int32_t> hb(np + 1);
    for (int q = 0; q <= np; ++q) hb[q] = (int32_t)(((int64_t)q * n) / np);
    AMG_ALLOC(h, bnd, int32_t, np + 1);
    // on the handle's stream, after the allocation's zero fill; hb must outlive the copy
    AMG_CK(h, cudaMemcpyAsync(bnd, hb.data(), sizeof(int32_t) * (np + 1), cudaMemcpyHostToDevice, s));
    AMG_CK(h, cudaStreamSynchronize(s));
  }
  while (cur.n > cs && h->nl < maxl) {
    int32_t *agg, *open_idx, *mate;
    AMG_ALLOC(h, agg, int32_t, cur.n);
    AMG_ALLOC(h, open_idx, int32_t, cur.n);
    AMG_ALLOC(h, mate, int32_t, cur.n);
    int nc = 0;
    auto tm0 = std::chrono::steady_clock::now();
    amg_status st = pairwise_step(h, cur, np, bnd, agg, open_idx, mate, &nc);
    if (st != AMG_OK) return st;
    auto tm1 = std::chrono::steady_clock::now();
    h->match_ms += std::chrono::duration<double, std::milli>(tm1 - tm0).count();
    if (nc == cur.n) {  // no edge matched
      amg_release(h, agg);
      amg_release(h, open_idx);
      amg_release(h, mate);
      break;
    }
    PCsr nxt;
    st = galerkin_step(h, cur, agg, open_idx, mate, nc, &nxt);
    if (st != AMG_OK) return st;
    AMG_CK(h, cudaStreamSynchronize(s));
    h->galerkin_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tm1).count();
    k_compose<<<amg_blocks(comp_n), AMG_BLOCK, 0, s>>>(comp_n, comp, agg);
    if (np > 1) k_update_bnd<<<1, 256, 0, s>>>(np, bnd, agg, cur.n, nc);
    amg_release(h, agg);
    amg_release(h, open_idx);
    amg_release(h, mate);
    if (cur_owned) {
      amg_release(h, cur.rp);
      amg_release(h, cur.ci);
      amg_release(h, cur.v);
    }
    cur = nxt;
    cur_owned = true;
    h->npair++;
    ++group;
    if (group == ssteps || cur.n <= cs) {
      Level& P = h->L[h->nl - 1];
      Level& C = h->L[h->nl];
      P.agg = comp;
      C.n = cur.n;
      C.nnz = cur.nnz;
      C.rp = cur.rp;
      C.ci = cur.ci;
      C.v = cur.v;
      cur_owned = false;
      h->nl++;
      AMG_ALLOC(h, comp, int32_t, cur.n);
      k_iota<<<amg_blocks(cur.n), AMG_BLOCK, 0, s>>>(cur.n, comp);
      comp_n = cur.n;
      group = 0;
    }
  }
  if (group > 0) {
    Level& P = h->L[h->nl - 1];
    Level& C = h->L[h->nl];
    P.agg = comp;
    C.n = cur.n;
    C.nnz = cur.nnz;
    C.rp = cur.rp;
    C.ci = cur.ci;
    C.v = cur.v;
    h->nl++;
  } else {
    amg_release(h, comp);
  }

  // w-normalised prolongators: level matrices by the general sparse product
  if (h->p.prolong_scale == 1 && h->nl > 1) {
    AMG_CK(h, cudaStreamSynchronize(s));
    auto t0 = std::chrono::steady_clock::now();
    amg_status st = amg_normalise_hierarchy(h);
    if (st != AMG_OK) return st;
    AMG_CK(h, cudaStreamSynchronize(s));
    h->spgemm_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }

  return amg_finish_setup(h);
}

// Everything a solve needs beyond the level matrices and aggregation maps:
// member lists, tile heights, l1 diagonals and D, low-precision copies, the
// fused-bottom plan, work vectors and graphs.  Shared by amg_setup and
// amg_load (checkpoint.cu).
amg_status amg_finish_setup(amg_handle* h) {
  cudaStream_t s = h->stream;
  // per-level smoother data, members lists and low-precision copies
  const bool lowp = h->p.precision != AMG_FP64 && h->nl > 1;
  for (int k = 0; k < h->nl; ++k) {
    Level& L = h->L[k];
    L.lowp = lowp && k < h->nl - 1;
    AMG_CK(h, cudaMemsetAsync(h->dev_flags, 0, sizeof(int), s));
    k_maxrow<<<amg_blocks(L.n), AMG_BLOCK, 0, s>>>(L.n, L.rp, h->dev_flags);
    int mr = 0;
    amg_status st0 = sync_read(h, h->dev_flags, &mr);
    if (st0 != AMG_OK) return st0;
    AMG_CK(h, cudaMemsetAsync(h->dev_flags, 0, sizeof(int), s));
    L.maxrow = mr;
    k_bandwidth<<<amg_blocks(L.n), AMG_BLOCK, 0, s>>>(L.n, L.rp, L.ci, h->dev_flags);
    int bwd = 0;
    st0 = sync_read(h, h->dev_flags, &bwd);
    if (st0 != AMG_OK) return st0;
    AMG_CK(h, cudaMemsetAsync(h->dev_flags, 0, sizeof(int), s));
    L.bw = bwd;
    const int vb = L.lowp ? ((h->p.precision == AMG_FP32_BF16FINE && k == 0) ? 2 : 4) : 8;
    L.Rd = amg_tile_rows(mr, 8);   // non-pipelined kernels (their tile buffer falls back to direct loads)
    L.R = amg_tile_rows(mr, vb);
    const bool big = L.n >= h->small_rows;
    // pipelined kernels: the tallest tile (power of two, 8 .. 256 / min_tpr
    // rows) whose tiles all fit a stage, from the largest number of entries of
    // any tile of that height (rows of average length share a tile with the
    // longest ones, so this beats sizing by the longest row)
    int tmax[6];  // tile_max for R = 256 >> i
    for (int i = 0; i < 6; ++i) {
      k_tile_max<<<amg_blocks((L.n + (256 >> i) - 1) / (256 >> i)), AMG_BLOCK, 0, s>>>(L.n, L.rp, 256 >> i, h->dev_flags);
      st0 = sync_read(h, h->dev_flags, &tmax[i]);
      if (st0 != AMG_OK) return st0;
      AMG_CK(h, cudaMemsetAsync(h->dev_flags, 0, sizeof(int), s));
    }
    const int rmax = PIPE_CONSUMERS / std::max(1, h->min_tpr);
    auto fit = [&](int cap) {  // tallest fitting tile height, 0: none
      for (int i = 0; i < 6; ++i)
        if ((256 >> i) <= rmax && tmax[i] <= cap) return 256 >> i;
      return 0;
    };
    const int cap8 = amg_pipe_tile_bytes(8) / 12;
    const int Rp = fit(amg_pipe_tile_bytes(vb) / (vb + 4));
    const int Rpd = fit(cap8);
    L.piped = h->use_pipe && Rpd > 0;
    L.pipe = h->use_pipe && big && Rp > 0;
    if (L.piped) L.Rd = Rpd;
    if (L.pipe) L.R = Rp;
    // FP64 values and rows too long for one thread per row in a normal stage:
    // a 4x stage takes 256-row tiles of up to 8192 entries (fewer FP64
    // instructions per row than several threads per row with a shuffle
    // reduction; FP64 issue limits these kernels on this part)
    // forms: 2 = 2x stages, 128 rows, 2 threads per row; 4 = 4x stages, 256
    // rows, one thread per row; 5 = two consumer groups, four 2x stages, 128
    // rows, one thread per row
    const int sbig = h->use_big;
    const int rbig = sbig == 4 ? 256 : 128;                          // rows per tile
    const int scale = sbig == 4 ? 4 : 2;                             // stage scale
    const int tpr_big = sbig == 2 ? 2 : 1;
    // (only on levels with at least one tile per multiprocessor: one block per
    // multiprocessor runs this form, and smaller levels want more, shorter tiles)
    const bool big_rows = (sbig == 2 || sbig == 4 || sbig == 5) && h->min_tpr <= tpr_big &&
                          tmax[rbig == 256 ? 0 : 1] <= cap8 * scale &&
                          (int64_t)(L.n + rbig - 1) / rbig >= (int64_t)amg_num_sms();
    if (L.pipe && vb == 8 && L.R < rbig && big_rows) {
      L.R = rbig;
      L.sb = sbig;
    }
    if (L.piped && L.Rd < rbig && big_rows) {
      L.Rd = rbig;
      L.sbd = sbig;
    }
    // two consumer groups with half the threads per row (tiles of 32-128 rows):
    // use_ng 1 on every kernel of the level (27-point 128^3 FP64 solve 29.6 ->
    // 28.1 ms, level-1 sweep 29.5 -> 24.4 us; 7-point log-normal 256^3 FP32
    // 46.9 -> 46.3 ms; levels of 256-row tiles unchanged), 2 on the FP64 outer
    // kernels only
    if (h->use_ng == 1 && L.pipe && L.sb == 1 && L.R >= 32 && L.R <= 128) L.sb = 6;
    if (h->use_ng >= 1 && L.piped && L.sbd == 1 && L.Rd >= 32 && L.Rd <= 128) L.sbd = 6;
    // pattern-coded columns (pattern.cu), read by the pipelined forms that have
    // a pattern variant: standard stages with tiles of 64-256 rows, two groups
    if (L.pipe || L.piped) {
      amg_status sp = amg_build_patterns(h, k);
      if (sp != AMG_OK) return sp;
    }
    // pattern-coded float levels with tiles of 32-128 rows take two consumer
    // groups with use_ng 2 as well (27-point 128^3 FP32 level-0 sweep 75.4 ->
    // 56.4 us, solve 17.3 -> 16.0 ms)
    if (h->use_ng >= 1 && L.pid && vb < 8 && L.pipe && L.sb == 1 && L.R >= 32 && L.R <= 128) L.sb = 6;
    // FP64 forms with several threads per row (27-point levels) keep CSR
    // columns: FP64-issue bound, their kernels gain nothing from fewer bytes
    // (27-point 128^3 sweep 166 vs 163 us) and the V-cycle measured slower
    // (1.94 vs 1.74 ms)
    auto pat_form = [&](int R, int sb, int value_bytes) {  // 2: one thread per row; 1: the other pattern forms
      if ((sb == 1 && R == 256) || (sb == 6 && R == 128)) return h->use_pat >= 2 ? 2 : 1;
      if (value_bytes == 8) return 0;
      return ((sb == 1 && R >= 64) || sb == 6) ? 1 : 0;
    };
    L.stage_rows = h->use_stage != 0;
    L.pat = L.pid && L.pipe ? pat_form(L.R, L.sb, vb) : 0;
    L.patd = L.pid && L.piped ? pat_form(L.Rd, L.sbd, 8) : 0;
    AMG_ALLOC(h, L.l1, double, L.n);
    AMG_ALLOC(h, L.dinv, double, L.n);
    if (L.lowp) {
      AMG_ALLOC(h, L.dinvf, float, L.n);
      bool bfine = (h->p.precision == AMG_FP32_BF16FINE && k == 0);
      if (bfine) AMG_ALLOC(h, L.vb, bf16, L.nnz);
      else AMG_ALLOC(h, L.vf, float, L.nnz);
      if (L.nnz)
        k_round_vals<<<amg_blocks(L.nnz), AMG_BLOCK, 0, s>>>(L.nnz, L.v, bfine ? nullptr : L.vf, bfine ? L.vb : nullptr);
      if (L.pw) {  // prolongator values of a float level
        AMG_ALLOC(h, L.pwf, float, L.n);
        AMG_ALLOC(h, L.pwmf, float, L.n);
        k_round_vals<<<amg_blocks(L.n), AMG_BLOCK, 0, s>>>(L.n, L.pw, L.pwf, nullptr);
        k_round_vals<<<amg_blocks(L.n), AMG_BLOCK, 0, s>>>(L.n, L.pwm, L.pwmf, nullptr);
      }
    }
    amg_status st = amg_level_diag(h, k);
    if (st != AMG_OK) return st;
    if (k < h->nl - 1 && !L.mptr) {
      st = build_members(h, L, h->L[k + 1].n);
      if (st != AMG_OK) return st;
    }
  }
  h->kb = h->nl;
  if (h->p.cycle != 0 && h->p.cycle != 2)
    return amg_fail(h, AMG_ERR_INVALID_ARG, "cycle must be 0 (V) or 2 (W)");
  AMG_CK(h, cudaStreamSynchronize(s));
  AMG_CK(h, cudaGetLastError());
  // the small levels in one cluster launch (unit prolongators only)
  if (h->use_bottom && h->p.cycle == 0 && h->p.prolong_scale == 0) {
    amg_status st = amg_plan_bottom(h);
    if (st != AMG_OK) return st;
  }
  return amg_prepare_solve(h);
}

void amg_read_hooks(amg_handle* h) {
  // test and tuning hooks (environment): AMG_PIPE=0 non-pipelined row kernels,
  // AMG_BOTTOM=0/1/2 bottom levels as separate
  // launches / in one cluster launch / by the owner-spread rule (default),
  // AMG_FUSE=0 restriction and prolongation as separate kernels,
  // AMG_BIG=0 no 4x stages for FP64 long-row levels,
  // AMG_PAIR=0/1/2 paired row passes never / where they pay / always,
  // AMG_PAIR_SLACK lag of the paired passes beyond the halo (tiles),
  // AMG_SMALL_ROWS, AMG_MIN_TPR row-kernel forms,
  // AMG_PAT=0/1 CSR columns on every level / pattern-coded columns located
  // by row pointers only (AMG_PAT=2: rows located from the tuple lengths
  // where one thread takes a row), AMG_STAGE=0 row data of the small-stage
  // pattern kernels loaded by the consumers instead of staged,
  // AMG_SUITOR_CAP step cap of the matching loop,
  // AMG_FAIL_ALLOC_AFTER make the k-th device allocation of the handle fail
  if (const char* e = getenv("AMG_SUITOR_CAP")) h->suitor_cap = atoll(e);
  if (const char* e = getenv("AMG_BOTTOM")) h->use_bottom = atoi(e);
  if (const char* e = getenv("AMG_SMALL_ROWS")) h->small_rows = atoi(e);
  if (const char* e = getenv("AMG_MIN_TPR")) h->min_tpr = atoi(e);
  if (const char* e = getenv("AMG_FUSE")) h->fuse = atoi(e);
  if (const char* e = getenv("AMG_PAIR")) h->use_pair = atoi(e);
  if (const char* e = getenv("AMG_BIG")) h->use_big = atoi(e);
  if (const char* e = getenv("AMG_PAIR_SLACK")) h->pair_slack = atoi(e);
  if (const char* e = getenv("AMG_FAIL_ALLOC_AFTER")) h->fail_alloc_after = atoi(e);
  if (const char* e = getenv("AMG_PIPE")) h->use_pipe = atoi(e);
  if (const char* e = getenv("AMG_NG")) h->use_ng = atoi(e);
  if (const char* e = getenv("AMG_PAT")) h->use_pat = atoi(e);
  if (const char* e = getenv("AMG_STAGE")) h->use_stage = atoi(e);
}

extern "C" amg_status amg_setup(const amg_csr* A, const amg_params* p, void* stream, amg_handle** out) {
  if (!out) return AMG_ERR_INVALID_ARG;
  *out = nullptr;
  if (!A || A->n <= 0 || A->nnz < A->n || !A->row_ptr || !A->col_idx || !A->val)
    return AMG_ERR_INVALID_ARG;
  auto t0 = std::chrono::steady_clock::now();
  amg_handle* h = new amg_handle();
  if (p) h->p = *p;
  else amg_params_default(&h->p);
  h->stream = (cudaStream_t)stream;
  amg_read_hooks(h);
  amg_status st = setup_impl(h, A);
  if (st != AMG_OK) {
    amg_set_setup_error(h->err);
    cudaStreamSynchronize(h->stream);
    amg_destroy(h);
    return st;
  }
  auto t1 = std::chrono::steady_clock::now();
  h->setup_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
  *out = h;
  return AMG_OK;
}
