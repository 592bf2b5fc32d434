// Pattern-coded column indices of a level matrix (setup side).
//
// The solve phase is bound by HBM traffic, and on a stencil level the 4-byte
// column index is a quarter of the bytes a row pass moves per entry.  Most rows
// of such a level share one tuple of column offsets (j - i for its entries in
// CSR order): interior rows of a 7-point Poisson matrix all have
// (-N^2, -N, -1, 0, 1, N, N^2), and the boundary rows fall into a few more
// tuples.  Where a level has at most 255 distinct tuples and their table (rows
// x (longest row + 1), with the lengths) has at most PAT_TAB_MAX entries, each row gets a
// one-byte id into a table of tuples and the pipelined row kernels read that
// byte instead of the row's column indices (rows.cuh).  The matrix values, the
// order of the entries and every multiply-add stay as they are, so results are
// bitwise those of the CSR form; only the bytes streamed per row change
// (8 or 4 or 2 per entry plus 1 per row, instead of 12, 8 or 6 per entry).
//
// Construction: every row hashes its tuple; the distinct hashes go into an
// open-addressing table (one insert per distinct hash per warp; the insert
// gives up once more than 255 tuples are seen, so irregular levels cost one
// pass); the table rows are ordered by hash on the host, so ids do not depend
// on the order the inserts landed in; each table row is copied from a row that
// inserted its hash; a second pass assigns every row its id and compares its
// tuple entry by entry with the table row.  Any difference (a hash
// collision) or overflow leaves the level on CSR columns.
#include <algorithm>

#include "amg_internal.cuh"

#define PAT_SLOTS 2048   // hash-table slots (a power of two)
#define PAT_MAX 255      // table rows (ids are one byte)
#define PAT_MAXK 32      // longest row a table row holds
#define PAT_MIN_ROWS 32768

enum { PAT_FULL = 1, PAT_MISMATCH = 2 };

__device__ __forceinline__ uint64_t pat_mix(uint64_t z) {  // SplitMix64 finaliser (Steele, Lea and Flood, 2014)
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// hash of row i's length and column offsets, never 0 (0 marks an empty slot)
__device__ __forceinline__ uint64_t pat_key(int i, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci) {
  const int p0 = rp[i], p1 = rp[i + 1];
  uint64_t h = pat_mix(0x9E3779B97F4A7C15ull + (uint64_t)(p1 - p0));
  for (int p = p0; p < p1; ++p) h = pat_mix(h ^ (uint64_t)(uint32_t)(ci[p] - i));
  return h | 1ull;
}

__device__ __forceinline__ unsigned pat_home(uint64_t key) { return (unsigned)(key >> 32) & (PAT_SLOTS - 1); }

// one insert per distinct key of a warp; linear probing, at most PAT_SLOTS steps
__global__ void k_pat_insert(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                             unsigned long long* keys, int* reps, int* count, int* flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < n && *(volatile int*)flags == 0;
  const uint64_t key = valid ? pat_key(i, rp, ci) : 0ull;
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  if (!valid || (int)(threadIdx.x & 31) != __ffs(peers) - 1) return;
  unsigned s = pat_home(key);
  for (int probe = 0; probe < PAT_SLOTS; ++probe, s = (s + 1) & (PAT_SLOTS - 1)) {
    if (*(volatile int*)flags) return;  // another warp has seen too many tuples
    unsigned long long k = *(volatile unsigned long long*)&keys[s];
    if (k == key) return;
    if (k == 0ull) {
      k = atomicCAS(&keys[s], 0ull, (unsigned long long)key);
      if (k == 0ull) {
        reps[s] = i;
        if (atomicAdd(count, 1) >= PAT_MAX) atomicOr(flags, PAT_FULL);
        return;
      }
      if (k == key) return;
    }
  }
  atomicOr(flags, PAT_FULL);
}

// row_ptr at rows 0, 32, 64, ... and nnz (the row kernels that give one thread
// to each row locate a warp's 32 rows from here and the tuple lengths)
__global__ void k_pat_chunk_base(int n, const int32_t* __restrict__ rp, int32_t* __restrict__ pcb) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int nc = (n + 31) / 32;
  if (c <= nc) pcb[c] = rp[min(32 * c, n)];
}

// table row id from its representative row (one warp per table row)
__global__ void k_pat_table(int npat, const int* __restrict__ reps, const int32_t* __restrict__ rp,
                            const int32_t* __restrict__ ci, int pk, int32_t* __restrict__ ptab, int* __restrict__ plen) {
  const int id = blockIdx.x;
  if (id >= npat) return;
  const int i = reps[id], p0 = rp[i], len = rp[i + 1] - p0;
  for (int j = threadIdx.x; j < pk; j += blockDim.x) ptab[(size_t)id * pk + j] = j < len ? ci[p0 + j] - i : 0;
  if (threadIdx.x == 0) plen[id] = len;
}

// every row: its id, and its tuple compared entry by entry with the table row
__global__ void k_pat_assign(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                             const unsigned long long* __restrict__ keys, const int* __restrict__ ids,
                             const int32_t* __restrict__ ptab, const int* __restrict__ plen, int pk,
                             uint8_t* __restrict__ pid, int* flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t key = pat_key(i, rp, ci);
  unsigned s = pat_home(key);
  int probe = 0;
  for (; probe < PAT_SLOTS && keys[s] != key && keys[s] != 0ull; ++probe) s = (s + 1) & (PAT_SLOTS - 1);
  const int id = probe < PAT_SLOTS && keys[s] == key ? ids[s] : -1;
  bool same = id >= 0;
  if (same) {
    const int p0 = rp[i], len = rp[i + 1] - p0;
    same = len == plen[id];
    for (int j = 0; same && j < len; ++j) same = ci[p0 + j] - i == ptab[(size_t)id * pk + j];
  }
  if (!same) {
    atomicOr(flags, PAT_MISMATCH);
    return;
  }
  pid[i] = (uint8_t)id;
}

amg_status amg_build_patterns(amg_handle* h, int k) {
  Level& L = h->L[k];
  if (!h->use_pat || L.pid || L.n < PAT_MIN_ROWS || L.maxrow < 1 || L.maxrow > PAT_MAXK) return AMG_OK;
  cudaStream_t s = h->stream;
  unsigned long long* keys = nullptr;
  int *reps = nullptr, *ids = nullptr, *cnt = nullptr;
  AMG_ALLOC(h, keys, unsigned long long, PAT_SLOTS);
  AMG_ALLOC(h, reps, int, PAT_SLOTS);
  AMG_ALLOC(h, ids, int, PAT_SLOTS);
  AMG_ALLOC(h, cnt, int, 2);  // count, flags
  auto release = [&]() {
    amg_release(h, keys);
    amg_release(h, reps);
    amg_release(h, ids);
    amg_release(h, cnt);
  };
  k_pat_insert<<<amg_blocks(L.n), AMG_BLOCK, 0, s>>>(L.n, L.rp, L.ci, keys, reps, cnt, cnt + 1);
  int hc[2] = {0, 0};
  AMG_CK(h, cudaMemcpyAsync(hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, s));
  AMG_CK(h, cudaStreamSynchronize(s));
  AMG_CK(h, cudaGetLastError());
  const int npat = hc[0];
  if (hc[1] || npat < 1 || npat > PAT_MAX || npat * (L.maxrow + 1) > PAT_TAB_MAX) {
    release();
    return AMG_OK;  // too many tuples: CSR columns
  }
  std::vector<unsigned long long> hk(PAT_SLOTS);
  std::vector<int> hr(PAT_SLOTS);
  AMG_CK(h, cudaMemcpyAsync(hk.data(), keys, sizeof(unsigned long long) * PAT_SLOTS, cudaMemcpyDeviceToHost, s));
  AMG_CK(h, cudaMemcpyAsync(hr.data(), reps, sizeof(int) * PAT_SLOTS, cudaMemcpyDeviceToHost, s));
  AMG_CK(h, cudaStreamSynchronize(s));
  std::vector<int> order;  // occupied slots by key
  for (int j = 0; j < PAT_SLOTS; ++j)
    if (hk[j]) order.push_back(j);
  std::sort(order.begin(), order.end(), [&](int a, int b) { return hk[a] < hk[b]; });
  std::vector<int> hid(PAT_SLOTS, -1), hrep(order.size());
  for (size_t r = 0; r < order.size(); ++r) {
    hid[order[r]] = (int)r;
    hrep[r] = hr[order[r]];
  }
  const int pk = L.maxrow;
  int32_t* ptab = nullptr;
  int* plen = nullptr;
  uint8_t* pid = nullptr;
  AMG_ALLOC(h, ptab, int32_t, (size_t)npat * pk);
  AMG_ALLOC(h, plen, int, npat);
  AMG_ALLOC(h, pid, uint8_t, L.n);
  // reps reused for the ordered representatives; the host vectors live until the synchronisation below
  AMG_CK(h, cudaMemcpyAsync(ids, hid.data(), sizeof(int) * PAT_SLOTS, cudaMemcpyHostToDevice, s));
  AMG_CK(h, cudaMemcpyAsync(reps, hrep.data(), sizeof(int) * hrep.size(), cudaMemcpyHostToDevice, s));
  k_pat_table<<<npat, 32, 0, s>>>(npat, reps, L.rp, L.ci, pk, ptab, plen);
  k_pat_assign<<<amg_blocks(L.n), AMG_BLOCK, 0, s>>>(L.n, L.rp, L.ci, keys, ids, ptab, plen, pk, pid, cnt + 1);
  AMG_CK(h, cudaMemcpyAsync(hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, s));
  AMG_CK(h, cudaStreamSynchronize(s));
  AMG_CK(h, cudaGetLastError());
  release();
  if (hc[1]) {  // a hash collision: keep CSR columns
    amg_release(h, plen);
    amg_release(h, ptab);
    amg_release(h, pid);
    return AMG_OK;
  }
  int32_t* pcb = nullptr;
  const int nc = (L.n + 31) / 32;
  AMG_ALLOC(h, pcb, int32_t, nc + 1);
  k_pat_chunk_base<<<amg_blocks(nc + 1), AMG_BLOCK, 0, s>>>(L.n, L.rp, pcb);
  AMG_CK(h, cudaGetLastError());
  L.pid = pid;
  L.ptab = ptab;
  L.plen = plen;
  L.pcb = pcb;
  L.npat = npat;
  L.pk = pk;
  return AMG_OK;
}
