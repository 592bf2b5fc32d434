// General sparse matrix product C = A B (CSR x CSR) and the w-normalised
// prolongators built with it.
//
// Sec. 3.1 gives the prolongator entries from the smooth vector w
// (P_{i,I} = w_i / |w restricted to aggregate I|, w^{k+1} = P^T w^k) and forms
// every coarse matrix as the Galerkin product P^T A P; Sec. 4.2 / Alg. 4 compute
// that product with a general sparse product in two phases (a symbolic phase
// that sizes every row of C, then a numeric phase that fills it).  The unit
// prolongator of the default hierarchy has a cheaper exact form (sums of
// entries, setup.cu); this file is the general product, used for the
// w-normalised form: A^{k+1} = R (A^k P) with R = P^T.
//
// Kernel: one warp per row of A.  Lane t owns the entries p = rp_a[i] + t,
// + t + 32, ... of the row and keeps for each a cursor into row ci_a[p] of B
// (global scratch, one int per entry of A).  B's rows are sorted, so the next
// column of row i of C is the warp minimum of the columns under the cursors;
// its value is the sum of a_p b_q over the entries whose cursor sits on that
// column, each lane summing its entries in ascending p, then a butterfly sum
// over the 32 lanes.  The order is fixed by the data alone, so the product is
// bitwise reproducible.  Each round advances at least one cursor: a row takes
// at most (products of the row) rounds.  Columns of C come out ascending.
#include <climits>

#include "amg_internal.cuh"

#define SPGEMM_BLOCK 256

template <bool NUMERIC>
__global__ void __launch_bounds__(SPGEMM_BLOCK)
    k_spgemm(int m, const int32_t* __restrict__ arp, const int32_t* __restrict__ aci, const double* __restrict__ av,
             const int32_t* __restrict__ brp, const int32_t* __restrict__ bci, const double* __restrict__ bv,
             int32_t* __restrict__ cur, int32_t* __restrict__ cnt_or_crp, int32_t* __restrict__ cci,
             double* __restrict__ cv) {
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (SPGEMM_BLOCK / 32);
  for (int i = (int)((blockIdx.x * SPGEMM_BLOCK + threadIdx.x) >> 5); i < m; i += warps) {
    const int p0 = arp[i], p1 = arp[i + 1];
    for (int p = p0 + lane; p < p1; p += 32) cur[p] = brp[aci[p]];
    int out = NUMERIC ? cnt_or_crp[i] : 0;
    for (;;) {
      int c = INT_MAX;
      for (int p = p0 + lane; p < p1; p += 32) {
        const int q = cur[p];
        if (q < brp[aci[p] + 1]) c = min(c, bci[q]);
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) c = min(c, __shfl_xor_sync(0xffffffffu, c, off));
      if (c == INT_MAX) break;
      double s = 0.0;
      for (int p = p0 + lane; p < p1; p += 32) {
        const int q = cur[p];
        if (q < brp[aci[p] + 1] && bci[q] == c) {
          if (NUMERIC) s = __fma_rn(av[p], bv[q], s);
          cur[p] = q + 1;
        }
      }
      if (NUMERIC) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) {
          cci[out] = c;
          cv[out] = s;
        }
      }
      ++out;
    }
    if (!NUMERIC && lane == 0) cnt_or_crp[i] = out;
  }
}

// shared with setup.cu's scan (defined there)
void amg_scan_exclusive(cudaStream_t s, int n, const int32_t* in, int32_t* out, int32_t* scratch, int32_t* total);
int amg_scan_scratch_ints(int n);

static int spgemm_grid(int m) {
  const int warps_per_block = SPGEMM_BLOCK / 32;
  const int want = (m + warps_per_block - 1) / warps_per_block;
  const int cap = amg_num_sms() * 8;
  return want < 1 ? 1 : (want < cap ? want : cap);
}

// C = A B into device buffers allocated from the handle (sorted columns).
// A: m rows; B: rows indexed by A's columns.  The caller checks sizes.
static amg_status spgemm_handle(amg_handle* h, int m, const int32_t* arp, const int32_t* aci, const double* av,
                                int64_t annz, const int32_t* brp, const int32_t* bci, const double* bv,
                                int32_t** crp_out, int32_t** cci_out, double** cv_out, int64_t* cnnz_out) {
  cudaStream_t s = h->stream;
  int32_t *cur, *cnt, *crp, *scratch, *total;
  AMG_ALLOC(h, cur, int32_t, annz > 0 ? annz : 1);
  AMG_ALLOC(h, cnt, int32_t, m);
  AMG_ALLOC(h, crp, int32_t, m + 1);
  AMG_ALLOC(h, scratch, int32_t, amg_scan_scratch_ints(m));
  AMG_ALLOC(h, total, int32_t, 1);
  const int grid = spgemm_grid(m);
  k_spgemm<false><<<grid, SPGEMM_BLOCK, 0, s>>>(m, arp, aci, av, brp, bci, bv, cur, cnt, nullptr, nullptr);
  amg_scan_exclusive(s, m, cnt, crp, scratch, total);
  AMG_CK(h, cudaMemcpyAsync(crp + m, total, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  int32_t nnz = 0;
  AMG_CK(h, cudaMemcpyAsync(&nnz, total, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  AMG_CK(h, cudaStreamSynchronize(s));
  int32_t* cci;
  double* cv;
  AMG_ALLOC(h, cci, int32_t, nnz > 0 ? nnz : 1);
  AMG_ALLOC(h, cv, double, nnz > 0 ? nnz : 1);
  k_spgemm<true><<<grid, SPGEMM_BLOCK, 0, s>>>(m, arp, aci, av, brp, bci, bv, cur, crp, cci, cv);
  AMG_CK(h, cudaGetLastError());
  amg_release(h, cur);
  amg_release(h, cnt);
  amg_release(h, scratch);
  amg_release(h, total);
  *crp_out = crp;
  *cci_out = cci;
  *cv_out = cv;
  *cnnz_out = nnz;
  return AMG_OK;
}

// ---------------------------------------------------------------------------
// w-normalised prolongators

// w^{k+1}_I = sqrt(sum over the members i of I, ascending, of w_i^2), each
// operation rounded on its own
__global__ void k_next_smooth(int nc, const int32_t* __restrict__ mptr, const int32_t* __restrict__ mem,
                              const double* __restrict__ w, double* __restrict__ wc) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  double s = 0.0;
  for (int m = mptr[I]; m < mptr[I + 1]; ++m) {
    const double wi = w[mem[m]];
    s = __dadd_rn(s, __dmul_rn(wi, wi));
  }
  wc[I] = __dsqrt_rn(s);
}

// P values: pw[i] = w_i / w^{k+1}_{agg(i)}; pwm[m] = pw[mem[m]] (member order);
// prp = 0, 1, ..., n (one entry per row of P)
__global__ void k_prolong_values(int n, const int32_t* __restrict__ agg, const double* __restrict__ w,
                                 const double* __restrict__ wc, double* __restrict__ pw, int32_t* __restrict__ prp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  prp[i] = i;
  if (i < n) pw[i] = __ddiv_rn(w[i], wc[agg[i]]);
}

__global__ void k_member_values(int n, const int32_t* __restrict__ mem, const double* __restrict__ pw,
                                double* __restrict__ pwm) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < n) pwm[m] = pw[mem[m]];
}

__global__ void k_fill(int n, double* __restrict__ a, double v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

// raises ST_BADCOL in flags where two CSR patterns differ
__global__ void k_same_pattern(int n, const int32_t* __restrict__ rp0, const int32_t* __restrict__ ci0,
                               const int32_t* __restrict__ rp1, const int32_t* __restrict__ ci1, int* flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  if (rp0[i] != rp1[i]) {
    atomicOr(flags, ST_BADCOL);
    return;
  }
  if (i == n) return;
  for (int p = rp0[i]; p < rp0[i + 1]; ++p)
    if (ci0[p] != ci1[p]) atomicOr(flags, ST_BADCOL);
}

// Level matrices of the w-normalised prolongators, from level 0 (w = 1, the
// input matrix) down: w^{k+1} = P_k^T w^k, T = A^k P_k, A^{k+1} = R_k T with
// R_k = P_k^T (the member lists with the P values).  The aggregates are those
// of the unit construction (the matching weights do not change under the
// diagonal scaling that relates the two forms), so the sparsity patterns are
// the unit ones; the values of every coarse level are replaced by the
// normalised ones.
amg_status amg_normalise_hierarchy(amg_handle* h) {
  cudaStream_t s = h->stream;
  Level& L0 = h->L[0];
  AMG_ALLOC(h, L0.wsv, double, L0.n);
  k_fill<<<amg_blocks(L0.n), AMG_BLOCK, 0, s>>>(L0.n, L0.wsv, 1.0);
  for (int k = 0; k + 1 < h->nl; ++k) {
    Level& F = h->L[k];
    Level& C = h->L[k + 1];
    if (!F.mptr) {
      amg_status st = amg_build_members(h, k);
      if (st != AMG_OK) return st;
    }
    AMG_ALLOC(h, C.wsv, double, C.n);
    AMG_ALLOC(h, F.pw, double, F.n);
    AMG_ALLOC(h, F.pwm, double, F.n);
    int32_t* prp;
    AMG_ALLOC(h, prp, int32_t, F.n + 1);
    k_next_smooth<<<amg_blocks(C.n), AMG_BLOCK, 0, s>>>(C.n, F.mptr, F.mem, F.wsv, C.wsv);
    k_prolong_values<<<amg_blocks(F.n + 1), AMG_BLOCK, 0, s>>>(F.n, F.agg, F.wsv, C.wsv, F.pw, prp);
    k_member_values<<<amg_blocks(F.n), AMG_BLOCK, 0, s>>>(F.n, F.mem, F.pw, F.pwm);
    // T = A^k P (n_k x n_{k+1}), then A^{k+1} = R T with R = P^T (rows: member lists)
    int32_t *trp, *tci, *crp, *cci;
    double *tv, *cv;
    int64_t tnnz = 0, cnnz = 0;
    amg_status st = spgemm_handle(h, F.n, F.rp, F.ci, F.v, F.nnz, prp, F.agg, F.pw, &trp, &tci, &tv, &tnnz);
    if (st != AMG_OK) return st;
    st = spgemm_handle(h, C.n, F.mptr, F.mem, F.pwm, F.n, trp, tci, tv, &crp, &cci, &cv, &cnnz);
    if (st != AMG_OK) return st;
    if (cnnz != C.nnz) return amg_fail(h, AMG_ERR_CUDA, "normalised level %d: %lld entries, unit pattern has %lld",
                                       k + 1, (long long)cnnz, (long long)C.nnz);
    AMG_CK(h, cudaMemsetAsync(h->dev_flags, 0, sizeof(int), s));
    k_same_pattern<<<amg_blocks(C.n + 1), AMG_BLOCK, 0, s>>>(C.n, C.rp, C.ci, crp, cci, h->dev_flags);
    int f = 0;
    AMG_CK(h, cudaMemcpyAsync(&f, h->dev_flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CK(h, cudaStreamSynchronize(s));
    if (f) return amg_fail(h, AMG_ERR_CUDA, "normalised level %d: pattern differs from the unit Galerkin product", k + 1);
    // the level keeps its (equal) pattern and takes the normalised values
    amg_release(h, C.v);
    C.v = cv;
    for (void* p : {(void*)prp, (void*)trp, (void*)tci, (void*)tv, (void*)crp, (void*)cci}) amg_release(h, p);
  }
  return AMG_OK;
}

amg_status amg_member_values(amg_handle* h, int k) {
  Level& F = h->L[k];
  if (!F.pwm) AMG_ALLOC(h, F.pwm, double, F.n);
  k_member_values<<<amg_blocks(F.n), AMG_BLOCK, 0, h->stream>>>(F.n, F.mem, F.pw, F.pwm);
  AMG_CK(h, cudaGetLastError());
  return AMG_OK;
}

// ---------------------------------------------------------------------------
// public general product (two calls: row pointers and the count, then the
// columns and values)

__global__ void k_check_csr(int m, int ncols, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                            int strict, int* flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int p0 = rp[i], p1 = rp[i + 1];
  if (p1 < p0) {
    atomicOr(flags, ST_BADPTR);
    return;
  }
  for (int p = p0; p < p1; ++p) {
    const int c = ci[p];
    if (c < 0 || c >= ncols || (strict && p > p0 && c <= ci[p - 1])) atomicOr(flags, ST_BADCOL);
  }
}

extern "C" amg_status amg_spgemm(int32_t m, int32_t k, int32_t n, const int32_t* a_row_ptr, const int32_t* a_col_idx,
                                 const double* a_val, const int32_t* b_row_ptr, const int32_t* b_col_idx,
                                 const double* b_val, int32_t* c_row_ptr, int32_t* c_col_idx, double* c_val,
                                 int64_t* nnz_c, void* stream) {
  if (m < 0 || k < 0 || n < 0 || !a_row_ptr || !b_row_ptr || !c_row_ptr || !nnz_c) {
    amg_set_setup_error("amg_spgemm: negative size or NULL pointer");
    return AMG_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool numeric = c_col_idx != nullptr;
  if (numeric && !c_val) {
    amg_set_setup_error("amg_spgemm: c_col_idx given without c_val");
    return AMG_ERR_INVALID_ARG;
  }
  if (m == 0) {
    *nnz_c = 0;
    if (!numeric && cudaMemsetAsync(c_row_ptr, 0, sizeof(int32_t), s) != cudaSuccess) return AMG_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? AMG_OK : AMG_ERR_CUDA;
  }
  int32_t ends[4] = {0, 0, 0, 0};
  if (cudaMemcpyAsync(&ends[0], a_row_ptr + m, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&ends[1], b_row_ptr + k, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    amg_set_setup_error("amg_spgemm: reading the row pointers failed");
    return AMG_ERR_CUDA;
  }
  const int32_t annz = ends[0], bnnz = ends[1];
  if (annz < 0 || bnnz < 0 || (annz > 0 && (!a_col_idx || !a_val)) || (bnnz > 0 && (!b_col_idx || !b_val))) {
    amg_set_setup_error("amg_spgemm: bad row pointers or NULL column/value arrays");
    return AMG_ERR_INVALID_ARG;
  }
  // scratch: structure flags, cursors (one per entry of A), counts and scan space
  const int tiles = amg_scan_scratch_ints(m);
  const size_t bytes = sizeof(int32_t) * (4 + (size_t)(annz > 0 ? annz : 1) + (size_t)m + (size_t)tiles + 2);
  int32_t* scr = nullptr;
  if (cudaMallocAsync((void**)&scr, bytes, s) != cudaSuccess) {
    amg_set_setup_error("amg_spgemm: scratch allocation failed");
    return AMG_ERR_OOM;
  }
  int* flags = scr;
  int32_t* cur = scr + 4;
  int32_t* cnt = cur + (annz > 0 ? annz : 1);
  int32_t* scan = cnt + m;
  int32_t* total = scan + tiles;
  amg_status st = AMG_OK;
  int f = 0;
  int32_t nnz = 0;
  cudaMemsetAsync(flags, 0, sizeof(int), s);
  if (!numeric) {
    k_check_csr<<<amg_blocks(m), AMG_BLOCK, 0, s>>>(m, k, a_row_ptr, a_col_idx, 0, flags);
    if (k > 0) k_check_csr<<<amg_blocks(k), AMG_BLOCK, 0, s>>>(k, n, b_row_ptr, b_col_idx, 1, flags);
    cudaMemcpyAsync(&f, flags, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) st = AMG_ERR_CUDA;
    else if (f) {
      amg_set_setup_error("amg_spgemm: row pointers not monotone, a column out of range, or a row of B "
                          "not strictly ascending");
      st = AMG_ERR_INVALID_ARG;
    }
  }
  if (st == AMG_OK) {
    const int grid = spgemm_grid(m);
    if (!numeric) {
      k_spgemm<false><<<grid, SPGEMM_BLOCK, 0, s>>>(m, a_row_ptr, a_col_idx, a_val, b_row_ptr, b_col_idx, b_val, cur,
                                                     cnt, nullptr, nullptr);
      amg_scan_exclusive(s, m, cnt, c_row_ptr, scan, total);
      cudaMemcpyAsync(c_row_ptr + m, total, sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(&nnz, total, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    } else {
      k_spgemm<true><<<grid, SPGEMM_BLOCK, 0, s>>>(m, a_row_ptr, a_col_idx, a_val, b_row_ptr, b_col_idx, b_val, cur,
                                                    c_row_ptr, c_col_idx, c_val);
      cudaMemcpyAsync(&nnz, c_row_ptr + m, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    }
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
      amg_set_setup_error("amg_spgemm: kernel launch failed");
      st = AMG_ERR_CUDA;
    }
  }
  cudaFreeAsync(scr, s);
  if (cudaStreamSynchronize(s) != cudaSuccess && st == AMG_OK) st = AMG_ERR_CUDA;
  if (st == AMG_OK) *nnz_c = nnz;
  return st;
}
