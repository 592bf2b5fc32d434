// Saving a built hierarchy to a file and loading it back.
//
// The paper amortises one setup over many solves (Sec. 5.2 reports setup and
// solve separately; its library keeps the hierarchy between solves).  A file
// lets the hierarchy outlive the process: amg_load rebuilds a handle from it
// without the matching and the Galerkin products.
//
// The file holds what the setup decides (level matrices, aggregation maps,
// the damping of every level, and for the w-normalised prolongator its smooth
// vector and values); everything derived from those (member lists, l1
// diagonals, D, low-precision copies, kernel forms, work vectors, graphs) is
// recomputed on load by the same code as in amg_setup, so a loaded handle
// computes bit for bit what the saved one did.
//
// Layout (little-endian as the host writes it):
//   "AMGHIER1"; uint32 version (1); uint32 q = number of int32 fields of
//   amg_params; int32 params[q]; int32 num_levels; int32 num_pairwise;
//   per level k: int32 n; int64 nnz; int32 row_ptr[n+1]; int32 col_idx[nnz];
//     float64 val[nnz]; int32 has_omega; [float64 omega[n]];
//     k < last: int32 agg[n]; prolong_scale = 1: float64 w[n], k < last: float64 p[n];
//   "AMGEND01".
#include <chrono>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "amg_internal.cuh"

namespace {

constexpr char kMagic[8] = {'A', 'M', 'G', 'H', 'I', 'E', 'R', '1'};
constexpr char kTrailer[8] = {'A', 'M', 'G', 'E', 'N', 'D', '0', '1'};
constexpr uint32_t kVersion = 1;
constexpr uint32_t kParams = sizeof(amg_params) / sizeof(int32_t);

struct FileCloser {
  void operator()(FILE* f) const {
    if (f) fclose(f);
  }
};
using File = std::unique_ptr<FILE, FileCloser>;

// device array -> file (through a host copy)
template <typename T>
bool put_dev(amg_handle* h, FILE* f, const T* dev, size_t count) {
  if (count == 0) return true;
  std::vector<T> host(count);
  if (cudaMemcpyAsync(host.data(), dev, sizeof(T) * count, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return false;
  return fwrite(host.data(), sizeof(T), count, f) == count;
}

template <typename T>
bool put(FILE* f, const T& v) {
  return fwrite(&v, sizeof(T), 1, f) == 1;
}

template <typename T>
bool get(FILE* f, T& v) {
  return fread(&v, sizeof(T), 1, f) == 1;
}

// file -> new device array of the handle
template <typename T>
amg_status get_dev(amg_handle* h, FILE* f, T** dev, size_t count, const char* what) {
  *dev = static_cast<T*>(amg_alloc(h, sizeof(T) * (count ? count : 1)));
  if (!*dev) return amg_fail(h, AMG_ERR_OOM, "device allocation for %s failed", what);
  if (count == 0) return AMG_OK;
  std::vector<T> host(count);
  if (fread(host.data(), sizeof(T), count, f) != count)
    return amg_fail(h, AMG_ERR_INVALID_ARG, "file ends inside %s", what);
  AMG_CK(h, cudaMemcpyAsync(*dev, host.data(), sizeof(T) * count, cudaMemcpyHostToDevice, h->stream));
  AMG_CK(h, cudaStreamSynchronize(h->stream));  // host must outlive the copy
  return AMG_OK;
}

}  // namespace

extern "C" amg_status amg_save(const amg_handle* hc, const char* path) {
  if (!hc || !path) return AMG_ERR_INVALID_ARG;
  amg_handle* h = const_cast<amg_handle*>(hc);  // only the stream and the error text are used
  File f(fopen(path, "wb"));
  if (!f) return amg_fail(h, AMG_ERR_INVALID_ARG, "cannot open %s for writing", path);
  FILE* fp = f.get();
  bool ok = fwrite(kMagic, 1, 8, fp) == 8 && put(fp, kVersion) && put(fp, kParams) &&
            fwrite(&h->p, sizeof(int32_t), kParams, fp) == kParams && put(fp, (int32_t)h->nl) &&
            put(fp, (int32_t)h->npair);
  for (int k = 0; ok && k < h->nl; ++k) {
    const Level& L = h->L[k];
    const bool last = k == h->nl - 1;
    ok = put(fp, (int32_t)L.n) && put(fp, (int64_t)L.nnz) && put_dev(h, fp, L.rp, (size_t)L.n + 1) &&
         put_dev(h, fp, L.ci, (size_t)L.nnz) && put_dev(h, fp, L.v, (size_t)L.nnz) &&
         put(fp, (int32_t)(L.omega ? 1 : 0)) && (!L.omega || put_dev(h, fp, L.omega, (size_t)L.n)) &&
         (last || put_dev(h, fp, L.agg, (size_t)L.n));
    if (ok && h->p.prolong_scale == 1)
      ok = put_dev(h, fp, L.wsv, (size_t)L.n) && (last || put_dev(h, fp, L.pw, (size_t)L.n));
  }
  ok = ok && fwrite(kTrailer, 1, 8, fp) == 8;
  if (!ok) return amg_fail(h, AMG_ERR_CUDA, "writing %s failed (disk or device copy)", path);
  if (fclose(f.release()) != 0) return amg_fail(h, AMG_ERR_CUDA, "closing %s failed", path);
  return AMG_OK;
}

// the fields of amg_params that decide the hierarchy (the file's must be kept)
static bool same_hierarchy_fields(const amg_params& a, const amg_params& b) {
  return a.aggr_steps == b.aggr_steps && a.max_levels == b.max_levels && a.coarse_size == b.coarse_size &&
         a.num_parts == b.num_parts && a.prolong_scale == b.prolong_scale;
}

static amg_status load_impl(amg_handle* h, const char* path, const amg_params* p) {
  File f(fopen(path, "rb"));
  if (!f) return amg_fail(h, AMG_ERR_INVALID_ARG, "cannot open %s", path);
  FILE* fp = f.get();
  char magic[8];
  uint32_t version = 0, q = 0;
  if (fread(magic, 1, 8, fp) != 8 || memcmp(magic, kMagic, 8) != 0)
    return amg_fail(h, AMG_ERR_INVALID_ARG, "%s is not a saved hierarchy", path);
  if (!get(fp, version) || version != kVersion || !get(fp, q) || q != kParams)
    return amg_fail(h, AMG_ERR_INVALID_ARG, "%s: unsupported version or parameter block", path);
  amg_params saved;
  if (fread(&saved, sizeof(int32_t), kParams, fp) != kParams)
    return amg_fail(h, AMG_ERR_INVALID_ARG, "%s: file ends inside the parameters", path);
  if (p && !same_hierarchy_fields(saved, *p))
    return amg_fail(h, AMG_ERR_INVALID_ARG,
                    "%s: aggr_steps, max_levels, coarse_size, num_parts and prolong_scale must equal the saved ones",
                    path);
  h->p = p ? *p : saved;
  int32_t nl = 0, npair = 0;
  if (!get(fp, nl) || !get(fp, npair) || nl < 1 || nl > AMG_MAXL || npair < 0)
    return amg_fail(h, AMG_ERR_INVALID_ARG, "%s: bad level count", path);
  AMG_ALLOC(h, h->dev_flags, int, 1);
  AMG_ALLOC(h, h->zero_flag, int, 4);
  h->nl = nl;
  h->npair = npair;
  for (int k = 0; k < nl; ++k) {
    Level& L = h->L[k];
    const bool last = k == nl - 1;
    int32_t n = 0, has_omega = 0;
    int64_t nnz = 0;
    if (!get(fp, n) || !get(fp, nnz) || n < 1 || nnz < n || nnz >= (1ll << 31))
      return amg_fail(h, AMG_ERR_INVALID_ARG, "%s: bad size of level %d", path, k);
    if (k > 0 && n >= h->L[k - 1].n) return amg_fail(h, AMG_ERR_INVALID_ARG, "%s: level %d does not coarsen", path, k);
    L.n = n;
    L.nnz = nnz;
    amg_status st = get_dev(h, fp, &L.rp, (size_t)n + 1, "row pointers");
    if (st == AMG_OK) st = get_dev(h, fp, &L.ci, (size_t)nnz, "column indices");
    if (st == AMG_OK) st = get_dev(h, fp, &L.v, (size_t)nnz, "values");
    if (st != AMG_OK) return st;
    if (!get(fp, has_omega)) return amg_fail(h, AMG_ERR_INVALID_ARG, "%s: file ends in level %d", path, k);
    if (has_omega && (st = get_dev(h, fp, &L.omega, (size_t)n, "damping")) != AMG_OK) return st;
    if (!last && (st = get_dev(h, fp, &L.agg, (size_t)n, "aggregation map")) != AMG_OK) return st;
    if (h->p.prolong_scale == 1) {
      if ((st = get_dev(h, fp, &L.wsv, (size_t)n, "smooth vector")) != AMG_OK) return st;
      if (!last && (st = get_dev(h, fp, &L.pw, (size_t)n, "prolongator values")) != AMG_OK) return st;
    }
  }
  if (fread(magic, 1, 8, fp) != 8 || memcmp(magic, kTrailer, 8) != 0)
    return amg_fail(h, AMG_ERR_INVALID_ARG, "%s: truncated or corrupt (no end mark)", path);
  // the CSR and the maps came from a file: check them like a caller's matrix
  // (structure on every level, aggregation maps in range) before any kernel uses them
  for (int k = 0; k < nl; ++k) {
    const Level& L = h->L[k];
    int32_t ends[2] = {0, 0};
    AMG_CK(h, cudaMemcpyAsync(&ends[0], L.rp, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    AMG_CK(h, cudaMemcpyAsync(&ends[1], L.rp + L.n, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    AMG_CK(h, cudaStreamSynchronize(h->stream));
    if (ends[0] != 0 || ends[1] != L.nnz) return amg_fail(h, AMG_ERR_INVALID_ARG, "%s: level %d: bad row pointers", path, k);
    amg_status st = amg_check_level(h, k, k < nl - 1 ? h->L[k + 1].n : 0);
    if (st != AMG_OK) return st;
  }
  for (int k = 0; k + 1 < nl; ++k) {
    amg_status st = amg_build_members(h, k);
    if (st != AMG_OK) return st;
    if (h->p.prolong_scale == 1 && (st = amg_member_values(h, k)) != AMG_OK) return st;
  }
  return amg_finish_setup(h);
}

extern "C" amg_status amg_saved_params(const char* path, amg_params* out) {
  if (!path || !out) return AMG_ERR_INVALID_ARG;
  File f(fopen(path, "rb"));
  char magic[8];
  uint32_t version = 0, q = 0;
  amg_params p;
  if (!f || fread(magic, 1, 8, f.get()) != 8 || memcmp(magic, kMagic, 8) != 0 || !get(f.get(), version) ||
      version != kVersion || !get(f.get(), q) || q != kParams ||
      fread(&p, sizeof(int32_t), kParams, f.get()) != kParams) {
    amg_set_setup_error(std::string("amg_saved_params: ") + path + " is not a readable saved hierarchy");
    return AMG_ERR_INVALID_ARG;
  }
  *out = p;
  return AMG_OK;
}

extern "C" amg_status amg_load(const char* path, const amg_params* p, void* stream, amg_handle** out) {
  if (!out) return AMG_ERR_INVALID_ARG;
  *out = nullptr;
  if (!path) return AMG_ERR_INVALID_ARG;
  amg_handle* h = new amg_handle();
  h->stream = (cudaStream_t)stream;
  amg_read_hooks(h);
  auto t0 = std::chrono::steady_clock::now();
  amg_status st = load_impl(h, path, p);
  if (st != AMG_OK) {
    amg_set_setup_error(h->err);
    cudaStreamSynchronize(h->stream);
    amg_destroy(h);
    return st;
  }
  h->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = h;
  return AMG_OK;
}
