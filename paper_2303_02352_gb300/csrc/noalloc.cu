// amg_residual_norm_noalloc: the true-residual kernel of the solver, callable
// without a handle and without any device allocation.
//
// Who needs it: code that may not call cudaMalloc or cudaFree itself, for
// example a plugin or framework component whose host process owns every byte
// of device memory through its own allocator (a raw cudaMalloc would bypass
// that allocator's budget and fragment its pool), or a latency-sensitive loop
// that cannot afford the device synchronisation cudaMalloc/cudaFree may
// imply.  Such a caller passes only its own inputs and outputs.
//
// The reduction's scratch (one pair of partial sums per block and a ticket
// counter) lives in the file-scope device array below, so the library holds it
// on every GPU that loads it, for the life of the process.  Its size bounds the
// problem: at most AMG_NOALLOC_MAX_BLOCKS blocks of AMG_NOALLOC_ROWS rows.
// All calls share the array: calls that overlap on the GPU (different streams
// without ordering between them) race on it and give wrong results.
#include <mutex>

#include "amg_internal.cuh"

#define AMG_NOALLOC_ROWS 256
#define AMG_NOALLOC_MAX_BLOCKS 8192
#define AMG_NOALLOC_MAX_ROWS (AMG_NOALLOC_ROWS * AMG_NOALLOC_MAX_BLOCKS)  // 2,097,152 rows
#define AMG_NOALLOC_MAX_DEVICES 64

// [0, 2*MAX_BLOCKS): per-block partial sums; element 2*MAX_BLOCKS: ticket counter
static __device__ __align__(256) double g_noalloc_scratch[2 * AMG_NOALLOC_MAX_BLOCKS + 32];

// r = b - A x (r optional), norms[0] = |b - A x|_2, norms[1] = |b|_2.
// One thread per row; deterministic fixed-order reduction.
__global__ void __launch_bounds__(AMG_NOALLOC_ROWS)
    k_resid_norm_noalloc(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                         const double* __restrict__ v, const double* __restrict__ b, const double* __restrict__ x,
                         double* __restrict__ r, double* __restrict__ norms, double* scratch) {
  __shared__ double red[64];
  double acc[2] = {0.0, 0.0};
  const int row = blockIdx.x * AMG_NOALLOC_ROWS + threadIdx.x;
  if (row < n) {
    double s = 0.0;
    for (int p = rp[row]; p < rp[row + 1]; ++p) s += v[p] * x[ci[p]];
    const double bi = b[row], ri = bi - s;
    if (r) r[row] = ri;
    acc[0] = ri * ri;
    acc[1] = bi * bi;
  }
  unsigned* counter = reinterpret_cast<unsigned*>(scratch + 2 * AMG_NOALLOC_MAX_BLOCKS);
  if (grid_sum<2>(acc, scratch, counter, red) && threadIdx.x == 0) {
    norms[0] = sqrt(acc[0]);
    norms[1] = sqrt(acc[1]);
  }
}

static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[AMG_NOALLOC_MAX_DEVICES];

// Device address of the scratch array on the current device.  Host code only
// holds a stand-in for the array's name, so the address is looked up once per
// device (with that device current) and cached.
static amg_status noalloc_scratch(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= AMG_NOALLOC_MAX_DEVICES) {
    amg_set_setup_error("amg_residual_norm_noalloc: no usable current device");
    return AMG_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      amg_set_setup_error(std::string("amg_residual_norm_noalloc: cudaGetSymbolAddress failed: ") +
                          cudaGetErrorString(e));
      return AMG_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return AMG_OK;
}

extern "C" amg_status amg_residual_norm_noalloc(const amg_csr* A, const double* b, const double* x, double* r,
                                                double* norms, void* stream) {
  if (!A || !b || !x || !norms || !A->row_ptr || !A->col_idx || !A->val || A->n <= 0) {
    amg_set_setup_error("amg_residual_norm_noalloc: NULL pointer or empty matrix");
    return AMG_ERR_INVALID_ARG;
  }
  if (A->n > AMG_NOALLOC_MAX_ROWS) {
    amg_set_setup_error("amg_residual_norm_noalloc: n = " + std::to_string(A->n) + " exceeds the maximum of " +
                        std::to_string(AMG_NOALLOC_MAX_ROWS) + " rows set by its fixed scratch array");
    return AMG_ERR_TOO_LARGE;
  }
  double* scratch = nullptr;
  amg_status st = noalloc_scratch(&scratch);
  if (st != AMG_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the ticket counter must start at zero (the array keeps the previous call's contents)
  cudaError_t e = cudaMemsetAsync(scratch + 2 * AMG_NOALLOC_MAX_BLOCKS, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) {
    const int blocks = (A->n + AMG_NOALLOC_ROWS - 1) / AMG_NOALLOC_ROWS;
    k_resid_norm_noalloc<<<blocks, AMG_NOALLOC_ROWS, 0, s>>>(A->n, A->row_ptr, A->col_idx, A->val, b, x, r, norms,
                                                            scratch);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    amg_set_setup_error(std::string("amg_residual_norm_noalloc: ") + cudaGetErrorString(e));
    return AMG_ERR_CUDA;
  }
  return AMG_OK;
}
