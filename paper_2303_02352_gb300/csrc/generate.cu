// Problem generators on the device.  The paper's benchmark (Sec. 5, App. A) has
// the library generate the 7-point Poisson matrix on each process instead of
// reading it; here the 7- and 27-point stencil matrices of the benchmark and of
// the variable-coefficient studies are written straight into device memory,
// with their right-hand sides, so a large problem needs no host matrix and no
// host-to-device copy.
//
// The matrices are the host generator's (paper_2303_02352_gb300/workloads.py)
// bit for bit: unknowns numbered x + N y + N^2 z, Dirichlet unknowns
// eliminated, entries of a row in ascending column order (the stencil offsets
// sorted by their linear offset), link coefficient 2 k_i k_j / (k_i + k_j)
// divided by |d|^2 off the axes, a link leaving the domain using k_i, the
// diagonal summing the links in offset order; every operation is rounded on
// its own so no contraction changes a bit.  The coefficient of a cell is the
// value of its block (blocks of block^3 cells): the caller passes those few
// values, computed on the host with the host's exp/log/cos and rounded to
// float32, so both sides start from the same numbers.
#include "amg_internal.cuh"

// a(t): stored entries along one axis for coordinate t (itself and the
// neighbours inside [0, N)); A(t) = a(0) + ... + a(t-1)
__device__ __forceinline__ long long ax_cnt(int t, int N) { return 1 + (t > 0) + (t < N - 1); }
__device__ __forceinline__ long long ax_pre(int t) { return t == 0 ? 0 : 2 + 3ll * (t - 1); }

// first entry of row (x, y, z): the number of entries of all rows before it
__device__ __forceinline__ long long row_start(int points, int N, int x, int y, int z) {
  const long long T = 3ll * N - 2;
  if (points == 27)  // a row holds a(x) a(y) a(z) entries
    return ax_pre(z) * T * T + ax_cnt(z, N) * ax_pre(y) * T + ax_cnt(z, N) * ax_cnt(y, N) * ax_pre(x);
  // 7 points: a(x) + a(y) + a(z) - 2 entries
  return 2ll * N * T * z + (long long)N * N * (ax_pre(z) - 2ll * z) + T * y +
         (long long)N * (ax_pre(y) + (ax_cnt(z, N) - 2) * y) + ax_pre(x) + x * (ax_cnt(y, N) + ax_cnt(z, N) - 2);
}

__device__ __forceinline__ double cell_k(const float* kb, int nb, int block, int x, int y, int z) {
  return (double)kb[(x / block) + nb * (y / block) + nb * nb * (z / block)];
}

// one thread per row; kb == nullptr: the integer Poisson stencil (links 1)
__global__ void k_stencil(int N, int points, const float* __restrict__ kb, int nb, int block,
                          int32_t* __restrict__ rp, int32_t* __restrict__ ci, double* __restrict__ val) {
  const long long n = (long long)N * N * N;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  if (i == n) {
    const long long T = 3ll * N - 2;
    rp[n] = (int32_t)(points == 27 ? T * T * T : 7ll * N * N * N - 6ll * N * N);
    return;
  }
  const int x = (int)(i % N), y = (int)((i / N) % N), z = (int)(i / ((long long)N * N));
  long long p = row_start(points, N, x, y, z);
  rp[i] = (int32_t)p;
  const double ki = kb ? cell_k(kb, nb, block, x, y, z) : 1.0;
  // entries in ascending column order: offsets sorted by (dz, dy, dx); the
  // diagonal's slot is filled once its row sum is known
  double diag = 0.0;
  long long pdiag = -1;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int d2 = dx * dx + dy * dy + dz * dz;
        if (points == 7 && d2 > 1) continue;
        if (d2 == 0) {
          ci[p] = (int32_t)i;
          pdiag = p++;
          continue;
        }
        const int a = x + dx, b = y + dy, c = z + dz;
        const bool inside = a >= 0 && a < N && b >= 0 && b < N && c >= 0 && c < N;
        double link, link_out;
        if (!kb) {
          link = 1.0;
          link_out = 1.0;
        } else {
          const double kj = inside ? cell_k(kb, nb, block, a, b, c) : ki;
          link = __ddiv_rn(__dmul_rn(2.0, __dmul_rn(ki, kj)), __dadd_rn(ki, kj));
          link_out = ki;
        }
        if (d2 != 1) {
          link = __ddiv_rn(link, (double)d2);
          link_out = __ddiv_rn(link_out, (double)d2);
        }
        diag = __dadd_rn(diag, inside ? link : link_out);
        if (inside) {
          ci[p] = (int32_t)(a + (long long)N * b + (long long)N * N * c);
          val[p] = -link;
          ++p;
        }
      }
  val[pdiag] = diag;
}

// SplitMix64 (Steele, Lea and Flood, 2014): output idx of the stream seeded
// with seed, as the host generator defines its streams
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t idx) {
  uint64_t z = seed + (idx + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// out_i = 2 U_i - 1, U_i from the top 53 bits of output i of stream seed
__global__ void k_random_vector(int64_t n, uint64_t seed, double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double u = (double)(splitmix64(seed, (uint64_t)i) >> 11) * (1.0 / 9007199254740992.0);
  out[i] = __dsub_rn(__dmul_rn(2.0, u), 1.0);
}

// y = A x, each row's products rounded, then summed in column order from the first
static __global__ void k_rhs(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                             const double* __restrict__ v, const double* __restrict__ x, double* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int p0 = rp[i], p1 = rp[i + 1];
  double s = __dmul_rn(v[p0], x[ci[p0]]);
  for (int p = p0 + 1; p < p1; ++p) s = __dadd_rn(s, __dmul_rn(v[p], x[ci[p]]));
  y[i] = s;
}

static bool stencil_size(int32_t N, int32_t points, int64_t* n, int64_t* nnz) {
  if (N < 3 || (points != 7 && points != 27)) return false;
  const long long T = 3ll * N - 2;
  *n = (long long)N * N * N;
  *nnz = points == 27 ? T * T * T : 7ll * N * N * N - 6ll * N * N;
  return *nnz < (1ll << 31);
}

extern "C" amg_status amg_stencil_size(int32_t N, int32_t points, int64_t* n, int64_t* nnz) {
  if (!n || !nnz) return AMG_ERR_INVALID_ARG;
  if (!stencil_size(N, points, n, nnz)) {
    amg_set_setup_error("amg_stencil_size: N must be >= 3, points 7 or 27, and nnz below 2^31");
    return AMG_ERR_INVALID_ARG;
  }
  return AMG_OK;
}

extern "C" amg_status amg_generate_stencil(int32_t N, int32_t points, const float* kblock, int32_t block,
                                           int32_t* row_ptr, int32_t* col_idx, double* val, void* stream) {
  int64_t n = 0, nnz = 0;
  if (!stencil_size(N, points, &n, &nnz) || !row_ptr || !col_idx || !val || (kblock && block < 1)) {
    amg_set_setup_error("amg_generate_stencil: bad size, points, block or NULL output");
    return AMG_ERR_INVALID_ARG;
  }
  if (!kblock && points == 27) {
    amg_set_setup_error("amg_generate_stencil: the 27-point stencil needs a coefficient field");
    return AMG_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* kdev = nullptr;
  int nb = 0;
  if (kblock) {  // the block values to the device (stream-ordered, freed after the launch)
    nb = (N + block - 1) / block;
    const size_t bytes = sizeof(float) * (size_t)nb * nb * nb;
    if (cudaMallocAsync((void**)&kdev, bytes, s) != cudaSuccess) {
      amg_set_setup_error("amg_generate_stencil: allocation of the block values failed");
      return AMG_ERR_OOM;
    }
    if (cudaMemcpyAsync(kdev, kblock, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) {
      cudaFreeAsync(kdev, s);
      amg_set_setup_error("amg_generate_stencil: copying the block values failed");
      return AMG_ERR_CUDA;
    }
  }
  const unsigned grid = (unsigned)((n + 1 + AMG_BLOCK - 1) / AMG_BLOCK);
  k_stencil<<<grid, AMG_BLOCK, 0, s>>>(N, points, kdev, nb, block, row_ptr, col_idx, val);
  cudaError_t e = cudaGetLastError();
  if (kdev) cudaFreeAsync(kdev, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // kblock is the caller's host memory
  if (e != cudaSuccess) {
    amg_set_setup_error(std::string("amg_generate_stencil: ") + cudaGetErrorString(e));
    return AMG_ERR_CUDA;
  }
  return AMG_OK;
}

extern "C" amg_status amg_random_vector(int64_t n, uint64_t seed, double* out, void* stream) {
  if (n < 0 || (n > 0 && !out)) {
    amg_set_setup_error("amg_random_vector: negative size or NULL output");
    return AMG_ERR_INVALID_ARG;
  }
  if (n == 0) return AMG_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_random_vector<<<(unsigned)((n + AMG_BLOCK - 1) / AMG_BLOCK), AMG_BLOCK, 0, s>>>(n, seed, out);
  if (cudaGetLastError() != cudaSuccess) {
    amg_set_setup_error("amg_random_vector: launch failed");
    return AMG_ERR_CUDA;
  }
  return AMG_OK;
}

extern "C" amg_status amg_csr_times(const amg_csr* A, const double* x, double* y, void* stream) {
  if (!A || A->n <= 0 || !A->row_ptr || !A->col_idx || !A->val || !x || !y) {
    amg_set_setup_error("amg_csr_times: NULL pointer or empty matrix");
    return AMG_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_rhs<<<amg_blocks(A->n), AMG_BLOCK, 0, s>>>(A->n, A->row_ptr, A->col_idx, A->val, x, y);
  if (cudaGetLastError() != cudaSuccess) {
    amg_set_setup_error("amg_csr_times: launch failed");
    return AMG_ERR_CUDA;
  }
  return AMG_OK;
}
