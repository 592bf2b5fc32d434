// Solve phase on the GPU: the V-cycle of Alg. 2 (read through the operator
// B^k of Sec. 3.1) with l1-Jacobi smoothing, and the flexible PCG of Alg. 1.
//
// All kernels are HBM-bound.  Row kernels give each CSR row a group of G lanes
// (G = power of two >= the average row length), so a warp reads a contiguous
// run of values and column indices; the group sums with shuffles and its first
// lane finishes the row (sweep update, residual, or the fused dot products).
// Every solve-phase kernel takes a `skip` flag and returns at once when it is
// set: the FCG iteration is replayed as a CUDA graph in batches and the
// iterations after convergence cost one flag read per kernel.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "amg_internal.cuh"

// ---------------------------------------------------------------------------
// Row tiles.  A block owns R consecutive rows (R = the level's tile height).
// The nonzeros of those rows, [rp[row0], rp[row0 + R]), are contiguous in CSR:
// the block copies their values and column indices into shared memory with
// 16-byte loads (every byte of A is read once, fully coalesced), then each
// thread finishes one row from shared memory and gathers the vector through
// L1/L2.  One thread per row keeps the floating-point work at one multiply-add
// per nonzero (no shuffle reduction), which matters for FP64 on this part.
// A tile whose nonzeros exceed the buffer reads A directly from global memory
// (the tile height is chosen from the longest row, so this is a fallback only
// for matrices with very long rows).

#define TILE_BYTES 24576

template <typename MT>
struct TileSmem {
  static constexpr int VE = 16 / (int)sizeof(MT);              // elements per 16 bytes
  static constexpr int CAP = TILE_BYTES / ((int)sizeof(MT) + 4);  // nonzeros per tile
  MT v[CAP + 2 * VE];
  int32_t c[CAP + 8];
};

// s = sum_j a_ij x_j for row row0 + threadIdx.x (0 for threads past row1);
// with SUB, s = init - sum_j a_ij x_j accumulated from init (the residual
// form of the sweeps: one FP64 operation per row fewer).
// Ends with the tile's nonzeros in shared memory; the caller must
// __syncthreads() before the next call on the same buffer.
template <int R, typename MT, typename XT, typename AT, bool SUB = false>
__device__ __forceinline__ AT tile_row_dot(TileSmem<MT>& sm, int row0, int row1, const int32_t* __restrict__ rp,
                                           const int32_t* __restrict__ ci, const MT* __restrict__ v,
                                           const XT* __restrict__ x, int n, AT init = 0) {
  constexpr int VE = TileSmem<MT>::VE, CAP = TileSmem<MT>::CAP;
  const int p0 = __ldg(&rp[row0]);
  const int p1 = __ldg(&rp[row1]);
  const int row = row0 + (int)threadIdx.x;
  int q0 = 0, q1 = 0;
  if (row < row1) {
    q0 = __ldg(&rp[row]);
    q1 = __ldg(&rp[row + 1]);
  }
  AT s = SUB ? init : (AT)0;
  if (p1 - p0 <= CAP) {
    const int a0 = p0 & ~(VE - 1);
    const int nv = (p1 - a0 + VE - 1) / VE;
    const uint4* gv = reinterpret_cast<const uint4*>(v + a0);
    uint4* dv = reinterpret_cast<uint4*>(sm.v);
    for (int k = threadIdx.x; k < nv; k += R) dv[k] = __ldg(gv + k);
    const int c0 = p0 & ~3;
    const int nc = (p1 - c0 + 3) >> 2;
    const uint4* gc = reinterpret_cast<const uint4*>(ci + c0);
    uint4* dc = reinterpret_cast<uint4*>(sm.c);
    for (int k = threadIdx.x; k < nc; k += R) dc[k] = __ldg(gc + k);
    __syncthreads();
#pragma unroll 8
    for (int q = q0; q < q1; ++q) {
      const AT t = (AT)to_acc(sm.v[q - a0]) * (AT)__ldg(&x[amg_chk(sm.c[q - c0], n)]);
      if constexpr (SUB) s -= t;
      else s += t;
    }
  } else {
#pragma unroll 4
    for (int q = q0; q < q1; ++q) {
      const AT t = (AT)to_acc(__ldg(&v[q])) * (AT)__ldg(&x[amg_chk(__ldg(&ci[q]), n)]);
      if constexpr (SUB) s -= t;
      else s += t;
    }
  }
  return s;
}

// Elementwise kernels handle EW elements per thread, strided by the whole grid
// (every load stays coalesced; EW independent loads are in flight per thread).
#define EW 4
static inline int ew_blocks(int64_t n) { return (int)((n + (int64_t)AMG_BLOCK * EW - 1) / ((int64_t)AMG_BLOCK * EW)); }

// first sweep from z = 0: z = D r (the level input may be FP64 and the level
// float: then the rounded input is also kept in rcopy for the later sweeps)
template <typename RT, typename VT>
__global__ void __launch_bounds__(AMG_BLOCK) k_first(int n, const VT* __restrict__ dinv, const RT* __restrict__ r,
                                                     VT* __restrict__ rcopy, VT* __restrict__ z, const int* skip) {
  pdl_trigger();
  pdl_wait();
  if (*skip) return;
  const int T = gridDim.x * blockDim.x, i0 = blockIdx.x * blockDim.x + threadIdx.x;
  VT ri[EW], di[EW];
#pragma unroll
  for (int u = 0; u < EW; ++u) {
    const int i = i0 + u * T;
    if (i < n) {
      ri[u] = (VT)r[i];
      di[u] = dinv[i];
    }
  }
#pragma unroll
  for (int u = 0; u < EW; ++u) {
    const int i = i0 + u * T;
    if (i < n) {
      if (rcopy) rcopy[i] = ri[u];
      z[i] = di[u] * ri[u];
    }
  }
}

// l1-Jacobi sweep z_out = z + D (r - A z)
template <int R, typename MT, typename VT, typename OT>
__global__ void __launch_bounds__(R) k_sweep(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                             const MT* __restrict__ v, const VT* __restrict__ dinv,
                                             const VT* __restrict__ r, const VT* __restrict__ z,
                                             OT* __restrict__ zout, const int* skip) {
  pdl_trigger();
  pdl_wait();
  if (*skip) return;
  __shared__ __align__(16) TileSmem<MT> sm;
  const int row0 = blockIdx.x * R, row1 = min(row0 + R, n);
  const int row = row0 + threadIdx.x;
  const VT ri = row < row1 ? r[row] : (VT)0;
  const VT s = tile_row_dot<R, MT, VT, VT, true>(sm, row0, row1, rp, ci, v, z, n, ri);  // r_i - (A z)_i
  if (row < row1) zout[row] = (OT)(z[row] + dinv[row] * s);
}

// residual t = r - A z
template <int R, typename MT, typename VT>
__global__ void __launch_bounds__(R) k_resid(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                             const MT* __restrict__ v, const VT* __restrict__ r,
                                             const VT* __restrict__ z, VT* __restrict__ tout, const int* skip) {
  pdl_trigger();
  pdl_wait();
  if (*skip) return;
  __shared__ __align__(16) TileSmem<MT> sm;
  const int row0 = blockIdx.x * R, row1 = min(row0 + R, n);
  const int row = row0 + threadIdx.x;
  const VT ri = row < row1 ? r[row] : (VT)0;
  const VT s = tile_row_dot<R, MT, VT, VT, true>(sm, row0, row1, rp, ci, v, z, n, ri);  // r_i - (A z)_i
  if (row < row1) tout[row] = s;
}

// plain y = A x (FP64), for the public amg_spmv
template <int R>
__global__ void __launch_bounds__(R) k_spmv(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                            const double* __restrict__ v, const double* __restrict__ x,
                                            double* __restrict__ y) {
  __shared__ __align__(16) TileSmem<double> sm;
  const int row0 = blockIdx.x * R, row1 = min(row0 + R, n);
  const double s = tile_row_dot<R, double, double, double>(sm, row0, row1, rp, ci, v, x, n);
  const int row = row0 + threadIdx.x;
  if (row < row1) y[row] = s;
}

// r_c[J] = sum over the members i of aggregate J (ascending) of t_i (one
// coarse row per thread: the member loads of a row depend on each other, so
// more rows per thread would only serialise them)
// (pwm: the prolongator's values in member order for a non-unit prolongator,
// r_c[J] = sum_i p_i t_i; nullptr for the unit one)
template <typename VT, typename CT>
__global__ void __launch_bounds__(AMG_BLOCK) k_restrict(int nc, const int32_t* __restrict__ mptr, const int32_t* __restrict__ mem,
                                                        const VT* __restrict__ t, CT* __restrict__ rc, const int* skip,
                                                        int n, const VT* __restrict__ pwm) {
  pdl_trigger();
  pdl_wait();
  if (*skip) return;
  const int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= nc) return;
  VT s = 0;
  if (pwm)
    for (int m = mptr[J]; m < mptr[J + 1]; ++m) s += pwm[m] * t[amg_chk(mem[m], n)];
  else
    for (int m = mptr[J]; m < mptr[J + 1]; ++m) s += t[amg_chk(mem[m], n)];
  rc[J] = (CT)s;
}

// restriction fused with the coarse level's first sweep from zero:
// r_c[J] = sum over the members i of J (ascending) of t_i, z_c[J] = D_c[J] r_c[J]
// (the same roundings as the restriction followed by the first sweep)
template <typename VT, typename CT>
__global__ void __launch_bounds__(AMG_BLOCK) k_restrict_first(int nc, const int32_t* __restrict__ mptr,
                                                              const int32_t* __restrict__ mem, const VT* __restrict__ t,
                                                              const CT* __restrict__ dinv_c, CT* __restrict__ rc,
                                                              CT* __restrict__ zc, const int* skip, int n,
                                                              const VT* __restrict__ pwm) {
  pdl_trigger();
  pdl_wait();
  if (*skip) return;
  const int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= nc) return;
  VT s = 0;
  if (pwm)
    for (int m = mptr[J]; m < mptr[J + 1]; ++m) s += pwm[m] * t[amg_chk(mem[m], n)];
  else
    for (int m = mptr[J]; m < mptr[J + 1]; ++m) s += t[amg_chk(mem[m], n)];
  const CT r = (CT)s;
  rc[J] = r;
  zc[J] = dinv_c[J] * r;
}

// z_i += z_c[agg(i)]  (unit piecewise-constant prolongator), or
// z_i += p_i z_c[agg(i)] with the prolongator's values pw (nullptr: unit)
template <typename VT, typename CT>
__global__ void __launch_bounds__(AMG_BLOCK) k_prolong(int n, const int32_t* __restrict__ agg, const CT* __restrict__ zc,
                                                       VT* __restrict__ z, const int* skip, int nc,
                                                       const VT* __restrict__ pw) {
  pdl_trigger();
  pdl_wait();
  if (*skip) return;
  const int T = gridDim.x * blockDim.x, i0 = blockIdx.x * blockDim.x + threadIdx.x;
  int a[EW];
  VT zz[EW], pp[EW];
#pragma unroll
  for (int u = 0; u < EW; ++u) {
    const int i = i0 + u * T;
    a[u] = 0;
    pp[u] = 1;
    if (i < n) {
      a[u] = agg[i];
      zz[u] = z[i];
      if (pw) pp[u] = pw[i];
    }
  }
#pragma unroll
  for (int u = 0; u < EW; ++u) {
    const int i = i0 + u * T;
    if (i < n) z[i] = pw ? zz[u] + pp[u] * (VT)zc[amg_chk(a[u], nc)] : zz[u] + (VT)zc[amg_chk(a[u], nc)];
  }
}

// prolongator values of a level in the level's vector type (nullptr: unit)
template <typename VT>
static const VT* pw_of(const Level& L) {
  if constexpr (sizeof(VT) == 8) return (const VT*)L.pw;
  else return (const VT*)L.pwf;
}
template <typename VT>
static const VT* pwm_of(const Level& L) {
  if constexpr (sizeof(VT) == 8) return (const VT*)L.pwm;
  else return (const VT*)L.pwmf;
}

template <typename VT, typename OT>
__global__ void k_copy(int n, const VT* __restrict__ a, OT* __restrict__ b, const int* skip) {
  pdl_trigger();
  pdl_wait();
  if (*skip) return;
  const int T = gridDim.x * blockDim.x, i0 = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
  for (int u = 0; u < EW; ++u) {
    const int i = i0 + u * T;
    if (i < n) b[i] = (OT)a[i];
  }
}

template <typename VT>
__global__ void k_add(int n, const VT* __restrict__ x, VT* __restrict__ y, const int* skip) {
  pdl_trigger();
  pdl_wait();
  if (*skip) return;
  const int T = gridDim.x * blockDim.x, i0 = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
  for (int u = 0; u < EW; ++u) {
    const int i = i0 + u * T;
    if (i < n) y[i] += x[i];
  }
}

template <typename VT>
__global__ void k_zero(int n, VT* __restrict__ a, const int* skip) {
  pdl_trigger();
  pdl_wait();
  if (*skip) return;
  const int T = gridDim.x * blockDim.x, i0 = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
  for (int u = 0; u < EW; ++u) {
    const int i = i0 + u * T;
    if (i < n) a[i] = (VT)0;
  }
}

// ---------------------------------------------------------------------------
// Alg. 1 kernels (FP64, level-0 matrix).  The row kernels run a persistent
// grid of red_grid blocks over the row tiles; the scalar work of each step is
// done by the last block of the grid-wide reduction (fixed order: the result
// does not depend on timing).

enum { RES_INIT = 0, RES_TRUE = 1, RES_NORM = 2 };

// scalar bookkeeping after r = b - A u (acc[0] = |r|^2, acc[1] = |b|^2)
// RES_INIT: iteration 0.  RES_TRUE: the stop test on the true residual, run
// when the recursive residual dropped below tol (need_true = 1) or
// periodically in mixed precision (need_true = 2).  RES_NORM: exit report.
template <int MODE>
__device__ __forceinline__ void fcg_residual_epilogue(FcgState* st, const double (&acc)[2]) {
  if (MODE == RES_INIT) {
    const double nb = sqrt(acc[1]);
    st->nb = nb;
    st->it = 0;
    st->need_true = 0;
    st->status = AMG_OK;
    st->rho = 0.0;
    if (nb == 0.0) {
      st->res = 0.0;
      st->true_res = 0.0;
      if (st->hist_len > 0) st->hist[0] = 0.0;
      st->done = 1;
    } else {
      const double res = sqrt(acc[0]) / nb;
      st->res = res;
      if (st->hist_len > 0) st->hist[0] = res;
      st->true_res = res;
      st->done = (res < st->tol) || (st->maxit <= 0);
      if (!(res < st->tol) && st->maxit <= 0) st->status = AMG_NOT_CONVERGED;
    }
  } else if (MODE == RES_TRUE) {
    const double tr = sqrt(acc[0]) / st->nb;
    const int it = st->it;
    st->true_res = tr;
    if (tr < st->tol) {
      if (st->need_true == 2 && it < st->hist_len) st->hist[it] = tr;
      st->res = tr;
      st->status = AMG_OK;
      st->done = 1;
    } else {
      if (it < st->hist_len) st->hist[it] = tr;
      st->res = tr;
      if (it >= st->maxit) {
        st->status = AMG_NOT_CONVERGED;
        st->done = 1;
      }
    }
    st->need_true = 0;
  } else {
    st->true_res = st->nb > 0 ? sqrt(acc[0]) / st->nb : 0.0;
  }
}

// Non-pipelined variants (levels whose rows are too long for a pipeline tile).
// RES_INIT: r = b - A u, |r|^2, |b|^2.  RES_TRUE: r = b - A u when asked.
// RES_NORM: |b - A u| / |b| only.
template <int R, int MODE>
__global__ void __launch_bounds__(R) k_fcg_resid(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                                 const double* __restrict__ v, const double* __restrict__ b,
                                                 const double* __restrict__ u, double* __restrict__ r, FcgState* st,
                                                 double* partial, unsigned* counter) {
  pdl_trigger();
  pdl_wait();
  if (MODE == RES_TRUE && (st->done || !st->need_true)) return;
  __shared__ __align__(16) TileSmem<double> sm;
  __shared__ double red[64];
  double acc[2] = {0.0, 0.0};
  const int ntiles = (n + R - 1) / R;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int row0 = tile * R, row1 = min(row0 + R, n);
    const double s = tile_row_dot<R, double, double, double>(sm, row0, row1, rp, ci, v, u, n);
    const int row = row0 + threadIdx.x;
    if (row < row1) {
      const double bi = b[row], ri = bi - s;
      if (MODE != RES_NORM) r[row] = ri;
      acc[0] += ri * ri;
      if (MODE == RES_INIT) acc[1] += bi * bi;
    }
    __syncthreads();
  }
  if (!grid_sum<2>(acc, partial, counter, red) || threadIdx.x != 0) return;
  fcg_residual_epilogue<MODE>(st, acc);
}

// v = A w;  alpha = w.r, beta = w.v, gamma = w.q;  rho and the step scalars
template <int R>
__global__ void __launch_bounds__(R) k_fcg_spmv_dots(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                                     const double* __restrict__ v, const double* __restrict__ w,
                                                     const double* __restrict__ r, const double* __restrict__ q,
                                                     double* __restrict__ vout, FcgState* st, double* partial,
                                                     unsigned* counter) {
  pdl_trigger();
  pdl_wait();
  if (st->done) return;
  __shared__ __align__(16) TileSmem<double> sm;
  __shared__ double red[96];
  const bool first = st->it == 0;
  double acc[3] = {0.0, 0.0, 0.0};
  const int ntiles = (n + R - 1) / R;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int row0 = tile * R, row1 = min(row0 + R, n);
    const double s = tile_row_dot<R, double, double, double>(sm, row0, row1, rp, ci, v, w, n);
    const int row = row0 + threadIdx.x;
    if (row < row1) {
      const double wi = w[row];
      vout[row] = s;
      acc[0] += wi * r[row];
      acc[1] += wi * s;
      if (!first) acc[2] += wi * q[row];
    }
    __syncthreads();
  }
  if (!grid_sum<3>(acc, partial, counter, red) || threadIdx.x != 0) return;
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
}

// d = w - g d; q = v - g q; u += a d; r -= a q; |r|^2; stop bookkeeping
__global__ void __launch_bounds__(AMG_BLOCK) k_fcg_axpy(int n, const double* __restrict__ w, const double* __restrict__ vv,
                                                        double* __restrict__ d, double* __restrict__ q,
                                                        double* __restrict__ u, double* __restrict__ r, FcgState* st,
                                                        double* partial, unsigned* counter) {
  pdl_trigger();
  pdl_wait();
  if (st->done) return;
  __shared__ double red[32];
  const bool first = st->it == 0;
  const double g = st->g, a = st->a;
  double acc[1] = {0.0};
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    double di, qi;
    if (first) {
      di = w[i];
      qi = vv[i];
    } else {
      di = w[i] - g * d[i];
      qi = vv[i] - g * q[i];
    }
    d[i] = di;
    q[i] = qi;
    u[i] += a * di;
    const double ri = r[i] - a * qi;
    r[i] = ri;
    acc[0] += ri * ri;
  }
  if (!grid_sum<1>(acc, partial, counter, red) || threadIdx.x != 0) return;
  if (st->timing) return;
  const int it = st->it + 1;
  st->it = it;
  const double res = sqrt(acc[0]) / st->nb;
  st->res = res;
  if (it < st->hist_len) st->hist[it] = res;
  const bool periodic = st->mixed && st->true_every > 0 && (it % st->true_every) == 0;
  st->need_true = (res < st->tol) ? 1 : (periodic ? 2 : 0);
  if (!st->need_true && it >= st->maxit) {
    st->status = AMG_NOT_CONVERGED;
    st->done = 1;
  }
}

// AMG_PDL: 0 off, 1 every solve-phase kernel, 2 the V-cycle kernels only (default:
// measured best; on the outer reduction kernels it costs more than it saves)
static int pdl_mode() {
  static int on = -1;
  if (on < 0) {
    const char* e = getenv("AMG_PDL");
    on = e ? atoi(e) : 2;
  }
  return on;
}
static thread_local bool g_outer_launch = false;  // set while the outer FCG kernels are launched
bool amg_pdl_enabled() {
  const int m = pdl_mode();
  return m == 1 || (m == 2 && !g_outer_launch);
}
struct OuterLaunch {
  OuterLaunch() { g_outer_launch = true; }
  ~OuterLaunch() { g_outer_launch = false; }
};

int amg_num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

#include "rows.cuh"
#include "pair.cuh"
#include "bottom.cuh"

// ---------------------------------------------------------------------------
// launch helpers (dispatch on the tile height and on the pipeline depth)

#define DISPATCH_R(RR, CALL)                          \
  switch (RR) {                                       \
    case 256: { constexpr int TR = 256; CALL; } break; \
    case 128: { constexpr int TR = 128; CALL; } break; \
    case 64: { constexpr int TR = 64; CALL; } break;   \
    default: { constexpr int TR = 32; CALL; } break;   \
  }

// pipelined kernels: two stages (measured best); dispatch on threads per row
#define DISPATCH_TPR(TT, CALL)                          \
  switch (TT) {                                         \
    case 1: { constexpr int TP = 1; CALL; } break;      \
    case 2: { constexpr int TP = 2; CALL; } break;      \
    case 4: { constexpr int TP = 4; CALL; } break;      \
    case 8: { constexpr int TP = 8; CALL; } break;      \
    case 16: { constexpr int TP = 16; CALL; } break;    \
    default: { constexpr int TP = 32; CALL; } break;    \
  }

// sb = 6 (any value type, tiles of R = 128, 64 or 32 rows): two consumer
// groups of 128 threads take the tiles in turn from four standard stages, each
// with half the threads per row of the standard form (1, 2, 4 for R = 128,
// 64, 32).  Fewer shuffle reductions and fewer idle lanes per row, where the
// FP64 issue rate limits the standard form; half the resident blocks.
#define DISPATCH_NG(RR, CALL)                                  \
  switch (RR) {                                                \
    case 128: { constexpr int TP = 1; CALL; } break;           \
    case 64: { constexpr int TP = 2; CALL; } break;            \
    default: { constexpr int TP = 4; CALL; } break;            \
  }

// pattern-coded forms: standard stages with 1, 2 or 4 threads per row (tiles
// of 256, 128, 64 rows) and the two-group form; the setup enables the pattern
// form of a level only for these (pat_form in setup.cu)
#define DISPATCH_TPR_PAT(TT, CALL)                      \
  switch (TT) {                                         \
    case 1: { constexpr int TP = 1; CALL; } break;      \
    case 2: { constexpr int TP = 2; CALL; } break;      \
    default: { constexpr int TP = 4; CALL; } break;     \
  }

// the pattern-coded columns of level L in a row kernel's arguments (form: the
// column form of this launch's kernel, Level::pat / patd); pcb set selects the
// form that locates rows from the tuple lengths
template <typename MT, typename VT, typename OT>
static inline void use_patterns(RowArgs<MT, VT, OT>& a, const Level& L, int form) {
  if (!form || !L.pid) return;
  a.pid = L.pid;
  a.ptab = L.ptab;
  a.pk = L.pk;
  a.ptab_n = L.npat * L.pk;
  a.plen = L.plen;
  a.npat = L.npat;
  a.pcb = form == 2 ? L.pcb : nullptr;
  a.stage_rows = L.stage_rows ? 1 : 0;
}

// sb = 2 / 4: FP64 level with long rows in 2x / 4x stages (R = 128 with two
// threads per row / R = 256 with one); sb = 5: two consumer groups taking
// tiles in turn, R = 128 rows with one thread per row, four 2x stages
template <int MODE, typename MT, typename VT, typename OT>
static void launch_rows(cudaStream_t s, int R, int sb, const RowArgs<MT, VT, OT>& a0) {
  // the forms with a row-data area move the row pointers and row vectors by
  // bulk copy where every source is 16-byte aligned (the library's own
  // buffers are)
  RowArgs<MT, VT, OT> b = a0;
  auto al = [](const void* p) { return ((uintptr_t)p & 15u) == 0; };
  b.stage_rows = a0.stage_rows && al(a0.rp) && al(a0.x) && al(a0.r) && al(a0.dinv) && al(a0.b);
  const RowArgs<MT, VT, OT>& a = b;
  if constexpr (MODE != PM_SWEEP_PROLONG) {  // latency-bound levels only: no pattern form
    if (a.pid) {
      if (b.pcb) {  // one thread per row: R = 128 in two groups, or R = 256
        if (sb == 6) launch_pipe<1, 4, MODE, MT, VT, OT, 1, 2, 2>(s, b);
        else launch_pipe<1, 2, MODE, MT, VT, OT, 1, 1, 2>(s, b);
      } else if (sb == 6) {
        DISPATCH_NG(R, (launch_pipe<TP, 4, MODE, MT, VT, OT, 1, 2, 1>(s, b)));
      } else {
        DISPATCH_TPR_PAT(PIPE_CONSUMERS / R, (launch_pipe<TP, 2, MODE, MT, VT, OT, 1, 1, 1>(s, b)));
      }
      return;
    }
  }
  if (sb == 6) {
    DISPATCH_NG(R, (launch_pipe<TP, 4, MODE, MT, VT, OT, 1, 2>(s, a)));
    return;
  }
  if constexpr (sizeof(MT) == 8) {
    if (sb == 5) {
      launch_pipe<1, 4, MODE, MT, VT, OT, 2, 2>(s, a);
      return;
    }
    if (sb == 4) {
      launch_pipe<1, 2, MODE, MT, VT, OT, 4>(s, a);
      return;
    }
    if (sb == 2) {
      launch_pipe<2, 2, MODE, MT, VT, OT, 2>(s, a);
      return;
    }
  }
  DISPATCH_TPR(PIPE_CONSUMERS / R, (launch_pipe<TP, 2, MODE, MT, VT, OT>(s, a)));
}

template <typename MT, typename VT, typename OT>
static void launch_sweep(cudaStream_t s, const Level& L, const MT* vals, const VT* dinv, const VT* r, const VT* z, OT* out,
                         const int* skip, int* flags) {
  const int R = L.R;
  if (L.pipe) {
    RowArgs<MT, VT, OT> a{L.n, L.rp, L.ci, vals, z, dinv, r, nullptr, nullptr, out, skip, nullptr, nullptr, nullptr, flags};
    a.stage_rows = L.stage_rows ? 1 : 0;
    use_patterns(a, L, L.pat);
    launch_rows<PM_SWEEP>(s, R, L.sb, a);
    return;
  }
  const int nb = (L.n + R - 1) / R;
  DISPATCH_R(R, (amg_launch(k_sweep<TR, MT, VT, OT>, dim3(nb), dim3(TR), 0, s, L.n, L.rp, L.ci, vals, dinv, r, z, out, skip)));
}

// grid of the pipelined row kernel of `MODE` on a level with tiles of R rows
template <int MODE, typename MT, typename VT, typename OT>
static int rows_grid(int R, int sb, int n) {
  if (sb == 6) {
    int g = 0;
    DISPATCH_NG(R, (g = pipe_grid<TP, 4, MODE, MT, VT, OT, 1, 2>(n)));
    return g;
  }
  if constexpr (sizeof(MT) == 8) {
    if (sb == 5) return pipe_grid<1, 4, MODE, MT, VT, OT, 2, 2>(n);
    if (sb == 4) return pipe_grid<1, 2, MODE, MT, VT, OT, 4>(n);
    if (sb == 2) return pipe_grid<2, 2, MODE, MT, VT, OT, 2>(n);
  }
  int g = 0;
  DISPATCH_TPR(PIPE_CONSUMERS / R, (g = pipe_grid<TP, 2, MODE, MT, VT, OT>(n)));
  return g;
}

// sweep of a coarse level fused with the prolongation of its result into the
// finer level's iterate zf.  Only where every block of the sweep has at most
// one tile (a latency-bound level: the fused kernel saves a launch); on larger
// levels the member scatter inside the tile loop costs more than the separate
// prolongation kernel (measured).  false: nothing launched.
template <typename MT, typename VT>
static bool launch_sweep_prolong(cudaStream_t s, const Level& C, const MT* vals, const VT* dinv, const VT* r, const VT* z,
                                 VT* out, const int* skip, int* flags, const Level& F, void* zf, bool any_size = false) {
  if (!C.pipe || F.pw) return false;  // unit prolongators only
  const int tiles = (C.n + C.R - 1) / C.R;
  if (!any_size && rows_grid<PM_SWEEP_PROLONG, MT, VT, VT>(C.R, C.sb, C.n) < tiles) return false;
  RowArgs<MT, VT, VT> a{C.n, C.rp, C.ci, vals, z, dinv, r, nullptr, nullptr, out, skip, nullptr, nullptr, nullptr, flags,
                        F.mptr, F.mem, zf, F.lowp ? 0 : 1, F.n};
  launch_rows<PM_SWEEP_PROLONG>(s, C.R, C.sb, a);
  return true;
}

template <typename MT, typename VT>
static void launch_resid(cudaStream_t s, const Level& L, const MT* vals, const VT* r, const VT* z, VT* t, const int* skip,
                         int* flags) {
  const int R = L.R;
  if (L.pipe) {
    RowArgs<MT, VT, VT> a{L.n, L.rp, L.ci, vals, z, nullptr, r, nullptr, nullptr, t, skip, nullptr, nullptr, nullptr, flags};
    a.stage_rows = L.stage_rows ? 1 : 0;
    use_patterns(a, L, L.pat);
    launch_rows<PM_RESID>(s, R, L.sb, a);
    return;
  }
  const int nb = (L.n + R - 1) / R;
  DISPATCH_R(R, (amg_launch(k_resid<TR, MT, VT>, dim3(nb), dim3(TR), 0, s, L.n, L.rp, L.ci, vals, r, z, t, skip)));
}

// two consecutive row passes of level L in one launch (pair.cuh): a sweep
// z1 = z0 + D (r - A z0), then MODE2 on z1 into out.  false (nothing
// launched) where the level runs the non-pipelined kernels, has no pairing
// state, or (use_pair = 1) has too few tiles for the lag to leave room for
// reuse through L2.
template <int MODE2, typename MT, typename VT, typename OT>
static bool launch_pair(amg_handle* h, cudaStream_t s, const Level& L, const MT* vals, const VT* dinv, const VT* r,
                        const VT* z0, VT* z1, OT* out, const int* skip, bool force = false) {
  if (!(h->use_pair || force) || !L.pipe || !L.pctl || L.sb != 1) return false;
  const int R = L.R;
  const int ntiles = (L.n + R - 1) / R;
  const int halo = (L.bw + R - 1) / R;
  int grid = 0;
  DISPATCH_TPR(PIPE_CONSUMERS / R, (grid = pair_grid<TP, PAIR_STAGES, MODE2, MT, VT, OT>(L.n)));
  const int lag = halo + PAIR_CHUNK + 1 + (h->pair_slack >= 0 ? h->pair_slack : 2 * grid);
  if (h->use_pair == 1 && !force && ntiles < 2 * lag) return false;
  PairArgs<MT, VT, OT> a{L.n, L.rp, L.ci, vals, dinv, r, z0, z1, out, skip, h->dev_flags, L.pctl, L.pcnt, halo, lag};
  DISPATCH_TPR(PIPE_CONSUMERS / R, (launch_pair_tpr<TP, PAIR_STAGES, MODE2, MT, VT, OT>(s, a)));
  return true;
}

// zeroes the paired-pass state of every level (after a bounded wait expired)
static void pair_reset(amg_handle* h) {
  for (int k = 0; k < h->nl; ++k) {
    Level& L = h->L[k];
    if (!L.pctl) continue;
    const int ntiles = (L.n + L.R - 1) / L.R;
    cudaMemsetAsync(L.pctl, 0, sizeof(PairCtl), h->stream);
    cudaMemsetAsync(L.pcnt, 0, sizeof(unsigned) * (size_t)ntiles, h->stream);
  }
}

// outer kernels on level 0 (FP64 values)
static void launch_dots(amg_handle* h, cudaStream_t s) {
  OuterLaunch outer;
  Level& L = h->L[0];
  if (L.piped) {
    RowArgs<double, double, double> a{L.n, L.rp, L.ci, L.v, h->w, nullptr, h->r, nullptr, h->q, h->v,
                                      nullptr, h->st, h->partial, h->counter, h->dev_flags};
    use_patterns(a, L, L.patd);
    launch_rows<PM_DOTS>(s, L.Rd, L.sbd, a);
    return;
  }
  DISPATCH_R(L.Rd, (k_fcg_spmv_dots<TR><<<h->red_grid, TR, 0, s>>>(L.n, L.rp, L.ci, L.v, h->w, h->r, h->q, h->v, h->st,
                                                                   h->partial, h->counter)));
}

template <int MODE>
static void launch_fcg_resid(amg_handle* h, cudaStream_t s) {
  OuterLaunch outer;
  Level& L = h->L[0];
  constexpr int PM = MODE == RES_INIT ? PM_RINIT : (MODE == RES_TRUE ? PM_RTRUE : PM_RNORM);
  if (L.piped) {
    RowArgs<double, double, double> a{L.n, L.rp, L.ci, L.v, h->u, nullptr, nullptr, h->b, nullptr,
                                      MODE == RES_NORM ? nullptr : h->r, nullptr, h->st, h->partial, h->counter,
                                      h->dev_flags};
    use_patterns(a, L, L.patd);
    launch_rows<PM>(s, L.Rd, L.sbd, a);
    return;
  }
  DISPATCH_R(L.Rd, (k_fcg_resid<TR, MODE><<<h->red_grid, TR, 0, s>>>(L.n, L.rp, L.ci, L.v, h->b, h->u,
                                                                     MODE == RES_NORM ? nullptr : h->r, h->st,
                                                                     h->partial, h->counter)));
}

// ---------------------------------------------------------------------------
// V-cycle recording.  Level k < nl-1 runs in VT (double, or float when the
// hierarchy is low precision); the coarsest level always runs in FP64.

struct VRec {
  amg_handle* h;
  cudaStream_t s;
  const int* skip;
  int launches = 0;
  double bytes = 0.0;  // algorithmic bytes of the recorded launches
  void add(double b) {
    launches++;
    bytes += b;
  }
};

// algorithmic bytes: a row pass reads the row pointers, every value and column
// index once, and (by cache reuse) the gathered vector once
// index once; with pattern-coded columns (form 1) one id byte per row replaces
// the column indices (the table of offsets is a few KB), and form 2 reads one
// row pointer per 32 rows instead of one per row
static double row_pass(const Level& L, double sv, int form = 0) {
  if (!form || !L.pid) return (double)L.nnz * (sv + 4.0) + 4.0 * (L.n + 1.0);
  const double ptrs = form == 2 ? 4.0 * ((L.n + 31) / 32 + 1.0) : 4.0 * (L.n + 1.0);
  return (double)L.nnz * sv + ptrs + (double)L.n;
}
static double val_bytes(const Level& L) { return L.lowp ? (L.vb ? 2.0 : 4.0) : 8.0; }
static double vec_bytes(const Level& L) { return L.lowp ? 4.0 : 8.0; }

// prolongation target handed to a coarse level: the finer level and its
// iterate.  The coarse level's last sweep adds its result to that iterate
// (PM_SWEEP_PROLONG) and sets `done`; otherwise the caller prolongs.
struct Prol {
  const Level* F;
  void* z;
  bool done;
};

// extra algorithmic bytes of a sweep that also prolongs: the aggregates'
// member pointers and ids, read-modify-write of the finer iterate
static double prolong_fused_bytes(const Level& F, const Level& C) {
  return 4.0 * (C.n + 1.0) + 4.0 * F.n + 2.0 * vec_bytes(F) * F.n;
}

// coarsest level: `sweeps` l1-Jacobi sweeps from zero on r (double); returns the
// buffer that holds the result.  first_done: the restriction already wrote the
// first sweep's result D r into za.
static double* rec_coarse(VRec& R, int k, const double* r, double* final_out, bool first_done = false,
                          Prol* pro = nullptr) {
  Level& L = R.h->L[k];
  double* za = (double*)L.za;
  double* zb = (double*)L.zb;
  int sweeps = R.h->p.coarse_sweeps;
  const double n = L.n;
  double* cur = za;
  if (sweeps <= 0) {
    double* o = final_out ? final_out : za;
    amg_launch(k_zero<double>, dim3(ew_blocks(L.n)), dim3(AMG_BLOCK), 0, R.s, L.n, o, R.skip);
    R.add(8.0 * n);
    return o;
  }
  double* o = za;
  if (!first_done) {
    if (sweeps == 1 && final_out) o = final_out;
    amg_launch(k_first<double, double>, dim3(ew_blocks(L.n)), dim3(AMG_BLOCK), 0, R.s, L.n, L.dinv, r, nullptr, o, R.skip);
    R.add(24.0 * n);
  }
  cur = o;
  for (int sw = 1; sw < sweeps; ++sw) {
    double* nxt = (sw == sweeps - 1 && final_out) ? final_out : (cur == za ? zb : za);
    if (sw == sweeps - 1 && pro &&
        launch_sweep_prolong<double, double>(R.s, L, L.v, L.dinv, r, cur, nxt, R.skip, R.h->dev_flags, *pro->F, pro->z)) {
      pro->done = true;
      R.add(row_pass(L, 8.0) + 32.0 * n + prolong_fused_bytes(*pro->F, L));
    } else {
      launch_sweep<double, double, double>(R.s, L, L.v, L.dinv, r, cur, nxt, R.skip, R.h->dev_flags);
      R.add(row_pass(L, 8.0, L.pat) + 32.0 * n);
    }
    cur = nxt;
  }
  return cur;
}

// level k in type VT with matrix values MT.  rin: level input (RT = double at
// level 0, VT elsewhere).  final_out (level 0 only): where the last sweep writes.
// first_done: the restriction already wrote the first sweep's result into za.
// pro: where the last post-smoothing sweep prolongs its result (if it can).
template <typename VT, typename MT, typename RT>
static VT* rec_level(VRec& R, int k, const RT* rin, double* final_out, bool first_done = false, Prol* pro = nullptr);

// ---------------------------------------------------------------------------
// fused bottom: plan (at setup) and recording

struct BotPlan {
  BotArgs a;
  int cs = 0;      // cluster size
  int smem = 0;    // dynamic shared memory per block
  double bytes = 0.0;
};

void amg_free_bottom(amg_handle* h) {
  delete h->bot;
  h->bot = nullptr;
}

static int align16(int x) { return (x + 15) & ~15; }

// layout of the bottom levels kb .. nl-1 for a cluster of cs blocks; returns
// the shared memory per block.  rps[j] / mps[j]: host copies of level kb+j's
// row pointers and member pointers.
static long long bottom_layout(amg_handle* h, int kb, int cs, BotArgs& a, const std::vector<std::vector<int32_t>>& rps,
                               const std::vector<std::vector<int32_t>>& mps) {
  a.nb = h->nl - kb;
  long long off = 0;
  for (int j = 0; j < a.nb; ++j) {
    const Level& L = h->L[kb + j];
    const bool coarsest = kb + j == h->nl - 1;
    BotLevel& B = a.L[j];
    const int es = coarsest ? 8 : (L.lowp ? 4 : 8);  // vector and value bytes
    const int chunk = (L.n + cs - 1) / cs;
    B.n = L.n;
    B.chunk = chunk;
    B.magic = ((1ull << 32) + (unsigned long long)chunk - 1) / (unsigned long long)chunk;
    B.rp = L.rp;
    B.ci = L.ci;
    B.v = (!coarsest && L.lowp) ? (const void*)L.vf : (const void*)L.v;
    B.dinv = (!coarsest && L.lowp) ? (const void*)L.dinvf : (const void*)L.dinv;
    int emax = 0;
    for (int c = 0; c <= BOT_MAX_CS; ++c) B.e0[c] = rps[j][std::min(c * chunk, L.n)];
    for (int c = 0; c < cs; ++c) emax = std::max(emax, B.e0[c + 1] - B.e0[c]);
    int cchunk = 0, mmax = 0;
    if (!coarsest) {
      const Level& C = h->L[kb + j + 1];
      cchunk = (C.n + cs - 1) / cs;
      for (int c = 0; c <= BOT_MAX_CS; ++c) B.m0[c] = mps[j][std::min(c * cchunk, C.n)];
      for (int c = 0; c < cs; ++c) mmax = std::max(mmax, B.m0[c + 1] - B.m0[c]);
      B.agg = L.agg;
      B.mptr = L.mptr;
      B.mem = L.mem;
    } else {
      B.agg = B.mptr = B.mem = nullptr;
      for (int c = 0; c <= BOT_MAX_CS; ++c) B.m0[c] = 0;
    }
    auto take = [&](long long bytes) {
      const int o = (int)off;
      off += align16((int)bytes);
      return o;
    };
    B.o_rp = take(4ll * (chunk + 1));
    B.o_ci = take(4ll * emax);
    B.o_v = take((long long)es * emax);
    B.o_dinv = take((long long)es * chunk);
    B.o_agg = coarsest ? 0 : take(4ll * chunk);
    B.o_mptr = coarsest ? 0 : take(4ll * (cchunk + 1));
    B.o_mem = coarsest ? 0 : take(4ll * mmax);
    B.o_r = take((long long)es * chunk);
    B.o_za = take((long long)es * chunk);
    B.o_zb = take((long long)es * chunk);
    B.o_t = take((long long)es * chunk);
  }
  return off;
}

// mean number of distinct owner blocks that one warp-wide load of the row
// kernel reaches: warps take 32 consecutive rows of a block, load u takes the
// u-th entry of each row.  Loads that reach several blocks are served one
// block after another, so the fused bottom pays off only where this stays
// near 1 (regular stencil hierarchies: 1.1-1.3; irregular 27-point coarse
// levels: 1.9-2.5).
static double owner_spread(const std::vector<int32_t>& rp, const std::vector<int32_t>& ci, int n, int chunk) {
  double tot = 0.0, cnt = 0.0;
  for (int r0 = 0; r0 < n; r0 += chunk) {
    const int r1 = std::min(n, r0 + chunk);
    for (int w0 = r0; w0 < r1; w0 += 32) {
      const int w1 = std::min(r1, w0 + 32);
      int len = 0;
      for (int i = w0; i < w1; ++i) len = std::max(len, rp[i + 1] - rp[i]);
      for (int u = 0; u < len; ++u) {
        int owners[32], no = 0;
        for (int i = w0; i < w1; ++i) {
          if (rp[i] + u >= rp[i + 1]) continue;
          const int o = ci[rp[i] + u] / chunk;
          bool seen = false;
          for (int q = 0; q < no; ++q) seen = seen || owners[q] == o;
          if (!seen) owners[no++] = o;
        }
        tot += no;
        cnt += 1.0;
      }
    }
  }
  return cnt > 0.0 ? tot / cnt : 1.0;
}

// the first level kb >= 1 from which every level has at most BOT_MAX_ROWS rows
// and whose slices fit one cluster's shared memory (16 blocks, else 8).  In
// the automatic mode (use_bottom = 2) the plan is kept only where every
// bottom level's owner spread is at most 1.5.
amg_status amg_plan_bottom(amg_handle* h) {
  amg_free_bottom(h);
  h->kb = h->nl;
  int k0 = 1;
  while (k0 < h->nl && (h->L[k0].n > BOT_MAX_ROWS || h->nl - k0 > BOT_MAXL)) ++k0;
  if (k0 >= h->nl) return AMG_OK;
  std::vector<std::vector<int32_t>> rps(h->nl - k0), mps(h->nl - k0);
  for (int k = k0; k < h->nl; ++k) {
    const Level& L = h->L[k];
    rps[k - k0].resize(L.n + 1);
    AMG_CK(h, cudaMemcpyAsync(rps[k - k0].data(), L.rp, 4ull * (L.n + 1), cudaMemcpyDeviceToHost, h->stream));
    if (k < h->nl - 1) {
      const int nc = h->L[k + 1].n;
      mps[k - k0].resize(nc + 1);
      AMG_CK(h, cudaMemcpyAsync(mps[k - k0].data(), L.mptr, 4ull * (nc + 1), cudaMemcpyDeviceToHost, h->stream));
    }
  }
  AMG_CK(h, cudaStreamSynchronize(h->stream));
  for (int kb = k0; kb < h->nl; ++kb) {
    std::vector<std::vector<int32_t>> r(rps.begin() + (kb - k0), rps.end()), m(mps.begin() + (kb - k0), mps.end());
    for (int cs : {16, 8}) {
      BotPlan P;
      const long long smem = bottom_layout(h, kb, cs, P.a, r, m);
      if (smem > BOT_SMEM_MAX) continue;
      const bool fits = h->L[kb].lowp ? bottom_fits<float>(cs, (int)smem) : bottom_fits<double>(cs, (int)smem);
      if (!fits) continue;
      if (h->use_bottom == 2) {
        for (int k = kb; k < h->nl; ++k) {
          const Level& L = h->L[k];
          std::vector<int32_t> ci(L.nnz);
          AMG_CK(h, cudaMemcpyAsync(ci.data(), L.ci, 4ull * L.nnz, cudaMemcpyDeviceToHost, h->stream));
          AMG_CK(h, cudaStreamSynchronize(h->stream));
          if (owner_spread(rps[k - k0], ci, L.n, (L.n + cs - 1) / cs) > 1.5) return AMG_OK;
        }
      }
      P.cs = cs;
      P.smem = (int)smem;
      h->bot = new BotPlan(P);
      h->kb = kb;
      return AMG_OK;
    }
  }
  return AMG_OK;
}

// the bottom levels kb .. nl-1 in one cluster launch; result in L[kb].za
static void rec_bottom(VRec& R) {
  amg_handle* h = R.h;
  const int kb = h->kb;
  BotPlan& P = *h->bot;
  BotArgs a = P.a;
  a.pre = h->p.pre_sweeps;
  a.post = h->p.post_sweeps;
  a.csweeps = h->p.coarse_sweeps;
  a.skip = R.skip;
  a.r_in = h->L[kb].r;
  a.z_out = h->L[kb].za;
  double bytes = 0.0;  // the algorithmic bytes of the passes it replaces
  for (int j = 0; j < a.nb; ++j) {
    Level& L = h->L[kb + j];
    const bool coarsest = kb + j == h->nl - 1;
    const double n = L.n, sx = coarsest ? 8.0 : vec_bytes(L), sv = coarsest ? 8.0 : val_bytes(L);
    if (coarsest) {
      bytes += 3.0 * sx * n + (h->p.coarse_sweeps - 1) * (row_pass(L, sv) + 4.0 * sx * n);
    } else {
      const Level& C = h->L[kb + j + 1];
      const bool cc = kb + j + 1 == h->nl - 1;
      const double nc = C.n, sc = cc ? 8.0 : vec_bytes(C);
      bytes += 3.0 * sx * n + (h->p.pre_sweeps - 1 + h->p.post_sweeps) * (row_pass(L, sv) + 4.0 * sx * n);
      bytes += row_pass(L, sv) + 3.0 * sx * n;                           // residual
      bytes += 4.0 * (nc + 1) + 4.0 * n + sx * n + sc * nc;              // restriction
      bytes += 4.0 * n + sc * nc + 2.0 * sx * n;                         // prolongation
    }
  }
  if (h->L[kb].lowp) launch_bottom<float>(R.s, a, P.cs, P.smem);
  else launch_bottom<double>(R.s, a, P.cs, P.smem);
  R.add(bytes);
}

template <typename VT>
static void rec_child(VRec& R, int k, const VT* t, VT* z) {
  amg_handle* h = R.h;
  Level& L = h->L[k];
  Level& C = h->L[k + 1];
  const int ncb = amg_blocks(C.n);
  const double sx = sizeof(VT), n = L.n, nc = C.n;
  const double wb = L.pw ? sx * n : 0.0;  // prolongator values read by a non-unit restriction / prolongation
  if (k + 1 == h->kb) {  // the bottom levels in one launch
    const double sc = vec_bytes(C);
    if (k + 1 == h->nl - 1) {
      amg_launch(k_restrict<VT, double>, dim3(amg_blocks(C.n)), dim3(AMG_BLOCK), 0, R.s, C.n, L.mptr, L.mem, t, (double*)C.r, R.skip, L.n, pwm_of<VT>(L));
      R.add(wb + 4.0 * (nc + 1) + 4.0 * n + sx * n + 8.0 * nc);
      rec_bottom(R);
      amg_launch(k_prolong<VT, double>, dim3(ew_blocks(L.n)), dim3(AMG_BLOCK), 0, R.s, L.n, L.agg, (const double*)C.za, z, R.skip, C.n, pw_of<VT>(L));
    } else {
      amg_launch(k_restrict<VT, VT>, dim3(amg_blocks(C.n)), dim3(AMG_BLOCK), 0, R.s, C.n, L.mptr, L.mem, t, (VT*)C.r, R.skip, L.n, pwm_of<VT>(L));
      R.add(wb + 4.0 * (nc + 1) + 4.0 * n + sx * n + sc * nc);
      rec_bottom(R);
      amg_launch(k_prolong<VT, VT>, dim3(ew_blocks(L.n)), dim3(AMG_BLOCK), 0, R.s, L.n, L.agg, (const VT*)C.za, z, R.skip, C.n, pw_of<VT>(L));
    }
    R.add(wb + 4.0 * n + sc * nc + 2.0 * sx * n);
    return;
  }
  const bool wcyc = h->p.cycle == 2;
  // restriction fused with the coarse level's first sweep, prolongation with
  // its last sweep (not in the W-cycle, whose correction sums two visits)
  const bool fuse = h->fuse && !wcyc;
  Prol pro{&L, (void*)z, false};
  if (k + 1 == h->nl - 1) {  // coarsest: FP64
    const bool fr = fuse && h->p.coarse_sweeps > 0;
    if (fr) {
      amg_launch(k_restrict_first<VT, double>, dim3(amg_blocks(C.n)), dim3(AMG_BLOCK), 0, R.s, C.n, L.mptr, L.mem, t,
                 (const double*)C.dinv, (double*)C.r, (double*)C.za, R.skip, L.n, pwm_of<VT>(L));
      R.add(wb + 4.0 * (nc + 1) + 4.0 * n + sx * n + 24.0 * nc);
    } else {
      amg_launch(k_restrict<VT, double>, dim3(amg_blocks(C.n)), dim3(AMG_BLOCK), 0, R.s, C.n, L.mptr, L.mem, t, (double*)C.r, R.skip, L.n, pwm_of<VT>(L));
      R.add(wb + 4.0 * (nc + 1) + 4.0 * n + sx * n + 8.0 * nc);
    }
    double* zc = rec_coarse(R, k + 1, (const double*)C.r, nullptr, fr, fuse ? &pro : nullptr);
    if (wcyc) {  // W-cycle: e = z_c;  r2 = r_c - A_c e;  e += B_c r2
      double* e = (double*)C.e;
      double* r2 = (double*)C.r2;
      amg_launch(k_copy<double, double>, dim3(ew_blocks(C.n)), dim3(AMG_BLOCK), 0, R.s, C.n, zc, e, R.skip);
      launch_resid<double, double>(R.s, C, C.v, (const double*)C.r, e, r2, R.skip, h->dev_flags);
      double* zc2 = rec_coarse(R, k + 1, r2, nullptr);
      amg_launch(k_add<double>, dim3(ew_blocks(C.n)), dim3(AMG_BLOCK), 0, R.s, C.n, zc2, e, R.skip);
      R.add(16.0 * nc);
      R.add(row_pass(C, 8.0, C.pat) + 24.0 * nc);
      R.add(24.0 * nc);
      zc = e;
    }
    if (!pro.done) {
      amg_launch(k_prolong<VT, double>, dim3(ew_blocks(L.n)), dim3(AMG_BLOCK), 0, R.s, L.n, L.agg, zc, z, R.skip, C.n, pw_of<VT>(L));
      R.add(wb + 4.0 * n + 8.0 * nc + 2.0 * sx * n);
    }
  } else {
    const double sc = vec_bytes(C);
    const bool fr = fuse && h->p.pre_sweeps > 0;
    if (fr) {
      const VT* dc = C.lowp ? (const VT*)C.dinvf : (const VT*)C.dinv;
      amg_launch(k_restrict_first<VT, VT>, dim3(amg_blocks(C.n)), dim3(AMG_BLOCK), 0, R.s, C.n, L.mptr, L.mem, t, dc,
                 (VT*)C.r, (VT*)C.za, R.skip, L.n, pwm_of<VT>(L));
      R.add(wb + 4.0 * (nc + 1) + 4.0 * n + sx * n + 3.0 * sc * nc);
    } else {
      amg_launch(k_restrict<VT, VT>, dim3(amg_blocks(C.n)), dim3(AMG_BLOCK), 0, R.s, C.n, L.mptr, L.mem, t, (VT*)C.r, R.skip, L.n, pwm_of<VT>(L));
      R.add(wb + 4.0 * (nc + 1) + 4.0 * n + sx * n + sc * nc);
    }
    Prol* pp = fuse ? &pro : nullptr;
    VT* zc;
    if (C.lowp) zc = (VT*)rec_level<float, float, float>(R, k + 1, (const float*)C.r, nullptr, fr, pp);
    else zc = (VT*)rec_level<double, double, double>(R, k + 1, (const double*)C.r, nullptr, fr, pp);
    if (wcyc) {
      VT* e = (VT*)C.e;
      VT* r2 = (VT*)C.r2;
      amg_launch(k_copy<VT, VT>, dim3(ew_blocks(C.n)), dim3(AMG_BLOCK), 0, R.s, C.n, zc, e, R.skip);
      if (C.lowp) launch_resid<float, float>(R.s, C, C.vf, (const float*)C.r, (const float*)e, (float*)r2, R.skip,
                                             h->dev_flags);
      else launch_resid<double, double>(R.s, C, C.v, (const double*)C.r, (const double*)e, (double*)r2, R.skip,
                                        h->dev_flags);
      VT* zc2;
      if (C.lowp) zc2 = (VT*)rec_level<float, float, float>(R, k + 1, (const float*)r2, nullptr);
      else zc2 = (VT*)rec_level<double, double, double>(R, k + 1, (const double*)r2, nullptr);
      amg_launch(k_add<VT>, dim3(ew_blocks(C.n)), dim3(AMG_BLOCK), 0, R.s, C.n, zc2, e, R.skip);
      R.add(2.0 * sc * nc);
      R.add(row_pass(C, val_bytes(C), C.pat) + 3.0 * sc * nc);
      R.add(3.0 * sc * nc);
      zc = e;
    }
    if (!pro.done) {
      amg_launch(k_prolong<VT, VT>, dim3(ew_blocks(L.n)), dim3(AMG_BLOCK), 0, R.s, L.n, L.agg, zc, z, R.skip, C.n, pw_of<VT>(L));
      R.add(wb + 4.0 * n + sc * nc + 2.0 * sx * n);
    }
  }
}

template <typename VT, typename MT, typename RT>
static VT* rec_level(VRec& R, int k, const RT* rin, double* final_out, bool first_done, Prol* pro) {
  amg_handle* h = R.h;
  Level& L = h->L[k];
  const MT* vals;
  if constexpr (std::is_same<MT, double>::value) vals = L.v;
  else if constexpr (std::is_same<MT, float>::value) vals = L.vf;
  else vals = L.vb;
  const VT* dinv;
  if constexpr (std::is_same<VT, double>::value) dinv = L.dinv;
  else dinv = L.dinvf;
  VT* za = (VT*)L.za;
  VT* zb = (VT*)L.zb;
  VT* t = (VT*)L.t;
  const int nb = amg_blocks(L.n);
  const double n = L.n, sx = sizeof(VT), sr = sizeof(RT), sv = sizeof(MT);
  // the level's own copy of its input, in VT
  const VT* r;
  VT* rcopy = nullptr;
  if constexpr (std::is_same<RT, VT>::value) {
    r = rin;
  } else {
    rcopy = L.r0f ? (VT*)L.r0f : (VT*)L.r;
    r = rcopy;
  }
  const double rc_bytes = rcopy ? sx * n : 0.0;
  // pre-smoothing from zero
  VT* cur = za;
  bool resid_done = false;
  if (h->p.pre_sweeps > 0) {
    if (!first_done) {
      amg_launch(k_first<RT, VT>, dim3(ew_blocks(L.n)), dim3(AMG_BLOCK), 0, R.s, L.n, dinv, rin, rcopy, za, R.skip);
      R.add(sr * n + 2.0 * sx * n + rc_bytes);
    }
    // sweeps 2 .. pre, paired where the level allows (two sweeps, or the last
    // sweep with the residual); byte counts per pass as for separate launches
    for (int left = h->p.pre_sweeps - 1; left > 0;) {
      VT* nxt = cur == za ? zb : za;
      if (left >= 2 && launch_pair<PM_SWEEP, MT, VT, VT>(h, R.s, L, vals, dinv, r, cur, nxt, cur, R.skip)) {
        R.add(2.0 * (row_pass(L, sv) + 4.0 * sx * n));
        left -= 2;
      } else if (left == 1 && launch_pair<PM_RESID, MT, VT, VT>(h, R.s, L, vals, dinv, r, cur, nxt, t, R.skip)) {
        R.add(row_pass(L, sv) + 4.0 * sx * n + row_pass(L, sv) + 3.0 * sx * n);
        cur = nxt;
        left = 0;
        resid_done = true;
      } else {
        launch_sweep<MT, VT, VT>(R.s, L, vals, dinv, r, cur, nxt, R.skip, h->dev_flags);
        R.add(row_pass(L, sv, L.pat) + 4.0 * sx * n);
        cur = nxt;
        --left;
      }
    }
  } else {
    if (rcopy) {
      amg_launch(k_copy<RT, VT>, dim3(ew_blocks(L.n)), dim3(AMG_BLOCK), 0, R.s, L.n, rin, rcopy, R.skip);
      R.add(sr * n + rc_bytes);
    }
    amg_launch(k_zero<VT>, dim3(ew_blocks(L.n)), dim3(AMG_BLOCK), 0, R.s, L.n, za, R.skip);
    R.add(sx * n);
  }
  // residual, restriction, coarse correction, prolongation
  if (!resid_done) {
    launch_resid<MT, VT>(R.s, L, vals, r, cur, t, R.skip, h->dev_flags);
    R.add(row_pass(L, sv, L.pat) + 3.0 * sx * n);
  }
  rec_child<VT>(R, k, t, cur);
  // post-smoothing
  const int post = h->p.post_sweeps;
  if (post == 0 && final_out) {
    amg_launch(k_copy<VT, double>, dim3(ew_blocks(L.n)), dim3(AMG_BLOCK), 0, R.s, L.n, cur, final_out, R.skip);
    R.add(sx * n + 8.0 * n);
    return nullptr;
  }
  for (int sw = 0; sw < post; ++sw) {
    VT* nxt = cur == za ? zb : za;
    // two sweeps in one launch where the level allows (not for a last sweep
    // that prolongs into the finer level)
    if (post - sw >= 2 && !(post - sw == 2 && pro)) {
      const bool last = post - sw == 2 && final_out;
      const bool paired = last ? launch_pair<PM_SWEEP, MT, VT, double>(h, R.s, L, vals, dinv, r, cur, nxt, final_out, R.skip)
                               : launch_pair<PM_SWEEP, MT, VT, VT>(h, R.s, L, vals, dinv, r, cur, nxt, cur, R.skip);
      if (paired) {
        R.add(2.0 * (row_pass(L, sv) + 4.0 * sx * n) + (last ? 8.0 * n - sx * n : 0.0));
        ++sw;
        if (last) return nullptr;
        continue;
      }
    }
    if (sw == post - 1 && final_out) {
      launch_sweep<MT, VT, double>(R.s, L, vals, dinv, r, cur, final_out, R.skip, h->dev_flags);
      R.add(row_pass(L, sv, L.pat) + 3.0 * sx * n + 8.0 * n);
      return nullptr;
    }
    if (sw == post - 1 && pro &&
        launch_sweep_prolong<MT, VT>(R.s, L, vals, dinv, r, cur, nxt, R.skip, h->dev_flags, *pro->F, pro->z)) {
      pro->done = true;
      R.add(row_pass(L, sv) + 4.0 * sx * n + prolong_fused_bytes(*pro->F, L));
    } else {
      launch_sweep<MT, VT, VT>(R.s, L, vals, dinv, r, cur, nxt, R.skip, h->dev_flags);
      R.add(row_pass(L, sv, L.pat) + 4.0 * sx * n);
    }
    cur = nxt;
  }
  return cur;
}

// w = B r on the handle's FCG vectors
static void record_vcycle(VRec& R, const double* r, double* w) {
  amg_handle* h = R.h;
  if (h->nl == 1) {
    rec_coarse(R, 0, r, w);
    return;
  }
  Level& L0 = h->L[0];
  if (!L0.lowp) rec_level<double, double, double>(R, 0, r, w);
  else if (L0.vb) rec_level<float, bf16, double>(R, 0, r, w);
  else rec_level<float, float, double>(R, 0, r, w);
}

// algorithmic bytes of the outer kernels: SpMV + dots reads A, gathers w,
// writes v, reads r and q; the axpys read w v d q u r and write d q u r
static double bytes_spmv_dots(const Level& L) { return row_pass(L, 8.0, L.patd) + 32.0 * L.n; }
static double bytes_axpy(const Level& L) { return 80.0 * L.n; }

static void record_iteration(VRec& R, bool precond) {
  amg_handle* h = R.h;
  Level& L = h->L[0];
  const int g = h->red_grid;
  FcgState* st = h->st;
  const int* skip = &st->done;
  R.skip = skip;
  if (precond) record_vcycle(R, h->r, h->w);
  else {
    amg_launch(k_copy<double, double>, dim3(ew_blocks(L.n)), dim3(AMG_BLOCK), 0, R.s, L.n, h->r, h->w, skip);
    R.add(16.0 * L.n);
  }
  launch_dots(h, R.s);
  R.add(bytes_spmv_dots(L));
  {
    OuterLaunch outer;
    amg_launch(k_fcg_axpy, dim3(h->ax_grid), dim3(AMG_BLOCK), 0, R.s, L.n, h->w, h->v, h->d, h->q, h->u, h->r, st,
               h->partial, h->counter);
  }
  R.add(bytes_axpy(L));
  // the true-residual check moves data only once per solve (at convergence)
  launch_fcg_resid<RES_TRUE>(h, R.s);
  R.add(0.0);
}

extern "C" amg_status amg_kernel_bytes(const amg_handle* h, int32_t which, int32_t level, double* bytes) {
  if (!h || !bytes || level < 0 || level >= h->nl) return AMG_ERR_INVALID_ARG;
  const Level& L = h->L[level];
  const double n = L.n, sx = vec_bytes(L), sv = val_bytes(L);
  const bool last = level == h->nl - 1;
  switch (which) {
    case 0: *bytes = row_pass(L, sv, L.pat) + 4.0 * sx * n; return AMG_OK;
    case 1: *bytes = row_pass(L, sv, L.pat) + 3.0 * sx * n; return AMG_OK;
    case 2:
    case 3: {
      if (last) return AMG_ERR_INVALID_ARG;
      const Level& C = h->L[level + 1];
      const double nc = C.n, sc = vec_bytes(C);
      *bytes = which == 2 ? 4.0 * (nc + 1) + 4.0 * n + sx * n + sc * nc : 4.0 * n + sc * nc + 2.0 * sx * n;
      return AMG_OK;
    }
    case 6:
    case 7: {
      if (last) return AMG_ERR_INVALID_ARG;
      const Level& C = h->L[level + 1];
      const double nc = C.n, sc = vec_bytes(C);
      *bytes = which == 6 ? 4.0 * (nc + 1) + 4.0 * n + sx * n + 3.0 * sc * nc
                          : row_pass(C, val_bytes(C)) + 4.0 * sc * nc + prolong_fused_bytes(L, C);
      return AMG_OK;
    }
    case 8: *bytes = row_pass(L, sv) + 5.0 * sx * n; return AMG_OK;  // matrix once; z0, r, D read; z1, z2 written
    case 4: *bytes = level == 0 ? bytes_spmv_dots(L) : 0.0; return level == 0 ? AMG_OK : AMG_ERR_INVALID_ARG;
    case 5: *bytes = level == 0 ? bytes_axpy(L) : 0.0; return level == 0 ? AMG_OK : AMG_ERR_INVALID_ARG;
    default: return AMG_ERR_INVALID_ARG;
  }
}

// ---------------------------------------------------------------------------
// preparation: work vectors, FCG state, graphs

amg_status amg_prepare_solve(amg_handle* h) {
  const int n = h->L[0].n;
  for (int k = 0; k < h->nl; ++k) {
    Level& L = h->L[k];
    size_t es = L.lowp ? sizeof(float) : sizeof(double);
    if (!(L.za = amg_alloc(h, es * L.n)) || !(L.zb = amg_alloc(h, es * L.n)) || !(L.t = amg_alloc(h, es * L.n)))
      return amg_fail(h, AMG_ERR_OOM, "work vectors of level %d", k);
    if (k > 0 && !(L.r = amg_alloc(h, es * L.n))) return amg_fail(h, AMG_ERR_OOM, "level input %d", k);
    if (k > 0 && h->p.cycle == 2 &&
        (!(L.e = amg_alloc(h, es * L.n)) || !(L.r2 = amg_alloc(h, es * L.n))))
      return amg_fail(h, AMG_ERR_OOM, "W-cycle vectors of level %d", k);
    if (k == 0 && L.lowp) AMG_ALLOC(h, L.r0f, float, L.n);
    if (L.pipe && !L.pctl) {  // paired-pass state (zero: epoch 0, watermark 0)
      const size_t ntiles = ((size_t)L.n + L.R - 1) / L.R;
      AMG_ALLOC(h, L.pctl, PairCtl, 1);
      AMG_ALLOC(h, L.pcnt, unsigned, ntiles);
      AMG_CK(h, cudaMemsetAsync(L.pctl, 0, sizeof(PairCtl), h->stream));
      AMG_CK(h, cudaMemsetAsync(L.pcnt, 0, sizeof(unsigned) * ntiles, h->stream));
    }
  }
  AMG_ALLOC(h, h->b, double, n);
  AMG_ALLOC(h, h->u, double, n);
  AMG_ALLOC(h, h->r, double, n);
  AMG_ALLOC(h, h->w, double, n);
  AMG_ALLOC(h, h->d, double, n);
  AMG_ALLOC(h, h->v, double, n);
  AMG_ALLOC(h, h->q, double, n);
  int dev = 0, sms = 148;
  AMG_CK(h, cudaGetDevice(&dev));
  AMG_CK(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t tiles = (n + h->L[0].Rd - 1) / h->L[0].Rd;
  h->red_grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)sms * 8));
  h->ax_grid = (int)std::max<int64_t>(1, std::min<int64_t>(amg_blocks(n), (int64_t)sms * 8));
  AMG_ALLOC(h, h->partial, double, (size_t)std::max(std::max(h->red_grid, h->ax_grid), 8192) * 4);
  AMG_ALLOC(h, h->counter, unsigned, 4);
  AMG_ALLOC(h, h->st, FcgState, 1);
  AMG_CK(h, cudaMallocHost((void**)&h->st_host, sizeof(FcgState)));
  memset(h->st_host, 0, sizeof(FcgState));
  h->hist_cap = 0;
  AMG_CK(h, cudaStreamSynchronize(h->stream));
  return amg_capture_graphs(h);
}

static void destroy_graphs(amg_handle* h) {
  if (h->g_vcycle) cudaGraphExecDestroy(h->g_vcycle);
  if (h->g_iter) cudaGraphExecDestroy(h->g_iter);
  if (h->g_iter_cg) cudaGraphExecDestroy(h->g_iter_cg);
  h->g_vcycle = h->g_iter = h->g_iter_cg = nullptr;
}

amg_status amg_capture_graphs(amg_handle* h) {
  destroy_graphs(h);
  // the graphs are captured even when use_graph = 0: the capture also counts
  // the launches and the algorithmic bytes of a V-cycle and of an iteration
  if (!h->cap) AMG_CK(h, cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
  auto capture = [&](auto&& body, cudaGraphExec_t* out, int* launches, double* bytes) -> amg_status {
    cudaGraph_t g = nullptr;
    AMG_CK(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    VRec R{h, h->cap, h->zero_flag};
    body(R);
    cudaError_t e = cudaStreamEndCapture(h->cap, &g);
    if (e != cudaSuccess) return amg_fail(h, AMG_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return amg_fail(h, AMG_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    if (launches) *launches = R.launches;
    if (bytes) *bytes = R.bytes;
    return AMG_OK;
  };
  amg_status st = capture([&](VRec& R) { record_vcycle(R, h->r, h->w); }, &h->g_vcycle, &h->launches_vcycle,
                          &h->bytes_vcycle);
  if (st != AMG_OK) return st;
  st = capture([&](VRec& R) { record_iteration(R, true); }, &h->g_iter, &h->launches_iter, &h->bytes_iter);
  if (st != AMG_OK) return st;
  st = capture([&](VRec& R) { record_iteration(R, false); }, &h->g_iter_cg, &h->launches_iter_cg, nullptr);
  if (st != AMG_OK) return st;
  AMG_CK(h, cudaGetLastError());
  return AMG_OK;
}

void amg_release_graphs(amg_handle* h) {
  destroy_graphs(h);
  if (h->cap) cudaStreamDestroy(h->cap);
  h->cap = nullptr;
  if (h->st_host) cudaFreeHost(h->st_host);
  h->st_host = nullptr;
}

// ---------------------------------------------------------------------------
// solves

// Self-check of the bounded-wait path: one block waits on an mbarrier phase
// that nothing completes; the wait must give up after limit_us and report.
__global__ void k_bounded_wait_check(uint64_t limit_ns, int* flags) {
  __shared__ unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0, limit_ns)) atomicOr(flags, ST_TIMEOUT);
}

extern "C" amg_status amg_check_bounded_wait(int32_t limit_us, void* stream) {
  if (limit_us <= 0 || limit_us > 2000000) return AMG_ERR_INVALID_ARG;
  int* flags = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMallocAsync((void**)&flags, sizeof(int), s) != cudaSuccess) return AMG_ERR_OOM;
  int host = 0;
  cudaMemsetAsync(flags, 0, sizeof(int), s);
  k_bounded_wait_check<<<1, 32, 0, s>>>((uint64_t)limit_us * 1000ull, flags);
  cudaMemcpyAsync(&host, flags, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(flags, s);
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return AMG_ERR_CUDA;
  return (host & ST_TIMEOUT) ? AMG_ERR_TIMEOUT : AMG_OK;
}

#ifdef AMG_CHECKED
// read and clear the bounds flag of this translation unit's kernels
static int take_bounds_flag() {
  int b = 0, z = 0;
  cudaMemcpyFromSymbol(&b, g_amg_bounds, sizeof(int));
  if (b) cudaMemcpyToSymbol(g_amg_bounds, &z, sizeof(int));
  return b;
}
#endif

// error bits raised by bounded device waits during the solve phase
static amg_status check_device_flags(amg_handle* h) {
  int f = 0;
  AMG_CK(h, cudaMemcpyAsync(&f, h->dev_flags, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  AMG_CK(h, cudaStreamSynchronize(h->stream));
#ifdef AMG_CHECKED
  if (take_bounds_flag()) return amg_fail(h, AMG_ERR_CUDA, "bounds check: a gather index was out of range");
#endif
  if (!f) return AMG_OK;
  AMG_CK(h, cudaMemsetAsync(h->dev_flags, 0, sizeof(int), h->stream));
  if (f & ST_TIMEOUT) {
    pair_reset(h);  // the paired-pass counters of an interrupted launch are behind
    return amg_fail(h, AMG_ERR_TIMEOUT, "a bounded wait of a row kernel expired");
  }
  return amg_fail(h, AMG_ERR_CUDA, "device error flags %d", f);
}

static amg_status ensure_hist(amg_handle* h, int maxit) {
  if (maxit + 1 <= h->hist_cap) return AMG_OK;
  if (h->hist) amg_release(h, h->hist);
  AMG_ALLOC(h, h->hist, double, (size_t)maxit + 1);
  h->hist_cap = maxit + 1;
  return AMG_OK;
}

static amg_status run_fcg(amg_handle* h, bool precond, double tol, int maxit, int32_t* iters, double* res_hist,
                          double* true_rel_res) {
  cudaStream_t s = h->stream;
  Level& L = h->L[0];
  const int n = L.n;
  if (maxit < 0) return amg_fail(h, AMG_ERR_INVALID_ARG, "maxit must be >= 0");
  if (!(tol >= 0.0)) return amg_fail(h, AMG_ERR_INVALID_ARG, "tol must be >= 0");
  amg_status st = ensure_hist(h, maxit);
  if (st != AMG_OK) return st;
  FcgState* hs = h->st_host;
  memset(hs, 0, sizeof(FcgState));
  hs->maxit = maxit;
  hs->tol = tol;
  hs->mixed = (h->p.precision != AMG_FP64) && precond;
  hs->true_every = h->p.true_res_every;
  hs->precflag = precond ? 1 : 0;
  hs->hist = h->hist;
  hs->hist_len = maxit + 1;
  AMG_CK(h, cudaMemcpyAsync(h->st, hs, sizeof(FcgState), cudaMemcpyHostToDevice, s));
  const int g = h->red_grid;
  launch_fcg_resid<RES_INIT>(h, s);
  AMG_CK(h, cudaGetLastError());
  int launches = 1;
  AMG_CK(h, cudaMemcpyAsync(hs, h->st, sizeof(FcgState), cudaMemcpyDeviceToHost, s));
  AMG_CK(h, cudaStreamSynchronize(s));
  if (hs->nb == 0.0) AMG_CK(h, cudaMemsetAsync(h->u, 0, sizeof(double) * (size_t)n, s));
  // Convergence reads: the first after graph_batch iterations, each later one
  // after as many iterations as the convergence factor observed since the
  // previous read predicts are still needed (at most 64, and not past maxit).
  // Iterations launched after the stop return at once but still cost their
  // launches; a short prediction only costs one more read.  graph_batch = 1
  // reads after every iteration.  The iterations themselves do not depend on
  // this spacing.
  int batch = std::max(1, h->p.graph_batch);
  double res_prev = hs->res;
  int it_prev = hs->it;
  while (!hs->done) {
    for (int j = 0; j < batch; ++j) {
      if (h->p.use_graph) {
        AMG_CK(h, cudaGraphLaunch(precond ? h->g_iter : h->g_iter_cg, s));
      } else {
        VRec R{h, s, &h->st->done};
        record_iteration(R, precond);
        AMG_CK(h, cudaGetLastError());
      }
      launches += precond ? h->launches_iter : h->launches_iter_cg;
    }
    AMG_CK(h, cudaMemcpyAsync(hs, h->st, sizeof(FcgState), cudaMemcpyDeviceToHost, s));
    AMG_CK(h, cudaStreamSynchronize(s));
    if (hs->done || h->p.graph_batch <= 1) continue;
    const int did = hs->it - it_prev;
    double need = (double)h->p.graph_batch;
    if (did > 0 && hs->res > 0.0 && hs->res < res_prev) {
      const double rate = std::pow(hs->res / res_prev, 1.0 / did);  // per iteration, in (0, 1)
      need = tol > 0.0 ? std::ceil(std::log(tol / hs->res) / std::log(rate)) : 64.0;
    }
    batch = (int)std::max(1.0, std::min({need, 64.0, (double)(maxit - hs->it)}));
    res_prev = hs->res;
    it_prev = hs->it;
  }
  if (hs->status != AMG_OK && hs->nb > 0.0) {
    launch_fcg_resid<RES_NORM>(h, s);
    ++launches;
    AMG_CK(h, cudaMemcpyAsync(hs, h->st, sizeof(FcgState), cudaMemcpyDeviceToHost, s));
    AMG_CK(h, cudaStreamSynchronize(s));
  }
  h->launches_last_solve = launches;
  amg_status fl = check_device_flags(h);
  if (fl != AMG_OK) return fl;
  if (iters) *iters = hs->it;
  if (true_rel_res) *true_rel_res = hs->true_res;
  if (res_hist) {
    AMG_CK(h, cudaMemcpyAsync(res_hist, h->hist, sizeof(double) * (size_t)(hs->it + 1), cudaMemcpyDeviceToHost, s));
    AMG_CK(h, cudaStreamSynchronize(s));
  }
  return (amg_status)hs->status;
}

static amg_status solve_common(amg_handle* h, bool precond, const double* b, double* x, bool host, double tol,
                               int32_t maxit, int32_t* iters, double* res_hist, double* true_rel_res) {
  if (!h) return AMG_ERR_INVALID_ARG;
  if (!b || !x) return amg_fail(h, AMG_ERR_INVALID_ARG, "b and x must not be NULL");
  const size_t bytes = sizeof(double) * (size_t)h->L[0].n;
  cudaMemcpyKind in = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  cudaMemcpyKind outk = host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  AMG_CK(h, cudaMemcpyAsync(h->b, b, bytes, in, h->stream));
  AMG_CK(h, cudaMemcpyAsync(h->u, x, bytes, in, h->stream));
  amg_status st = run_fcg(h, precond, tol, maxit, iters, res_hist, true_rel_res);
  if (st < 0 && st != AMG_ERR_BREAKDOWN) return st;
  AMG_CK(h, cudaMemcpyAsync(x, h->u, bytes, outk, h->stream));
  AMG_CK(h, cudaStreamSynchronize(h->stream));
  return st;
}

extern "C" amg_status amg_pcg_solve(amg_handle* h, const double* b, double* x, double tol, int32_t maxit,
                                    int32_t* iters, double* res_hist, double* true_rel_res) {
  return solve_common(h, true, b, x, false, tol, maxit, iters, res_hist, true_rel_res);
}

extern "C" amg_status amg_pcg_solve_host(amg_handle* h, const double* b, double* x, double tol, int32_t maxit,
                                         int32_t* iters, double* res_hist, double* true_rel_res) {
  return solve_common(h, true, b, x, true, tol, maxit, iters, res_hist, true_rel_res);
}

extern "C" amg_status amg_cg_solve(amg_handle* h, const double* b, double* x, double tol, int32_t maxit,
                                   int32_t* iters, double* res_hist, double* true_rel_res) {
  return solve_common(h, false, b, x, false, tol, maxit, iters, res_hist, true_rel_res);
}

static amg_status vcycle_on_handle(amg_handle* h) {
  if (h->p.use_graph) {
    AMG_CK(h, cudaGraphLaunch(h->g_vcycle, h->stream));
  } else {
    VRec R{h, h->stream, h->zero_flag};
    record_vcycle(R, h->r, h->w);
  }
  AMG_CK(h, cudaGetLastError());
  return AMG_OK;
}

extern "C" amg_status amg_vcycle(amg_handle* h, const double* r, double* z) {
  if (!h) return AMG_ERR_INVALID_ARG;
  if (!r || !z) return amg_fail(h, AMG_ERR_INVALID_ARG, "r and z must not be NULL");
  const size_t bytes = sizeof(double) * (size_t)h->L[0].n;
  AMG_CK(h, cudaMemcpyAsync(h->r, r, bytes, cudaMemcpyDeviceToDevice, h->stream));
  amg_status st = vcycle_on_handle(h);
  if (st != AMG_OK) return st;
  AMG_CK(h, cudaMemcpyAsync(z, h->w, bytes, cudaMemcpyDeviceToDevice, h->stream));
  AMG_CK(h, cudaStreamSynchronize(h->stream));
  return check_device_flags(h);
}

extern "C" amg_status amg_spmv(amg_handle* h, int32_t level, const double* x, double* y) {
  if (!h) return AMG_ERR_INVALID_ARG;
  if (level < 0 || level >= h->nl || !x || !y) return amg_fail(h, AMG_ERR_INVALID_ARG, "bad level or pointer");
  Level& L = h->L[level];
  const int nb = (L.n + L.Rd - 1) / L.Rd;
  DISPATCH_R(L.Rd, (k_spmv<TR><<<nb, TR, 0, h->stream>>>(L.n, L.rp, L.ci, L.v, x, y)));
  AMG_CK(h, cudaGetLastError());
  AMG_CK(h, cudaStreamSynchronize(h->stream));
  return AMG_OK;
}

// ---------------------------------------------------------------------------
// measurement helpers

extern "C" amg_status amg_time_vcycle(amg_handle* h, int32_t reps, double* ms) {
  if (!h || !ms || reps <= 0) return AMG_ERR_INVALID_ARG;
  cudaEvent_t e0, e1;
  AMG_CK(h, cudaEventCreate(&e0));
  AMG_CK(h, cudaEventCreate(&e1));
  amg_status st = vcycle_on_handle(h);  // warm-up
  if (st != AMG_OK) return st;
  AMG_CK(h, cudaEventRecord(e0, h->stream));
  for (int i = 0; i < reps; ++i) {
    st = vcycle_on_handle(h);
    if (st != AMG_OK) return st;
  }
  AMG_CK(h, cudaEventRecord(e1, h->stream));
  AMG_CK(h, cudaEventSynchronize(e1));
  float t = 0.f;
  AMG_CK(h, cudaEventElapsedTime(&t, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = (double)t / reps;
  return AMG_OK;
}

// launches one kernel of the solve phase on the level's own buffers
static amg_status launch_one(amg_handle* h, int which, int k) {
  Level& L = h->L[k];
  cudaStream_t s = h->stream;
  const int* skip = h->zero_flag;
  const int g = h->red_grid;
  const bool coarsest = (k == h->nl - 1);
  switch (which) {
    case 0:  // sweep
    case 1:  // residual
      if (!L.lowp) {
        const double* r = k == 0 ? h->r : (const double*)L.r;
        if (which == 0) launch_sweep<double, double, double>(s, L, L.v, L.dinv, r, (double*)L.za, (double*)L.zb, skip, h->dev_flags);
        else launch_resid<double, double>(s, L, L.v, r, (double*)L.za, (double*)L.t, skip, h->dev_flags);
      } else {
        const float* r = k == 0 ? L.r0f : (const float*)L.r;
        if (L.vb) {
          if (which == 0) launch_sweep<bf16, float, float>(s, L, L.vb, L.dinvf, r, (float*)L.za, (float*)L.zb, skip, h->dev_flags);
          else launch_resid<bf16, float>(s, L, L.vb, r, (float*)L.za, (float*)L.t, skip, h->dev_flags);
        } else {
          if (which == 0) launch_sweep<float, float, float>(s, L, L.vf, L.dinvf, r, (float*)L.za, (float*)L.zb, skip, h->dev_flags);
          else launch_resid<float, float>(s, L, L.vf, r, (float*)L.za, (float*)L.t, skip, h->dev_flags);
        }
      }
      break;
    case 2:
    case 3: {
      if (coarsest) return amg_fail(h, AMG_ERR_INVALID_ARG, "no restriction/prolongation on the coarsest level");
      Level& C = h->L[k + 1];
      bool ccoarse = (k + 1 == h->nl - 1);
      if (which == 2) {
        if (!L.lowp) amg_launch(k_restrict<double, double>, dim3(amg_blocks(C.n)), dim3(AMG_BLOCK), 0, s, C.n, L.mptr, L.mem, (double*)L.t, (double*)C.r, skip, L.n, L.pwm);
        else if (ccoarse) amg_launch(k_restrict<float, double>, dim3(amg_blocks(C.n)), dim3(AMG_BLOCK), 0, s, C.n, L.mptr, L.mem, (float*)L.t, (double*)C.r, skip, L.n, L.pwmf);
        else amg_launch(k_restrict<float, float>, dim3(amg_blocks(C.n)), dim3(AMG_BLOCK), 0, s, C.n, L.mptr, L.mem, (float*)L.t, (float*)C.r, skip, L.n, L.pwmf);
      } else {
        if (!L.lowp) amg_launch(k_prolong<double, double>, dim3(ew_blocks(L.n)), dim3(AMG_BLOCK), 0, s, L.n, L.agg, (double*)C.za, (double*)L.za, skip, C.n, L.pw);
        else if (ccoarse) amg_launch(k_prolong<float, double>, dim3(ew_blocks(L.n)), dim3(AMG_BLOCK), 0, s, L.n, L.agg, (double*)C.za, (float*)L.za, skip, C.n, L.pwf);
        else amg_launch(k_prolong<float, float>, dim3(ew_blocks(L.n)), dim3(AMG_BLOCK), 0, s, L.n, L.agg, (float*)C.za, (float*)L.za, skip, C.n, L.pwf);
      }
      break;
    }
    case 6:
    case 7: {
      if (coarsest) return amg_fail(h, AMG_ERR_INVALID_ARG, "no restriction/prolongation on the coarsest level");
      Level& C = h->L[k + 1];
      const bool ccoarse = (k + 1 == h->nl - 1);
      if (which == 6) {
        if (ccoarse && !L.lowp)
          amg_launch(k_restrict_first<double, double>, dim3(amg_blocks(C.n)), dim3(AMG_BLOCK), 0, s, C.n, L.mptr, L.mem,
                     (const double*)L.t, (const double*)C.dinv, (double*)C.r, (double*)C.za, skip, L.n, L.pwm);
        else if (ccoarse)
          amg_launch(k_restrict_first<float, double>, dim3(amg_blocks(C.n)), dim3(AMG_BLOCK), 0, s, C.n, L.mptr, L.mem,
                     (const float*)L.t, (const double*)C.dinv, (double*)C.r, (double*)C.za, skip, L.n, L.pwmf);
        else if (!L.lowp)
          amg_launch(k_restrict_first<double, double>, dim3(amg_blocks(C.n)), dim3(AMG_BLOCK), 0, s, C.n, L.mptr, L.mem,
                     (const double*)L.t, (const double*)C.dinv, (double*)C.r, (double*)C.za, skip, L.n, L.pwm);
        else
          amg_launch(k_restrict_first<float, float>, dim3(amg_blocks(C.n)), dim3(AMG_BLOCK), 0, s, C.n, L.mptr, L.mem,
                     (const float*)L.t, (const float*)C.dinvf, (float*)C.r, (float*)C.za, skip, L.n, L.pwmf);
      } else {
        bool ok;
        if (ccoarse || !C.lowp)
          ok = launch_sweep_prolong<double, double>(s, C, C.v, C.dinv, (const double*)C.r, (const double*)C.za,
                                                    (double*)C.zb, skip, h->dev_flags, L, L.za, true);
        else
          ok = launch_sweep_prolong<float, float>(s, C, C.vf, C.dinvf, (const float*)C.r, (const float*)C.za,
                                                  (float*)C.zb, skip, h->dev_flags, L, L.za, true);
        if (!ok) return amg_fail(h, AMG_ERR_INVALID_ARG, "level %d runs the non-pipelined kernels", k + 1);
      }
      break;
    }
    case 8: {  // two sweeps in one launch (za -> zb -> za)
      const double* r64 = k == 0 ? h->r : (const double*)L.r;
      bool ok;
      if (!L.lowp)
        ok = launch_pair<PM_SWEEP, double, double, double>(h, s, L, L.v, L.dinv, r64, (const double*)L.za, (double*)L.zb,
                                                           (double*)L.za, skip, true);
      else if (L.vb)
        ok = launch_pair<PM_SWEEP, bf16, float, float>(h, s, L, L.vb, L.dinvf, k == 0 ? L.r0f : (const float*)L.r,
                                                       (const float*)L.za, (float*)L.zb, (float*)L.za, skip, true);
      else
        ok = launch_pair<PM_SWEEP, float, float, float>(h, s, L, L.vf, L.dinvf, k == 0 ? L.r0f : (const float*)L.r,
                                                        (const float*)L.za, (float*)L.zb, (float*)L.za, skip, true);
      if (!ok) return amg_fail(h, AMG_ERR_INVALID_ARG, "level %d runs the non-pipelined kernels", k);
      break;
    }
    case 4:
      if (k != 0) return amg_fail(h, AMG_ERR_INVALID_ARG, "outer kernels run on level 0");
      launch_dots(h, s);
      break;
    case 5:
      if (k != 0) return amg_fail(h, AMG_ERR_INVALID_ARG, "outer kernels run on level 0");
      amg_launch(k_fcg_axpy, dim3(h->ax_grid), dim3(AMG_BLOCK), 0, s, L.n, h->w, h->v, h->d, h->q, h->u, h->r, h->st, h->partial, h->counter);
      break;
    default:
      return amg_fail(h, AMG_ERR_INVALID_ARG, "unknown kernel id %d", which);
  }
  AMG_CK(h, cudaGetLastError());
  return AMG_OK;
}

extern "C" amg_status amg_time_kernel(amg_handle* h, int32_t which, int32_t level, int32_t reps, double* ms) {
  if (!h || !ms || reps <= 0) return AMG_ERR_INVALID_ARG;
  if (level < 0 || level >= h->nl) return amg_fail(h, AMG_ERR_INVALID_ARG, "bad level");
  amg_status st = ensure_hist(h, 1);
  if (st != AMG_OK) return st;
  if (which >= 4) {  // the outer kernels need a live (not done) FCG state with it > 0
    FcgState* hs = h->st_host;
    memset(hs, 0, sizeof(FcgState));
    hs->it = 1;
    hs->timing = 1;
    hs->maxit = 1 << 30;
    hs->tol = 0.0;
    hs->nb = 1.0;
    hs->rho = 1.0;
    AMG_CK(h, cudaMemcpyAsync(h->st, hs, sizeof(FcgState), cudaMemcpyHostToDevice, h->stream));
  }
  cudaEvent_t e0, e1;
  AMG_CK(h, cudaEventCreate(&e0));
  AMG_CK(h, cudaEventCreate(&e1));
  st = launch_one(h, which, level);
  if (st != AMG_OK) return st;
  AMG_CK(h, cudaEventRecord(e0, h->stream));
  for (int i = 0; i < reps; ++i) {
    st = launch_one(h, which, level);
    if (st != AMG_OK) return st;
  }
  AMG_CK(h, cudaEventRecord(e1, h->stream));
  AMG_CK(h, cudaEventSynchronize(e1));
  float t = 0.f;
  AMG_CK(h, cudaEventElapsedTime(&t, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = (double)t / reps;
  return AMG_OK;
}
