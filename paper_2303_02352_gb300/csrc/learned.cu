// Learned l1-Jacobi damping and the adjoint of the V-cycle.
//
// A small network maps per-row features of each hierarchy level to a damping
// omega_i in (0, 2) that multiplies the l1-Jacobi diagonal, D_i = omega_i / M_ii
// (M_ii = sum_j |a_ij|, Sec. 3.1).  The network is 4 -> 32 -> 32 -> 1 with ReLU
// and omega = 2 sigmoid(out); weights are stored in bf16, arithmetic is float32.
// It is trained through the adjoint of the V-cycle (Alg. 2 / operator B^k of
// Sec. 3.1): reverse-mode differentiation of the FP64 V-cycle with respect to
// its input r and to every omega, recomputing each level's sweep iterates from
// the level's stored input instead of storing every sweep.
//
// Parameter layout: [W1 (32x4, row-major), b1 (32), W2 (32x32), b2 (32), W3 (32), b3].
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "amg_internal.cuh"

#define MLP_NP 1249
#define OFF_W1 0
#define OFF_B1 128
#define OFF_W2 160
#define OFF_B2 1184
#define OFF_W3 1216
#define OFF_B3 1248
#define MLP_BLOCK 256

// ---------------------------------------------------------------------------
// row features of a level:
//   f0 = a_ii / l1_i, f1 = ln l1_i - mean_{j in row i} ln l1_j,
//   f2 = nnz_i / 27,  f3 = level / 4

__global__ void k_features(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const double* __restrict__ v, const double* __restrict__ l1, float level,
                           float* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int p0 = rp[i], p1 = rp[i + 1];
  double d = 0.0, sl = 0.0;
  for (int p = p0; p < p1; ++p) {
    const int j = ci[p];
    if (j == i) d = v[p];
    sl += log(l1[j]);
  }
  const double li = l1[i];
  out[4 * (size_t)i + 0] = (float)(d / li);
  out[4 * (size_t)i + 1] = (float)(log(li) - sl / (double)(p1 - p0));
  out[4 * (size_t)i + 2] = (float)((double)(p1 - p0) / 27.0);
  out[4 * (size_t)i + 3] = level / 4.0f;
}

// ---------------------------------------------------------------------------
// network forward: omega_i (double) from the features of row i

__device__ __forceinline__ void load_weights(float* W, const bf16* __restrict__ w) {
  for (int p = threadIdx.x; p < MLP_NP; p += blockDim.x) W[p] = __bfloat162float(w[p]);
  __syncthreads();
}

__global__ void __launch_bounds__(MLP_BLOCK) k_mlp_fwd(int n, const float* __restrict__ f, const bf16* __restrict__ w,
                                                       double* __restrict__ omega) {
  __shared__ float W[MLP_NP];
  load_weights(W, w);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float x0 = f[4 * (size_t)i], x1 = f[4 * (size_t)i + 1], x2 = f[4 * (size_t)i + 2], x3 = f[4 * (size_t)i + 3];
  float h1[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    float a = W[OFF_B1 + j];
    a += W[OFF_W1 + 4 * j + 0] * x0;
    a += W[OFF_W1 + 4 * j + 1] * x1;
    a += W[OFF_W1 + 4 * j + 2] * x2;
    a += W[OFF_W1 + 4 * j + 3] * x3;
    h1[j] = fmaxf(a, 0.0f);
  }
  float o = W[OFF_B3];
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    float a = W[OFF_B2 + j];
#pragma unroll
    for (int k = 0; k < 32; ++k) a += W[OFF_W2 + 32 * j + k] * h1[k];
    o += W[OFF_W3 + j] * fmaxf(a, 0.0f);
  }
  omega[i] = (double)(2.0f / (1.0f + expf(-o)));
}

// ---------------------------------------------------------------------------
// network backward: per block of MLPB_ROWS rows, phase 1 (one thread per row)
// stores the row's input, activations and deltas in shared memory; phase 2
// (one thread per parameter) sums the parameter's gradient over the block's
// rows in row order.  A second kernel sums the block partials in block order.
// Deterministic.

#define MLPB_ROWS 128
#define MLPB_LD (MLPB_ROWS + 1)  // padded row stride: conflict-free column reads

struct MlpBwdSmem {
  float W[MLP_NP];
  float X[4][MLPB_LD];
  float H1[32][MLPB_LD];
  float H2[32][MLPB_LD];
  float DH1[32][MLPB_LD];
  float DH2[32][MLPB_LD];
  float D[MLPB_LD];
};

__global__ void __launch_bounds__(MLPB_ROWS) k_mlp_bwd(int n, const float* __restrict__ f, const bf16* __restrict__ w,
                                                       const double* __restrict__ domega, float* __restrict__ ws) {
  extern __shared__ __align__(16) unsigned char mlp_smem[];
  MlpBwdSmem& S = *reinterpret_cast<MlpBwdSmem*>(mlp_smem);
  load_weights(S.W, w);
  const float* W = S.W;
  const int r = threadIdx.x;
  const int i = blockIdx.x * MLPB_ROWS + r;
  const bool live = i < n;
  float x[4] = {0.f, 0.f, 0.f, 0.f};
  if (live)
#pragma unroll
    for (int k = 0; k < 4; ++k) x[k] = f[4 * (size_t)i + k];
#pragma unroll
  for (int k = 0; k < 4; ++k) S.X[k][r] = x[k];
  float h1[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    float a = W[OFF_B1 + j];
#pragma unroll
    for (int k = 0; k < 4; ++k) a += W[OFF_W1 + 4 * j + k] * x[k];
    h1[j] = fmaxf(a, 0.0f);
    S.H1[j][r] = h1[j];
  }
  float o = W[OFF_B3];
#pragma unroll 4
  for (int j = 0; j < 32; ++j) {
    float a = W[OFF_B2 + j];
#pragma unroll
    for (int k = 0; k < 32; ++k) a += W[OFF_W2 + 32 * j + k] * h1[k];
    const float h2 = fmaxf(a, 0.0f);
    S.H2[j][r] = h2;
    o += W[OFF_W3 + j] * h2;
  }
  float dout = 0.0f;
  if (live) {
    const float sg = 1.0f / (1.0f + expf(-o));
    dout = (float)domega[i] * 2.0f * sg * (1.0f - sg);
  }
  S.D[r] = dout;
#pragma unroll 4
  for (int j = 0; j < 32; ++j) S.DH2[j][r] = S.H2[j][r] > 0.0f ? dout * W[OFF_W3 + j] : 0.0f;
#pragma unroll 4
  for (int k = 0; k < 32; ++k) {
    float sacc = 0.0f;
#pragma unroll
    for (int j = 0; j < 32; ++j) sacc += W[OFF_W2 + 32 * j + k] * S.DH2[j][r];
    S.DH1[k][r] = h1[k] > 0.0f ? sacc : 0.0f;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < MLP_NP; p += MLPB_ROWS) {
    const float* a;
    const float* b = nullptr;
    if (p < OFF_B1) {
      a = S.DH1[(p - OFF_W1) >> 2];
      b = S.X[(p - OFF_W1) & 3];
    } else if (p < OFF_W2) {
      a = S.DH1[p - OFF_B1];
    } else if (p < OFF_B2) {
      a = S.DH2[(p - OFF_W2) >> 5];
      b = S.H1[(p - OFF_W2) & 31];
    } else if (p < OFF_W3) {
      a = S.DH2[p - OFF_B2];
    } else if (p < OFF_B3) {
      a = S.D;
      b = S.H2[p - OFF_W3];
    } else {
      a = S.D;
    }
    float acc = 0.0f;
    if (b)
      for (int q = 0; q < MLPB_ROWS; ++q) acc += a[q] * b[q];
    else
      for (int q = 0; q < MLPB_ROWS; ++q) acc += a[q];
    ws[(size_t)blockIdx.x * MLP_NP + p] = acc;
  }
}

__global__ void k_mlp_bwd_final(int nblocks, const float* __restrict__ ws, float* __restrict__ grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= MLP_NP) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += (double)ws[(size_t)b * MLP_NP + p];
  grad[p] = (float)s;
}

// Adam on the float32 master weights; writes the bf16 copy the network uses
__global__ void k_adam(int np, float* __restrict__ theta, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, bf16* __restrict__ wbf, float lr, float b1, float b2, float eps,
                       float bc1, float bc2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const float gp = g[p];
  const float mp = b1 * m[p] + (1.0f - b1) * gp;
  const float vp = b2 * v[p] + (1.0f - b2) * gp * gp;
  m[p] = mp;
  v[p] = vp;
  const float t = theta[p] - lr * (mp / bc1) / (sqrtf(vp / bc2) + eps);
  theta[p] = t;
  wbf[p] = __float2bfloat16_rn(t);
}

// omega -> D = omega / l1 (FP64 and, for low-precision levels, FP32)
__global__ void k_set_omega(int n, const double* __restrict__ om_in, double* __restrict__ om,
                            const double* __restrict__ l1, double* __restrict__ dinv, float* __restrict__ dinvf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double o = om_in ? om_in[i] : 1.0;
  om[i] = o;
  const double d = o / l1[i];
  dinv[i] = d;
  if (dinvf) dinvf[i] = __double2float_rn(d);
}

// ---------------------------------------------------------------------------
// FP64 V-cycle with recording, and its adjoint (simple thread-per-row kernels)

__global__ void k_ad_first(int n, const double* __restrict__ dinv, const double* __restrict__ r, double* __restrict__ z) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] = dinv[i] * r[i];
}

__global__ void k_ad_sweep(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const double* __restrict__ v, const double* __restrict__ dinv, const double* __restrict__ r,
                           const double* __restrict__ z, double* __restrict__ zout) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) s += v[p] * z[ci[p]];
  zout[i] = z[i] + dinv[i] * (r[i] - s);
}

__global__ void k_ad_resid(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const double* __restrict__ v, const double* __restrict__ r, const double* __restrict__ z,
                           double* __restrict__ t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) s += v[p] * z[ci[p]];
  t[i] = r[i] - s;
}

// out[J] = sum over the members of aggregate J of t (P^T t)
__global__ void k_ad_restrict(int nc, const int32_t* __restrict__ mptr, const int32_t* __restrict__ mem,
                              const double* __restrict__ t, double* __restrict__ out) {
  const int J = blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= nc) return;
  double s = 0.0;
  for (int m = mptr[J]; m < mptr[J + 1]; ++m) s += t[mem[m]];
  out[J] = s;
}

// out = z + P zc
__global__ void k_ad_prolong(int n, const int32_t* __restrict__ agg, const double* __restrict__ z,
                             const double* __restrict__ zc, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = z[i] + zc[agg[i]];
}

// adjoint of z' = z + D (r - A z) with input iterate zold:
//   domega_i += lam_i (r - A zold)_i / l1_i,  lr += D lam,  lam_out = lam - A^T (D lam)
// (A is symmetric, so A^T (D lam) is a row pass over A)
__global__ void k_adj_sweep(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                            const double* __restrict__ v, const double* __restrict__ dinv, const double* __restrict__ l1,
                            const double* __restrict__ r, const double* __restrict__ zold,
                            const double* __restrict__ lam, double* __restrict__ lam_out, double* __restrict__ lr,
                            double* __restrict__ dom) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s1 = 0.0, s2 = 0.0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    const int j = ci[p];
    s1 += v[p] * zold[j];
    s2 += v[p] * (dinv[j] * lam[j]);
  }
  const double t = r[i] - s1, li = lam[i];
  dom[i] += li * t / l1[i];
  lr[i] += dinv[i] * li;
  lam_out[i] = li - s2;
}

// adjoint of the first sweep from zero, z = D r
__global__ void k_adj_first(int n, const double* __restrict__ dinv, const double* __restrict__ l1,
                            const double* __restrict__ r, const double* __restrict__ lam, double* __restrict__ lr,
                            double* __restrict__ dom) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  dom[i] += lam[i] * r[i] / l1[i];
  lr[i] += dinv[i] * lam[i];
}

// adjoint of r_c = P^T (r - A z): with lam_res = P lam_rc,
//   lr += lam_res,  lam_out = lam - A^T lam_res
__global__ void k_adj_restrict(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                               const double* __restrict__ v, const int32_t* __restrict__ agg,
                               const double* __restrict__ lrc, const double* __restrict__ lam,
                               double* __restrict__ lam_out, double* __restrict__ lr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) s += v[p] * lrc[agg[ci[p]]];
  lr[i] += lrc[agg[i]];
  lam_out[i] = lam[i] - s;
}

struct AdjLevel {
  double* rin = nullptr;   // level input (levels > 0)
  double* zpre = nullptr;  // after pre-smoothing
  double* y0 = nullptr;    // start of post-smoothing (zpre + P z_c)
  double* zout = nullptr;  // level output (levels > 0)
  double* t = nullptr;     // residual
  double* lamA = nullptr;
  double* lamB = nullptr;
  double* lr = nullptr;    // dL / d rin
  double* lamc = nullptr;  // dL / d z_c (input of the coarser level's adjoint)
  std::vector<double*> it; // recomputed sweep iterates
};

struct AdjState {
  AdjLevel L[AMG_MAXL];
  std::vector<double*> rs;  // residuals r_0 .. r_m of the stationary loss
  double* lam_r = nullptr;  // dL / d r_t
  double* lam_z = nullptr;  // dL / d z_t
  double* scal = nullptr;   // two device doubles: |r|^2 results
};

void amg_adj_destroy(amg_handle* h) {
  delete h->adj;
  h->adj = nullptr;
}

static amg_status adj_prepare(amg_handle* h) {
  if (h->adj) return AMG_OK;
  h->adj = new AdjState();
  for (int k = 0; k < h->nl; ++k) {
    const int n = h->L[k].n;
    AdjLevel& A = h->adj->L[k];
    AMG_ALLOC(h, A.zpre, double, n);
    AMG_ALLOC(h, A.y0, double, n);
    AMG_ALLOC(h, A.t, double, n);
    AMG_ALLOC(h, A.lamA, double, n);
    AMG_ALLOC(h, A.lamB, double, n);
    AMG_ALLOC(h, A.lr, double, n);
    AMG_ALLOC(h, A.lamc, double, n);
    if (k > 0) {
      AMG_ALLOC(h, A.rin, double, n);
      AMG_ALLOC(h, A.zout, double, n);
    }
    const bool coarsest = k == h->nl - 1;
    int ns = coarsest ? h->p.coarse_sweeps : std::max(h->p.pre_sweeps, h->p.post_sweeps);
    ns = std::max(ns, 1);
    A.it.assign(ns, nullptr);
    for (int s = 0; s < ns; ++s) AMG_ALLOC(h, A.it[s], double, n);
  }
  AMG_CK(h, cudaStreamSynchronize(h->stream));
  return AMG_OK;
}

// sweeps from zstart (nullptr: from zero) on level k; writes the result to out
static void ad_smooth(amg_handle* h, int k, const double* r, const double* zstart, int sweeps, double* out) {
  const Level& L = h->L[k];
  cudaStream_t s = h->stream;
  const int nb = amg_blocks(L.n);
  if (sweeps <= 0) {
    if (zstart) cudaMemcpyAsync(out, zstart, sizeof(double) * L.n, cudaMemcpyDeviceToDevice, s);
    else cudaMemsetAsync(out, 0, sizeof(double) * L.n, s);
    return;
  }
  AdjLevel& A = h->adj->L[k];
  // iterate buffers: it[s] holds the input of sweep s
  const double* cur = zstart;
  for (int sw = 0; sw < sweeps; ++sw) {
    double* nxt = (sw == sweeps - 1) ? out : A.it[sw + 1 < (int)A.it.size() ? sw + 1 : 0];
    if (!cur) k_ad_first<<<nb, AMG_BLOCK, 0, s>>>(L.n, L.dinv, r, nxt);
    else k_ad_sweep<<<nb, AMG_BLOCK, 0, s>>>(L.n, L.rp, L.ci, L.v, L.dinv, r, cur, nxt);
    cur = nxt;
  }
}

// forward FP64 V-cycle from level k with recording
static void ad_forward(amg_handle* h, int k, const double* r, double* out) {
  const Level& L = h->L[k];
  AdjLevel& A = h->adj->L[k];
  cudaStream_t s = h->stream;
  if (k == h->nl - 1) {
    ad_smooth(h, k, r, nullptr, h->p.coarse_sweeps, out);
    return;
  }
  const Level& C = h->L[k + 1];
  AdjLevel& AC = h->adj->L[k + 1];
  ad_smooth(h, k, r, nullptr, h->p.pre_sweeps, A.zpre);
  k_ad_resid<<<amg_blocks(L.n), AMG_BLOCK, 0, s>>>(L.n, L.rp, L.ci, L.v, r, A.zpre, A.t);
  k_ad_restrict<<<amg_blocks(C.n), AMG_BLOCK, 0, s>>>(C.n, L.mptr, L.mem, A.t, AC.rin);
  ad_forward(h, k + 1, AC.rin, AC.zout);
  k_ad_prolong<<<amg_blocks(L.n), AMG_BLOCK, 0, s>>>(L.n, L.agg, A.zpre, AC.zout, A.y0);
  ad_smooth(h, k, r, A.y0, h->p.post_sweeps, out);
}

// adjoint of `sweeps` sweeps from zstart on level k: lam (dL/dz_final) is
// consumed; lr and dom accumulate.  Returns the buffer holding dL/dz_start.
static double* ad_smooth_adj(amg_handle* h, int k, const double* r, const double* zstart, int sweeps, double* lam,
                             double* lr, double* dom) {
  const Level& L = h->L[k];
  AdjLevel& A = h->adj->L[k];
  cudaStream_t s = h->stream;
  const int nb = amg_blocks(L.n);
  if (sweeps <= 0) return lam;
  // recompute the inputs of every sweep: it[0] = zstart (or zero), it[s] = sweep(it[s-1])
  if (zstart) cudaMemcpyAsync(A.it[0], zstart, sizeof(double) * L.n, cudaMemcpyDeviceToDevice, s);
  for (int sw = 1; sw < sweeps; ++sw) {
    if (sw == 1 && !zstart) k_ad_first<<<nb, AMG_BLOCK, 0, s>>>(L.n, L.dinv, r, A.it[1]);
    else k_ad_sweep<<<nb, AMG_BLOCK, 0, s>>>(L.n, L.rp, L.ci, L.v, L.dinv, r, A.it[sw - 1], A.it[sw]);
  }
  double* cur = lam;
  double* other = (lam == A.lamA) ? A.lamB : A.lamA;
  for (int sw = sweeps - 1; sw >= 0; --sw) {
    if (sw == 0 && !zstart) {
      k_adj_first<<<nb, AMG_BLOCK, 0, s>>>(L.n, L.dinv, L.l1, r, cur, lr, dom);
    } else {
      k_adj_sweep<<<nb, AMG_BLOCK, 0, s>>>(L.n, L.rp, L.ci, L.v, L.dinv, L.l1, r, A.it[sw], cur, other, lr, dom);
      std::swap(cur, other);
    }
  }
  return cur;
}

// adjoint of the V-cycle at level k: lam = dL/d(output) (a lamA/lamB buffer of
// the level, consumed); writes dL/dr into A.lr; dom[k..] accumulate
static void ad_backward(amg_handle* h, int k, const double* r, double* lam, double* const* dom) {
  const Level& L = h->L[k];
  AdjLevel& A = h->adj->L[k];
  cudaStream_t s = h->stream;
  cudaMemsetAsync(A.lr, 0, sizeof(double) * L.n, s);
  if (k == h->nl - 1) {
    ad_smooth_adj(h, k, r, nullptr, h->p.coarse_sweeps, lam, A.lr, dom[k]);
    return;
  }
  const Level& C = h->L[k + 1];
  AdjLevel& AC = h->adj->L[k + 1];
  // post-smoothing from y0
  double* ly0 = ad_smooth_adj(h, k, r, A.y0, h->p.post_sweeps, lam, A.lr, dom[k]);
  // y0 = zpre + P z_c:  dL/dz_c = P^T dL/dy0 (into the coarse level's lamA)
  k_ad_restrict<<<amg_blocks(C.n), AMG_BLOCK, 0, s>>>(C.n, L.mptr, L.mem, ly0, AC.lamA);
  ad_backward(h, k + 1, AC.rin, AC.lamA, dom);
  // r_c = P^T (r - A zpre)
  double* lzp = (ly0 == A.lamA) ? A.lamB : A.lamA;
  k_adj_restrict<<<amg_blocks(L.n), AMG_BLOCK, 0, s>>>(L.n, L.rp, L.ci, L.v, L.agg, AC.lr, ly0, lzp, A.lr);
  // pre-smoothing from zero
  ad_smooth_adj(h, k, r, nullptr, h->p.pre_sweeps, lzp, A.lr, dom[k]);
}

// ---------------------------------------------------------------------------
// training loss of the damping: m steps of the stationary iteration
// r_{t+1} = r_t - A B(omega) r_t on level 0, L = (1/m) ln(|r_m| / |r_0|)

// out = r - A z (the product summed first, then subtracted)
__global__ void k_loss_step(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                            const double* __restrict__ v, const double* __restrict__ r, const double* __restrict__ z,
                            double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) s += v[p] * z[ci[p]];
  out[i] = r[i] - s;
}

// out = -A x
__global__ void k_neg_spmv(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const double* __restrict__ v, const double* __restrict__ x, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int p = rp[i]; p < rp[i + 1]; ++p) s += v[p] * x[ci[p]];
  out[i] = -s;
}

// *out = |x|^2 (deterministic: per-block partials in a fixed order)
__global__ void __launch_bounds__(AMG_BLOCK) k_sqnorm(int n, const double* __restrict__ x, double* partial,
                                                      unsigned* counter, double* out) {
  __shared__ double red[32];
  double acc[1] = {0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) acc[0] += x[i] * x[i];
  if (grid_sum<1>(acc, partial, counter, red) && threadIdx.x == 0) *out = acc[0];
}

__global__ void k_scale_into(int n, const double* __restrict__ x, double a, double* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = a * x[i];
}

__global__ void k_add_into(int n, const double* __restrict__ x, double* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += x[i];
}

static amg_status sqnorm(amg_handle* h, const double* x, double* out_dev) {
  const int n = h->L[0].n;
  const int grid = std::max(1, std::min(h->ax_grid, amg_blocks(n)));
  k_sqnorm<<<grid, AMG_BLOCK, 0, h->stream>>>(n, x, h->partial, h->counter, out_dev);
  AMG_CK(h, cudaGetLastError());
  return AMG_OK;
}

// ---------------------------------------------------------------------------
// C ABI

extern "C" amg_status amg_features(amg_handle* h, int32_t level, float* feats) {
  if (!h) return AMG_ERR_INVALID_ARG;
  if (level < 0 || level >= h->nl || !feats) return amg_fail(h, AMG_ERR_INVALID_ARG, "bad level or pointer");
  const Level& L = h->L[level];
  k_features<<<amg_blocks(L.n), AMG_BLOCK, 0, h->stream>>>(L.n, L.rp, L.ci, L.v, L.l1, (float)level, feats);
  AMG_CK(h, cudaGetLastError());
  AMG_CK(h, cudaStreamSynchronize(h->stream));
  return AMG_OK;
}

extern "C" amg_status amg_set_omega(amg_handle* h, int32_t level, const double* omega) {
  if (!h) return AMG_ERR_INVALID_ARG;
  if (level < 0 || level >= h->nl) return amg_fail(h, AMG_ERR_INVALID_ARG, "bad level %d", level);
  Level& L = h->L[level];
  if (!L.omega) AMG_ALLOC(h, L.omega, double, L.n);
  k_set_omega<<<amg_blocks(L.n), AMG_BLOCK, 0, h->stream>>>(L.n, omega, L.omega, L.l1, L.dinv, L.dinvf);
  AMG_CK(h, cudaGetLastError());
  AMG_CK(h, cudaStreamSynchronize(h->stream));
  return AMG_OK;
}

extern "C" size_t amg_mlp_workspace_bytes(int32_t n) {
  const size_t blocks = (size_t)((n + MLPB_ROWS - 1) / MLPB_ROWS);
  return blocks * MLP_NP * sizeof(float);
}

extern "C" amg_status amg_mlp_forward(int32_t n, const float* feats, const uint16_t* w_bf16, double* omega,
                                      void* stream) {
  if (n < 0 || (n > 0 && (!feats || !w_bf16 || !omega))) return AMG_ERR_INVALID_ARG;
  if (n == 0) return AMG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  k_mlp_fwd<<<(n + MLP_BLOCK - 1) / MLP_BLOCK, MLP_BLOCK, 0, s>>>(n, feats, (const bf16*)w_bf16, omega);
  return cudaGetLastError() == cudaSuccess ? AMG_OK : AMG_ERR_CUDA;
}

extern "C" amg_status amg_mlp_backward(int32_t n, const float* feats, const uint16_t* w_bf16, const double* domega,
                                       float* grad, void* workspace, void* stream) {
  if (n <= 0 || !feats || !w_bf16 || !domega || !grad || !workspace) return AMG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = (n + MLPB_ROWS - 1) / MLPB_ROWS;
  float* ws = (float*)workspace;
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(k_mlp_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MlpBwdSmem));
    configured = true;
  }
  k_mlp_bwd<<<blocks, MLPB_ROWS, sizeof(MlpBwdSmem), s>>>(n, feats, (const bf16*)w_bf16, domega, ws);
  k_mlp_bwd_final<<<(MLP_NP + 255) / 256, 256, 0, s>>>(blocks, ws, grad);
  return cudaGetLastError() == cudaSuccess ? AMG_OK : AMG_ERR_CUDA;
}

extern "C" amg_status amg_adam_step(int32_t np, float* theta, const float* grad, float* m, float* v,
                                    uint16_t* w_bf16, float lr, float beta1, float beta2, float eps, int32_t t,
                                    void* stream) {
  if (np <= 0 || !theta || !grad || !m || !v || !w_bf16 || t < 1) return AMG_ERR_INVALID_ARG;
  const float bc1 = 1.0f - powf(beta1, (float)t), bc2 = 1.0f - powf(beta2, (float)t);
  k_adam<<<(np + 255) / 256, 256, 0, (cudaStream_t)stream>>>(np, theta, grad, m, v, (bf16*)w_bf16, lr, beta1, beta2,
                                                            eps, bc1, bc2);
  return cudaGetLastError() == cudaSuccess ? AMG_OK : AMG_ERR_CUDA;
}

extern "C" amg_status amg_apply_mlp(amg_handle* h, const uint16_t* w_bf16) {
  if (!h) return AMG_ERR_INVALID_ARG;
  int nmax = 0;
  for (int k = 0; k < h->nl; ++k) nmax = std::max(nmax, h->L[k].n);
  float* feats;
  double* om;
  AMG_ALLOC(h, feats, float, 4 * (size_t)nmax);
  AMG_ALLOC(h, om, double, nmax);
  for (int k = 0; k < h->nl; ++k) {
    Level& L = h->L[k];
    if (!L.omega) AMG_ALLOC(h, L.omega, double, L.n);
    k_features<<<amg_blocks(L.n), AMG_BLOCK, 0, h->stream>>>(L.n, L.rp, L.ci, L.v, L.l1, (float)k, feats);
    if (w_bf16)
      k_mlp_fwd<<<(L.n + MLP_BLOCK - 1) / MLP_BLOCK, MLP_BLOCK, 0, h->stream>>>(L.n, feats, (const bf16*)w_bf16, om);
    k_set_omega<<<amg_blocks(L.n), AMG_BLOCK, 0, h->stream>>>(L.n, w_bf16 ? om : nullptr, L.omega, L.l1, L.dinv,
                                                              L.dinvf);
  }
  AMG_CK(h, cudaGetLastError());
  AMG_CK(h, cudaStreamSynchronize(h->stream));
  amg_release(h, feats);
  amg_release(h, om);
  return AMG_OK;
}

extern "C" amg_status amg_vcycle_backward(amg_handle* h, const double* r, const double* dz, double* dr,
                                          double* const* domega) {
  if (!h) return AMG_ERR_INVALID_ARG;
  if (!r || !dz || !dr || !domega) return amg_fail(h, AMG_ERR_INVALID_ARG, "NULL pointer");
  for (int k = 0; k < h->nl; ++k)
    if (!domega[k]) return amg_fail(h, AMG_ERR_INVALID_ARG, "domega[%d] is NULL", k);
  if (h->p.cycle != 0) return amg_fail(h, AMG_ERR_INVALID_ARG, "the adjoint covers the V-cycle only");
  if (h->p.relax_type != 4) return amg_fail(h, AMG_ERR_INVALID_ARG, "the adjoint covers l1-Jacobi only");
  if (h->p.prolong_scale != 0) return amg_fail(h, AMG_ERR_INVALID_ARG, "the adjoint covers unit prolongators only");
  amg_status st = adj_prepare(h);
  if (st != AMG_OK) return st;
  cudaStream_t s = h->stream;
  const int n = h->L[0].n;
  for (int k = 0; k < h->nl; ++k) AMG_CK(h, cudaMemsetAsync(domega[k], 0, sizeof(double) * h->L[k].n, s));
  AdjLevel& A0 = h->adj->L[0];
  double* fwd_out = A0.t;  // scratch output of the recording forward pass (not needed)
  ad_forward(h, 0, r, h->nl == 1 ? A0.zpre : fwd_out);
  AMG_CK(h, cudaMemcpyAsync(A0.lamA, dz, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  ad_backward(h, 0, r, A0.lamA, domega);
  AMG_CK(h, cudaMemcpyAsync(dr, A0.lr, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  AMG_CK(h, cudaGetLastError());
  AMG_CK(h, cudaStreamSynchronize(s));
  return AMG_OK;
}

extern "C" amg_status amg_vcycle_loss(amg_handle* h, const double* r0, int32_t m, double* loss,
                                      double* const* domega) {
  if (!h) return AMG_ERR_INVALID_ARG;
  if (!r0 || !loss || m < 1) return amg_fail(h, AMG_ERR_INVALID_ARG, "NULL pointer or m < 1");
  if (domega)
    for (int k = 0; k < h->nl; ++k)
      if (!domega[k]) return amg_fail(h, AMG_ERR_INVALID_ARG, "domega[%d] is NULL", k);
  if (h->p.cycle != 0) return amg_fail(h, AMG_ERR_INVALID_ARG, "the loss covers the V-cycle only");
  if (domega && h->p.relax_type != 4) return amg_fail(h, AMG_ERR_INVALID_ARG, "the adjoint covers l1-Jacobi only");
  if (h->p.prolong_scale != 0) return amg_fail(h, AMG_ERR_INVALID_ARG, "the loss covers unit prolongators only");
  amg_status st = adj_prepare(h);
  if (st != AMG_OK) return st;
  AdjState& S = *h->adj;
  const Level& L0 = h->L[0];
  const int n = L0.n, nb = amg_blocks(n);
  cudaStream_t s = h->stream;
  while ((int)S.rs.size() < m + 1) {
    double* p = nullptr;
    AMG_ALLOC(h, p, double, n);
    S.rs.push_back(p);
  }
  if (!S.lam_r) {
    AMG_ALLOC(h, S.lam_r, double, n);
    AMG_ALLOC(h, S.lam_z, double, n);
    AMG_ALLOC(h, S.scal, double, 2);
  }
  AdjLevel& A0 = h->adj->L[0];
  double* z = A0.lamB;  // forward output (the adjoint's buffers are free during the forward steps)
  AMG_CK(h, cudaMemcpyAsync(S.rs[0], r0, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  for (int t = 0; t < m; ++t) {
    ad_forward(h, 0, S.rs[t], z);
    k_loss_step<<<nb, AMG_BLOCK, 0, s>>>(n, L0.rp, L0.ci, L0.v, S.rs[t], z, S.rs[t + 1]);
  }
  st = sqnorm(h, S.rs[0], S.scal);
  if (st != AMG_OK) return st;
  st = sqnorm(h, S.rs[m], S.scal + 1);
  if (st != AMG_OK) return st;
  double nrm[2] = {0.0, 0.0};
  AMG_CK(h, cudaMemcpyAsync(nrm, S.scal, sizeof(nrm), cudaMemcpyDeviceToHost, s));
  AMG_CK(h, cudaStreamSynchronize(s));
  if (!(nrm[0] > 0.0) || !(nrm[1] > 0.0)) return amg_fail(h, AMG_ERR_INVALID_ARG, "|r_0| or |r_m| is zero");
  *loss = (std::log(std::sqrt(nrm[1])) - std::log(std::sqrt(nrm[0]))) / m;
  if (!domega) return AMG_OK;
  // backward: dL/dr_m = r_m / (m |r_m|^2); r_{t+1} = r_t - A z_t gives
  // dL/dz_t = -A^T dL/dr_{t+1} (A symmetric) and dL/dr_t = dL/dr_{t+1} + B^T dL/dz_t
  for (int k = 0; k < h->nl; ++k) AMG_CK(h, cudaMemsetAsync(domega[k], 0, sizeof(double) * h->L[k].n, s));
  k_scale_into<<<nb, AMG_BLOCK, 0, s>>>(n, S.rs[m], 1.0 / ((double)m * nrm[1]), S.lam_r);
  for (int t = m - 1; t >= 0; --t) {
    k_neg_spmv<<<nb, AMG_BLOCK, 0, s>>>(n, L0.rp, L0.ci, L0.v, S.lam_r, A0.lamA);
    ad_forward(h, 0, S.rs[t], S.lam_z);  // re-records the V-cycle of step t (lamA is not touched)
    ad_backward(h, 0, S.rs[t], A0.lamA, domega);
    k_add_into<<<nb, AMG_BLOCK, 0, s>>>(n, A0.lr, S.lam_r);
  }
  AMG_CK(h, cudaGetLastError());
  AMG_CK(h, cudaStreamSynchronize(s));
  return AMG_OK;
}
