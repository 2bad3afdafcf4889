// Learned GMRES warm start (an addition to the method: any initial guess leaves the converged
// solution of Eq. 25 unchanged; only the iteration count moves).  A per-particle network maps
// features of the particle and its 16 nearest neighbours, in its body frame, to the body-frame
// spherical-harmonic coefficients of its density; the coefficients are synthesised on the grid and
// rotated to the lab frame as the initial guess.  Training data are (features, coefficients) pairs
// recorded from solved densities.  Weights are float32 masters with bfloat16 copies; the GEMMs read
// bfloat16 operands and accumulate in float32; Adam updates the masters.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace rbs {

namespace {

constexpr int kNeigh = 16;
constexpr int kFeat = 128;
constexpr int kHidden = 256;
constexpr float kGeluC = 0.7978845608028654f;  // sqrt(2 / pi)

// k nearest particles of the same suspension by centre distance (ties to the lower index); the
// squared distance is formed with round-to-nearest products and sums in a fixed order, so the same
// ordering results wherever it is evaluated in IEEE float64.
__global__ void k_knn(int n, const double* __restrict__ centre, const int* __restrict__ srange, int* __restrict__ knn) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double bd[kNeigh];
  int bj[kNeigh];
  for (int k = 0; k < kNeigh; ++k) {
    bd[k] = INFINITY;
    bj[k] = -1;
  }
  const double cx = centre[3 * i], cy = centre[3 * i + 1], cz = centre[3 * i + 2];
  for (int j = srange[2 * i]; j < srange[2 * i + 1]; ++j) {
    if (j == i) continue;
    const double dx = centre[3 * j] - cx, dy = centre[3 * j + 1] - cy, dz = centre[3 * j + 2] - cz;
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    if (!(d2 < bd[kNeigh - 1])) continue;  // equal distance: the earlier (lower) index stays
    int k = kNeigh - 1;
    while (k > 0 && d2 < bd[k - 1]) {
      bd[k] = bd[k - 1];
      bj[k] = bj[k - 1];
      --k;
    }
    bd[k] = d2;
    bj[k] = j;
  }
  for (int k = 0; k < kNeigh; ++k) knn[kNeigh * i + k] = bj[k];
}

// Feature rows (128 floats): R^T F, R^T T, semi-axes, then per neighbour R^T (c_j - c_i) and
// conj(q_i) q_j with a non-negative scalar part; zeros elsewhere.
__global__ void k_features(int n, const double* __restrict__ centre, const double* __restrict__ rot,
                           const double* __restrict__ quat, const double* __restrict__ axes, const double* __restrict__ FT,
                           const int* __restrict__ knn, float* __restrict__ X32, __nv_bfloat16* __restrict__ Xb) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* R = rot + 9 * i;
  float f[kFeat];
  for (int k = 0; k < kFeat; ++k) f[k] = 0.0f;
  for (int a = 0; a < 3; ++a) {
    f[a] = (float)(R[a] * FT[6 * i] + R[3 + a] * FT[6 * i + 1] + R[6 + a] * FT[6 * i + 2]);
    f[3 + a] = (float)(R[a] * FT[6 * i + 3] + R[3 + a] * FT[6 * i + 4] + R[6 + a] * FT[6 * i + 5]);
    f[6 + a] = (float)axes[3 * i + a];
  }
  double qi[4];
  double qn = 0.0;
  for (int a = 0; a < 4; ++a) {
    qi[a] = quat[4 * i + a];
    qn += qi[a] * qi[a];
  }
  qn = rsqrt(qn);
  for (int a = 0; a < 4; ++a) qi[a] *= qn;
  for (int k = 0; k < kNeigh; ++k) {
    const int j = knn[kNeigh * i + k];
    if (j < 0) continue;
    const double d0 = centre[3 * j] - centre[3 * i], d1 = centre[3 * j + 1] - centre[3 * i + 1],
                 d2 = centre[3 * j + 2] - centre[3 * i + 2];
    for (int a = 0; a < 3; ++a) f[9 + 7 * k + a] = (float)(R[a] * d0 + R[3 + a] * d1 + R[6 + a] * d2);
    double qj[4];
    double qjn = 0.0;
    for (int a = 0; a < 4; ++a) {
      qj[a] = quat[4 * j + a];
      qjn += qj[a] * qj[a];
    }
    qjn = rsqrt(qjn);
    for (int a = 0; a < 4; ++a) qj[a] *= qjn;
    // conj(qi) * qj
    const double w1 = qi[0], x1 = -qi[1], y1 = -qi[2], z1 = -qi[3];
    double r[4] = {w1 * qj[0] - x1 * qj[1] - y1 * qj[2] - z1 * qj[3], w1 * qj[1] + x1 * qj[0] + y1 * qj[3] - z1 * qj[2],
                   w1 * qj[2] - x1 * qj[3] + y1 * qj[0] + z1 * qj[1], w1 * qj[3] + x1 * qj[2] - y1 * qj[1] + z1 * qj[0]};
    const double sgn = r[0] < 0.0 ? -1.0 : 1.0;
    for (int a = 0; a < 4; ++a) f[12 + 7 * k + a] = (float)(sgn * r[a]);
  }
  for (int k = 0; k < kFeat; ++k) {
    X32[(size_t)kFeat * i + k] = f[k];
    Xb[(size_t)kFeat * i + k] = __float2bfloat16(f[k]);
  }
}

// Body-frame coefficients of a surface density: coef[i][c * nb + b] = sum_s An[b][s] (R_i^T mu_s)_c,
// one block per particle.
__global__ void k_targets(const long long* __restrict__ offset, const double* __restrict__ rot, const double* __restrict__ An,
                          int nb, int np, const double* __restrict__ mu, float* __restrict__ coef, int ld) {
  extern __shared__ double zb[];  // 3 np body-frame density
  const int i = blockIdx.x;
  const double* R = rot + 9 * i;
  const long long o = offset[i];
  for (int s = threadIdx.x; s < np; s += blockDim.x) {
    const double a = mu[3 * (o + s)], b = mu[3 * (o + s) + 1], c = mu[3 * (o + s) + 2];
    zb[s] = R[0] * a + R[3] * b + R[6] * c;
    zb[np + s] = R[1] * a + R[4] * b + R[7] * c;
    zb[2 * np + s] = R[2] * a + R[5] * b + R[8] * c;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < 3 * nb; r += blockDim.x) {
    const int comp = r / nb, b = r % nb;
    const double* row = An + (size_t)b * np;
    const double* z = zb + comp * np;
    double acc = 0.0;
    for (int s = 0; s < np; ++s) acc = fma(row[s], z[s], acc);
    coef[(size_t)ld * i + r] = (float)acc;
  }
}

// Initial guess from coefficients: mu0(node) = R_i sum_b coef_b Y_b(node).
__global__ void k_synthesize(int n, const long long* __restrict__ offset, const double* __restrict__ rot,
                             const double* __restrict__ Yg, int nb, int np, const float* __restrict__ coef, int ld,
                             double scale, double* __restrict__ mu0) {
  const int i = blockIdx.y;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || s >= np) return;
  const double* y = Yg + (size_t)s * nb;
  const float* cf = coef + (size_t)ld * i;
  double b0 = 0.0, b1 = 0.0, b2 = 0.0;
  for (int b = 0; b < nb; ++b) {
    b0 = fma((double)cf[b], y[b], b0);
    b1 = fma((double)cf[nb + b], y[b], b1);
    b2 = fma((double)cf[2 * nb + b], y[b], b2);
  }
  b0 *= scale;
  b1 *= scale;
  b2 *= scale;
  const double* R = rot + 9 * i;
  const long long g = offset[i] + s;
  mu0[3 * g + 0] = R[0] * b0 + R[1] * b1 + R[2] * b2;
  mu0[3 * g + 1] = R[3] * b0 + R[4] * b1 + R[5] * b2;
  mu0[3 * g + 2] = R[6] * b0 + R[7] * b1 + R[8] * b2;
}

__device__ __forceinline__ float gelu_f(float x) {
  return 0.5f * x * (1.0f + tanhf(kGeluC * (x + 0.044715f * x * x * x)));
}
__device__ __forceinline__ float gelu_grad_f(float x) {
  const float t = tanhf(kGeluC * (x + 0.044715f * x * x * x));
  return 0.5f * (1.0f + t) + 0.5f * x * (1.0f - t * t) * kGeluC * (1.0f + 3.0f * 0.044715f * x * x);
}

// C (M x N, float32) = op(A) op(B) with bfloat16 operands and float32 accumulation; op(A) is M x K
// (A stored K x M when TA), op(B) is K x N (B stored N x K when TB).  Epilogue: mode 0 C = acc,
// mode 1 C = acc + bias (float32 out), mode 2 Z = acc + bias, H = gelu(Z) in bfloat16.
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_gemm_bf16(int M, int N, int K, const __nv_bfloat16* __restrict__ A, int lda,
                                                   const __nv_bfloat16* __restrict__ B, int ldb, float* __restrict__ C,
                                                   int ldc, const float* __restrict__ bias, int mode,
                                                   __nv_bfloat16* __restrict__ H) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ float As[BK][BM + 1];
  __shared__ float Bs[BK][BN + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int l = threadIdx.x; l < BM * BK; l += 256) {
      const int r = TA ? l % BM : l / BK, kk = TA ? l / BM : l % BK;
      const int gr = row0 + r, gk = k0 + kk;
      float v = 0.0f;
      if (gr < M && gk < K) v = __bfloat162float(TA ? A[(size_t)gk * lda + gr] : A[(size_t)gr * lda + gk]);
      As[kk][r] = v;
    }
    for (int l = threadIdx.x; l < BK * BN; l += 256) {
      const int cc = TB ? l / BK : l % BN, kk = TB ? l % BK : l / BN;
      const int gk = k0 + kk, gc = col0 + cc;
      float v = 0.0f;
      if (gk < K && gc < N) v = __bfloat162float(TB ? B[(size_t)gc * ldb + gk] : B[(size_t)gk * ldb + gc]);
      Bs[kk][cc] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = row0 + ty + 16 * i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int cidx = col0 + tx + 16 * j;
      if (cidx >= N) continue;
      float v = acc[i][j];
      if (mode >= 1) v += bias[cidx];
      C[(size_t)r * ldc + cidx] = v;
      if (mode == 2) H[(size_t)r * ldc + cidx] = __float2bfloat16(gelu_f(v));
    }
  }
}

__global__ void k_to_bf16(const float* __restrict__ in, __nv_bfloat16* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16(in[i]);
}

// dY = 2 (y - t / scale) / (B D) (loss on the scaled targets), partial sums of the squared error.
__global__ void k_mse_grad(long long total, const float* __restrict__ y, const float* __restrict__ t, float inv_scale,
                           float norm, __nv_bfloat16* __restrict__ dYb, float* __restrict__ dY, double* __restrict__ loss) {
  __shared__ double red[256];
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const float d = y[i] - t[i] * inv_scale;
    acc += (double)d * d;
    const float g = 2.0f * d * norm;
    dY[i] = g;
    dYb[i] = __float2bfloat16(g);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0]);
}

// dZ = dH * gelu'(Z), in float32 and bfloat16.
__global__ void k_gelu_back(long long total, const float* __restrict__ dH, const float* __restrict__ Z, float* __restrict__ dZ,
                            __nv_bfloat16* __restrict__ dZb) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const float g = dH[i] * gelu_grad_f(Z[i]);
    dZ[i] = g;
    dZb[i] = __float2bfloat16(g);
  }
}

// column sums of an M x N float32 matrix (bias gradients)
__global__ void k_colsum(int M, int N, const float* __restrict__ A, float* __restrict__ out) {
  const int cidx = blockIdx.x * blockDim.x + threadIdx.x;
  if (cidx >= N) return;
  float s = 0.0f;
  for (int r = 0; r < M; ++r) s += A[(size_t)r * N + cidx];
  out[cidx] = s;
}

// gather rows idx[r] of a (rows x cols) matrix
template <typename T>
__global__ void k_gather_rows(int rows, int cols, const int* __restrict__ idx, const T* __restrict__ src, T* __restrict__ dst) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)rows * cols;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / cols, cc = i % cols;
    dst[i] = src[(size_t)idx[r] * cols + cc];
  }
}

// The same for minibatch number *step of a device permutation: rows perm[*step * rows + r].
template <typename T>
__global__ void k_gather_step(int rows, int cols, const int* __restrict__ perm, const int* __restrict__ step,
                              const T* __restrict__ src, T* __restrict__ dst) {
  const int* idx = perm + (long long)(*step) * rows;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)rows * cols;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / cols, cc = i % cols;
    dst[i] = src[(size_t)idx[r] * cols + cc];
  }
}

// Adam (Kingma & Ba) on float32 masters, refreshing the bfloat16 copy, with the step count t + 1 read
// from the device (bias corrections 1 - b^(t+1)).
__global__ void k_adam_dev(long long n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, float lr, float b1, float b2, float eps, const long long* __restrict__ t,
                           __nv_bfloat16* __restrict__ wb) {
  const float tt = (float)(*t + 1);
  const float c1 = 1.0f - powf(b1, tt), c2 = 1.0f - powf(b2, tt);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16(wi);
  }
}

__global__ void k_next_step(int* step, long long* t) {
  *step += 1;
  *t += 1;
}

}  // namespace

// ------------------------------------------------------------------------------------------
// Host side

struct WarmState {
  int grid = -1, nb = 0, np = 0, D = 0;
  // parameters: W1 (128 x 256), b1, W2 (256 x 256), b2, W3 (256 x D), b3, flattened in this order
  DevBuf<float> w, g, m, v;
  DevBuf<__nv_bfloat16> wb;
  long long nparam = 0;
  long long adam_t = 0;
  float out_scale = 1.0f;
  bool have_weights = false;
  // training set
  long long cap = 0, count = 0;
  DevBuf<__nv_bfloat16> Xs;
  DevBuf<float> Ys;
  // per-geometry scratch
  DevBuf<int> knn, srange;
  DevBuf<double> An, Yg;
  // activations (capacity rows)
  int act_rows = 0;
  DevBuf<float> x32, z1, z2, y, dy, dh, dz;
  DevBuf<__nv_bfloat16> xb, h1, h2, dyb, dzb;
  DevBuf<float> t;
  DevBuf<double> loss;
  size_t off[6] = {0, 0, 0, 0, 0, 0};
  // the training step as a CUDA graph (fixed batch size), launched on its own stream
  cudaGraphExec_t step_exec = nullptr;
  int step_batch = 0;
  int step_kernels = 0;
  std::vector<const void*> step_sig;
  cudaStream_t gs = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  DevBuf<int> perm, step;
  DevBuf<long long> t_dev;
  ~WarmState() {
    if (step_exec) cudaGraphExecDestroy(step_exec);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (gs) cudaStreamDestroy(gs);
  }
};

static size_t param_count(int D) {
  return (size_t)kFeat * kHidden + kHidden + (size_t)kHidden * kHidden + kHidden + (size_t)kHidden * D + D;
}

Status warm_prepare(Context& c) {
  if (!c.warm) c.warm = new WarmState();
  WarmState& W = *c.warm;
  if (c.grids.size() != 1)
    return Status::Err(RBS_EINVAL, "the learned warm start needs one (p, n_phi) grid for all particles");
  Grid& g = *c.grids[0];
  cudaStream_t s = c.stream;
  if (W.grid != 0 || W.nb != g.nbasis || W.np != g.np) {
    W.grid = 0;
    W.nb = g.nbasis;
    W.np = g.np;
    W.D = 3 * g.nbasis;
    W.nparam = (long long)param_count(W.D);
    RBS_TRY(W.w.alloc(W.nparam));
    RBS_TRY(W.g.alloc(W.nparam));
    RBS_TRY(W.m.alloc(W.nparam));
    RBS_TRY(W.v.alloc(W.nparam));
    RBS_TRY(W.wb.alloc(W.nparam));
    RBS_CUDA_TRY(cudaMemsetAsync(W.w.ptr, 0, sizeof(float) * W.nparam, s));
    W.have_weights = false;
    W.count = 0;
    W.off[0] = 0;
    W.off[1] = W.off[0] + (size_t)kFeat * kHidden;
    W.off[2] = W.off[1] + kHidden;
    W.off[3] = W.off[2] + (size_t)kHidden * kHidden;
    W.off[4] = W.off[3] + kHidden;
    W.off[5] = W.off[4] + (size_t)kHidden * W.D;
  }
  // analysis matrix and grid synthesis values of the grid (float64)
  if (W.An.n != (size_t)g.nbasis * g.np) {
    RBS_TRY(W.An.alloc((size_t)g.nbasis * g.np));
    RBS_TRY(W.Yg.alloc((size_t)g.nbasis * g.np));
    RBS_CUDA_TRY(cudaMemcpyAsync(W.An.ptr, g.d_an.ptr, sizeof(double) * W.An.n, cudaMemcpyDeviceToDevice, s));
    RBS_CUDA_TRY(cudaMemcpyAsync(W.Yg.ptr, g.d_yg.ptr, sizeof(double) * W.Yg.n, cudaMemcpyDeviceToDevice, s));
  }
  // suspension ranges for the neighbour search
  std::vector<int> sr(2 * (size_t)c.n);
  int i = 0;
  while (i < c.n) {
    int e = i + 1;
    while (e < c.n && c.sid[e] == c.sid[i]) ++e;
    for (int k = i; k < e; ++k) {
      sr[2 * k] = i;
      sr[2 * k + 1] = e;
    }
    i = e;
  }
  RBS_TRY(W.srange.alloc(sr.size()));
  RBS_CUDA_TRY(cudaMemcpyAsync(W.srange.ptr, sr.data(), sizeof(int) * sr.size(), cudaMemcpyHostToDevice, s));
  RBS_TRY(W.knn.alloc((size_t)kNeigh * c.n));
  return Status::Ok();
}

static Status ensure_rows(Context& c, int rows) {
  WarmState& W = *c.warm;
  if (W.act_rows >= rows) return Status::Ok();
  W.act_rows = rows;
  RBS_TRY(W.x32.alloc((size_t)rows * kFeat));
  RBS_TRY(W.xb.alloc((size_t)rows * kFeat));
  RBS_TRY(W.z1.alloc((size_t)rows * kHidden));
  RBS_TRY(W.h1.alloc((size_t)rows * kHidden));
  RBS_TRY(W.z2.alloc((size_t)rows * kHidden));
  RBS_TRY(W.h2.alloc((size_t)rows * kHidden));
  RBS_TRY(W.y.alloc((size_t)rows * W.D));
  RBS_TRY(W.dy.alloc((size_t)rows * W.D));
  RBS_TRY(W.dyb.alloc((size_t)rows * W.D));
  RBS_TRY(W.dh.alloc((size_t)rows * std::max(kHidden, W.D)));
  RBS_TRY(W.dz.alloc((size_t)rows * kHidden));
  RBS_TRY(W.dzb.alloc((size_t)rows * kHidden));
  RBS_TRY(W.t.alloc((size_t)rows * W.D));
  RBS_TRY(W.loss.alloc(1));
  return Status::Ok();
}

template <bool TA, bool TB>
static void gemm(Context& c, int M, int N, int K, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, float* C,
                 int ldc, const float* bias, int mode, __nv_bfloat16* H) {
  dim3 grd(cdiv(N, 64), cdiv(M, 64));
  c.stats.launches += 1;
  k_gemm_bf16<TA, TB><<<grd, 256, 0, c.stream>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, mode, H);
}

// Forward pass on rows of W.xb; leaves z1, h1, z2, h2 and y (scaled outputs).
static Status mlp_forward(Context& c, int rows) {
  WarmState& W = *c.warm;
  const __nv_bfloat16* wb = W.wb.ptr;
  const float* w = W.w.ptr;
  gemm<false, false>(c, rows, kHidden, kFeat, W.xb.ptr, kFeat, wb + W.off[0], kHidden, W.z1.ptr, kHidden, w + W.off[1], 2,
                     W.h1.ptr);
  gemm<false, false>(c, rows, kHidden, kHidden, W.h1.ptr, kHidden, wb + W.off[2], kHidden, W.z2.ptr, kHidden,
                     w + W.off[3], 2, W.h2.ptr);
  gemm<false, false>(c, rows, W.D, kHidden, W.h2.ptr, kHidden, wb + W.off[4], W.D, W.y.ptr, W.D, w + W.off[5], 1, nullptr);
  RBS_CUDA_TRY(cudaGetLastError());
  return Status::Ok();
}

// Gradients of the mean squared error against W.t (already scaled by 1 / out_scale inside) into W.g.
static Status mlp_backward(Context& c, int rows, double* loss_out) {
  WarmState& W = *c.warm;
  cudaStream_t s = c.stream;
  const __nv_bfloat16* wb = W.wb.ptr;
  float* g = W.g.ptr;
  const long long tot = (long long)rows * W.D;
  // with loss_out the loss of this batch is returned; without, the squared errors accumulate in W.loss
  if (loss_out) RBS_CUDA_TRY(cudaMemsetAsync(W.loss.ptr, 0, sizeof(double), s));
  c.stats.launches += 1;
  k_mse_grad<<<std::min(1024, cdiv(tot, 256)), 256, 0, s>>>(tot, W.y.ptr, W.t.ptr, 1.0f / W.out_scale,
                                                             1.0f / (float)tot, W.dyb.ptr, W.dy.ptr, W.loss.ptr);
  // layer 3
  gemm<true, false>(c, kHidden, W.D, rows, W.h2.ptr, kHidden, W.dyb.ptr, W.D, g + W.off[4], W.D, nullptr, 0, nullptr);
  c.stats.launches += 1;
  k_colsum<<<cdiv(W.D, 128), 128, 0, s>>>(rows, W.D, W.dy.ptr, g + W.off[5]);
  gemm<false, true>(c, rows, kHidden, W.D, W.dyb.ptr, W.D, wb + W.off[4], W.D, W.dh.ptr, kHidden, nullptr, 0, nullptr);
  c.stats.launches += 1;
  k_gelu_back<<<std::min(1024, cdiv((long long)rows * kHidden, 256)), 256, 0, s>>>((long long)rows * kHidden, W.dh.ptr,
                                                                                   W.z2.ptr, W.dz.ptr, W.dzb.ptr);
  // layer 2
  gemm<true, false>(c, kHidden, kHidden, rows, W.h1.ptr, kHidden, W.dzb.ptr, kHidden, g + W.off[2], kHidden, nullptr, 0,
                    nullptr);
  c.stats.launches += 1;
  k_colsum<<<cdiv(kHidden, 128), 128, 0, s>>>(rows, kHidden, W.dz.ptr, g + W.off[3]);
  gemm<false, true>(c, rows, kHidden, kHidden, W.dzb.ptr, kHidden, wb + W.off[2], kHidden, W.dh.ptr, kHidden, nullptr, 0,
                    nullptr);
  c.stats.launches += 1;
  k_gelu_back<<<std::min(1024, cdiv((long long)rows * kHidden, 256)), 256, 0, s>>>((long long)rows * kHidden, W.dh.ptr,
                                                                                   W.z1.ptr, W.dz.ptr, W.dzb.ptr);
  // layer 1
  gemm<true, false>(c, kFeat, kHidden, rows, W.xb.ptr, kFeat, W.dzb.ptr, kHidden, g + W.off[0], kHidden, nullptr, 0,
                    nullptr);
  c.stats.launches += 1;
  k_colsum<<<cdiv(kHidden, 128), 128, 0, s>>>(rows, kHidden, W.dz.ptr, g + W.off[1]);
  RBS_CUDA_TRY(cudaGetLastError());
  if (loss_out) {
    double l = 0.0;
    RBS_CUDA_TRY(cudaMemcpyAsync(&l, W.loss.ptr, sizeof(double), cudaMemcpyDeviceToHost, s));
    RBS_CUDA_TRY(cudaStreamSynchronize(s));
    *loss_out = l / (double)tot;
  }
  return Status::Ok();
}

// Features of the current configuration for forces and torques FT (device, n x 6) into W.x32 / W.xb.
static Status warm_features(Context& c, const double* FT_dev) {
  WarmState& W = *c.warm;
  RBS_TRY(ensure_rows(c, c.n));
  DevBuf<double> q;
  RBS_TRY(q.alloc(4 * (size_t)c.n));
  RBS_CUDA_TRY(cudaMemcpyAsync(q.ptr, c.quats.data(), sizeof(double) * 4 * c.n, cudaMemcpyHostToDevice, c.stream));
  c.stats.launches += 2;
  k_knn<<<cdiv(c.n, 128), 128, 0, c.stream>>>(c.n, c.d_centre.ptr, W.srange.ptr, W.knn.ptr);
  k_features<<<cdiv(c.n, 64), 64, 0, c.stream>>>(c.n, c.d_centre.ptr, c.d_rot.ptr, q.ptr, c.d_axes.ptr, FT_dev, W.knn.ptr,
                                                 W.x32.ptr, W.xb.ptr);
  RBS_CUDA_TRY(cudaGetLastError());
  RBS_CUDA_TRY(cudaStreamSynchronize(c.stream));
  return Status::Ok();
}

Status warm_guess(Context& c, const double* FT_dev, double* mu0) {
  RBS_TRY(warm_prepare(c));
  WarmState& W = *c.warm;
  if (!W.have_weights) return Status::Err(RBS_ESTATE, "learned warm start has no weights (train or load them first)");
  RBS_TRY(warm_features(c, FT_dev));
  RBS_TRY(mlp_forward(c, c.n));
  dim3 grd(cdiv(W.np, 128), c.n);
  c.stats.launches += 1;
  k_synthesize<<<grd, 128, 0, c.stream>>>(c.n, c.d_offset.ptr, c.d_rot.ptr, W.Yg.ptr, W.nb, W.np, W.y.ptr, W.D,
                                          (double)W.out_scale, mu0);
  RBS_CUDA_TRY(cudaGetLastError());
  return Status::Ok();
}

Status warm_record(Context& c, const double* FT_dev, const double* mu) {
  RBS_TRY(warm_prepare(c));
  WarmState& W = *c.warm;
  RBS_TRY(warm_features(c, FT_dev));
  if (W.count + c.n > W.cap) {
    long long cap = std::max<long long>(W.count + c.n, 2 * W.cap + 4096);
    DevBuf<__nv_bfloat16> X2;
    DevBuf<float> Y2;
    RBS_TRY(X2.alloc((size_t)cap * kFeat));
    RBS_TRY(Y2.alloc((size_t)cap * W.D));
    if (W.count) {
      RBS_CUDA_TRY(cudaMemcpyAsync(X2.ptr, W.Xs.ptr, sizeof(__nv_bfloat16) * W.count * kFeat, cudaMemcpyDeviceToDevice, c.stream));
      RBS_CUDA_TRY(cudaMemcpyAsync(Y2.ptr, W.Ys.ptr, sizeof(float) * W.count * W.D, cudaMemcpyDeviceToDevice, c.stream));
    }
    RBS_CUDA_TRY(cudaStreamSynchronize(c.stream));
    std::swap(W.Xs.ptr, X2.ptr);
    std::swap(W.Xs.n, X2.n);
    std::swap(W.Ys.ptr, Y2.ptr);
    std::swap(W.Ys.n, Y2.n);
    W.cap = cap;
  }
  RBS_CUDA_TRY(cudaMemcpyAsync(W.Xs.ptr + W.count * kFeat, W.xb.ptr, sizeof(__nv_bfloat16) * c.n * kFeat,
                               cudaMemcpyDeviceToDevice, c.stream));
  c.stats.launches += 1;
  k_targets<<<c.n, 128, sizeof(double) * 3 * W.np, c.stream>>>(c.d_offset.ptr, c.d_rot.ptr, W.An.ptr, W.nb, W.np, mu,
                                                                W.Ys.ptr + W.count * W.D, W.D);
  RBS_CUDA_TRY(cudaGetLastError());
  RBS_CUDA_TRY(cudaStreamSynchronize(c.stream));
  W.count += c.n;
  return Status::Ok();
}

Status warm_train(Context& c, int epochs, int batch, double lr, unsigned seed, double* final_loss) {
  RBS_TRY(warm_prepare(c));
  WarmState& W = *c.warm;
  if (W.count < 1) return Status::Err(RBS_ESTATE, "no recorded training samples");
  cudaStream_t s = c.stream;
  batch = std::max(1, std::min<int>(batch, (int)W.count));
  RBS_TRY(ensure_rows(c, batch));
  if (!W.have_weights) {
    // He-style initial weights from a seeded host generator, output scale from the targets' RMS
    std::vector<float> h(W.nparam, 0.0f);
    unsigned long long st = 0x9E3779B97F4A7C15ULL ^ seed;
    auto nrm = [&]() {
      double u1, u2;
      st = st * 6364136223846793005ULL + 1442695040888963407ULL;
      u1 = ((st >> 11) + 0.5) * (1.0 / 9007199254740992.0);
      st = st * 6364136223846793005ULL + 1442695040888963407ULL;
      u2 = ((st >> 11) + 0.5) * (1.0 / 9007199254740992.0);
      return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * kPi * u2);
    };
    for (size_t k = 0; k < (size_t)kFeat * kHidden; ++k) h[W.off[0] + k] = (float)(nrm() * std::sqrt(2.0 / kFeat));
    for (size_t k = 0; k < (size_t)kHidden * kHidden; ++k) h[W.off[2] + k] = (float)(nrm() * std::sqrt(2.0 / kHidden));
    for (size_t k = 0; k < (size_t)kHidden * W.D; ++k) h[W.off[4] + k] = (float)(nrm() * std::sqrt(1.0 / kHidden));
    RBS_CUDA_TRY(cudaMemcpyAsync(W.w.ptr, h.data(), sizeof(float) * W.nparam, cudaMemcpyHostToDevice, s));
    std::vector<float> ys((size_t)std::min<long long>(W.count, 65536) * W.D);
    RBS_CUDA_TRY(cudaMemcpyAsync(ys.data(), W.Ys.ptr, sizeof(float) * ys.size(), cudaMemcpyDeviceToHost, s));
    RBS_CUDA_TRY(cudaStreamSynchronize(s));
    double ss = 0.0;
    for (float v : ys) ss += (double)v * v;
    W.out_scale = (float)std::max(1e-30, std::sqrt(ss / std::max<size_t>(1, ys.size())));
    RBS_CUDA_TRY(cudaMemsetAsync(W.m.ptr, 0, sizeof(float) * W.nparam, s));
    RBS_CUDA_TRY(cudaMemsetAsync(W.v.ptr, 0, sizeof(float) * W.nparam, s));
    W.adam_t = 0;
    c.stats.launches += 1;
    k_to_bf16<<<1024, 256, 0, s>>>(W.w.ptr, W.wb.ptr, W.nparam);
    W.have_weights = true;
  }
  // Shuffled minibatches (host permutation, seeded, one upload per epoch).  One training step (gather,
  // forward, backward, Adam, step counters) is captured once as a CUDA graph on a private stream and
  // replayed for every minibatch; the loss is summed on the device and read once per epoch.
  const int steps = (int)(W.count / batch);
  std::vector<int> perm(W.count);
  RBS_TRY(W.perm.alloc(W.count));
  RBS_TRY(W.step.alloc(1));
  RBS_TRY(W.t_dev.alloc(1));
  if (!W.gs) {
    RBS_CUDA_TRY(cudaStreamCreateWithFlags(&W.gs, cudaStreamNonBlocking));
    RBS_CUDA_TRY(cudaEventCreateWithFlags(&W.ev_in, cudaEventDisableTiming));
    RBS_CUDA_TRY(cudaEventCreateWithFlags(&W.ev_out, cudaEventDisableTiming));
  }
  // the captured graph holds raw pointers: recapture when the batch size or any buffer it touches changed
  const std::vector<const void*> sig = {W.Xs.ptr, W.Ys.ptr, W.perm.ptr, W.step.ptr, W.t_dev.ptr, W.w.ptr, W.g.ptr,
                                        W.m.ptr,  W.v.ptr,  W.wb.ptr,   W.xb.ptr,   W.t.ptr,     W.z1.ptr, W.h1.ptr,
                                        W.z2.ptr, W.h2.ptr, W.y.ptr,    W.dy.ptr,   W.dyb.ptr,   W.dh.ptr, W.dz.ptr,
                                        W.dzb.ptr, W.loss.ptr};
  if (W.step_exec && (W.step_batch != batch || W.step_sig != sig)) {
    RBS_CUDA_TRY(cudaGraphExecDestroy(W.step_exec));
    W.step_exec = nullptr;
  }
  if (!W.step_exec && steps > 0) {
    const cudaStream_t user = c.stream;
    const long long launches0 = c.stats.launches;
    c.stream = W.gs;
    cudaGraph_t graph = nullptr;
    RBS_CUDA_TRY(cudaStreamBeginCapture(W.gs, cudaStreamCaptureModeThreadLocal));
    k_gather_step<__nv_bfloat16><<<256, 256, 0, W.gs>>>(batch, kFeat, W.perm.ptr, W.step.ptr, W.Xs.ptr, W.xb.ptr);
    k_gather_step<float><<<256, 256, 0, W.gs>>>(batch, W.D, W.perm.ptr, W.step.ptr, W.Ys.ptr, W.t.ptr);
    Status st1 = mlp_forward(c, batch);
    Status st2 = st1.ok() ? mlp_backward(c, batch, nullptr) : st1;
    k_adam_dev<<<1024, 256, 0, W.gs>>>(W.nparam, W.w.ptr, W.g.ptr, W.m.ptr, W.v.ptr, (float)lr, 0.9f, 0.999f, 1e-8f,
                                       W.t_dev.ptr, W.wb.ptr);
    k_next_step<<<1, 1, 0, W.gs>>>(W.step.ptr, W.t_dev.ptr);
    cudaError_t ce = cudaStreamEndCapture(W.gs, &graph);
    c.stream = user;
    W.step_kernels = (int)(c.stats.launches - launches0) + 4;
    c.stats.launches = launches0;
    RBS_TRY(st2);
    RBS_CUDA_TRY(ce);
    ce = cudaGraphInstantiate(&W.step_exec, graph, 0);
    cudaGraphDestroy(graph);
    RBS_CUDA_TRY(ce);
    W.step_batch = batch;
    W.step_sig = sig;
  }
  unsigned long long st = 0xD1B54A32D192ED03ULL ^ (seed * 2654435761ULL);
  double last = 0.0;
  for (int e = 0; e < epochs; ++e) {
    for (long long k = 0; k < W.count; ++k) perm[k] = (int)k;
    for (long long k = W.count - 1; k > 0; --k) {
      st = st * 6364136223846793005ULL + 1442695040888963407ULL;
      long long j = (long long)((st >> 33) % (unsigned long long)(k + 1));
      std::swap(perm[k], perm[j]);
    }
    if (steps == 0) continue;
    RBS_CUDA_TRY(cudaMemcpyAsync(W.perm.ptr, perm.data(), sizeof(int) * W.count, cudaMemcpyHostToDevice, s));
    RBS_CUDA_TRY(cudaMemsetAsync(W.step.ptr, 0, sizeof(int), s));
    RBS_CUDA_TRY(cudaMemcpyAsync(W.t_dev.ptr, &W.adam_t, sizeof(long long), cudaMemcpyHostToDevice, s));
    RBS_CUDA_TRY(cudaMemsetAsync(W.loss.ptr, 0, sizeof(double), s));
    RBS_CUDA_TRY(cudaEventRecord(W.ev_in, s));
    RBS_CUDA_TRY(cudaStreamWaitEvent(W.gs, W.ev_in, 0));
    for (int b = 0; b < steps; ++b) RBS_CUDA_TRY(cudaGraphLaunch(W.step_exec, W.gs));
    RBS_CUDA_TRY(cudaEventRecord(W.ev_out, W.gs));
    RBS_CUDA_TRY(cudaStreamWaitEvent(s, W.ev_out, 0));
    c.stats.launches += (long long)steps * W.step_kernels;
    W.adam_t += steps;
    double l = 0.0;
    RBS_CUDA_TRY(cudaMemcpyAsync(&l, W.loss.ptr, sizeof(double), cudaMemcpyDeviceToHost, s));
    RBS_CUDA_TRY(cudaStreamSynchronize(s));
    last = l / ((double)steps * batch * W.D);
  }
  RBS_CUDA_TRY(cudaStreamSynchronize(s));
  if (final_loss) *final_loss = last;
  return Status::Ok();
}

Status warm_weights(Context& c, float* out, const float* in, long long* count, float* scale_inout) {
  RBS_TRY(warm_prepare(c));
  WarmState& W = *c.warm;
  if (count) *count = W.nparam;
  if (out) {
    RBS_CUDA_TRY(cudaMemcpyAsync(out, W.w.ptr, sizeof(float) * W.nparam, cudaMemcpyDeviceToHost, c.stream));
    RBS_CUDA_TRY(cudaStreamSynchronize(c.stream));
    if (scale_inout) *scale_inout = W.out_scale;
  } else if (in) {
    RBS_CUDA_TRY(cudaMemcpyAsync(W.w.ptr, in, sizeof(float) * W.nparam, cudaMemcpyHostToDevice, c.stream));
    c.stats.launches += 1;
    k_to_bf16<<<1024, 256, 0, c.stream>>>(W.w.ptr, W.wb.ptr, W.nparam);
    RBS_CUDA_TRY(cudaGetLastError());
    RBS_CUDA_TRY(cudaStreamSynchronize(c.stream));
    W.out_scale = scale_inout ? *scale_inout : 1.0f;
    W.have_weights = true;
    W.adam_t = 0;
    RBS_CUDA_TRY(cudaMemsetAsync(W.m.ptr, 0, sizeof(float) * W.nparam, c.stream));
    RBS_CUDA_TRY(cudaMemsetAsync(W.v.ptr, 0, sizeof(float) * W.nparam, c.stream));
  }
  return Status::Ok();
}

// Host-buffer entry points for the parity tests: features, targets, forward, gradients.
Status warm_features_host(Context& c, const double* F, const double* T, float* X) {
  RBS_TRY(warm_prepare(c));
  std::vector<double> ft(6 * (size_t)c.n);
  for (int i = 0; i < c.n; ++i)
    for (int q = 0; q < 3; ++q) {
      ft[6 * i + q] = F[3 * i + q];
      ft[6 * i + 3 + q] = T[3 * i + q];
    }
  RBS_CUDA_TRY(cudaMemcpyAsync(c.d_FT.ptr, ft.data(), sizeof(double) * ft.size(), cudaMemcpyHostToDevice, c.stream));
  RBS_TRY(warm_features(c, c.d_FT.ptr));
  RBS_CUDA_TRY(cudaMemcpyAsync(X, c.warm->x32.ptr, sizeof(float) * c.n * kFeat, cudaMemcpyDeviceToHost, c.stream));
  RBS_CUDA_TRY(cudaStreamSynchronize(c.stream));
  return Status::Ok();
}

Status warm_targets_host(Context& c, const double* mu, float* coef) {
  RBS_TRY(warm_prepare(c));
  WarmState& W = *c.warm;
  RBS_CUDA_TRY(cudaMemcpyAsync(c.d_vec[0].ptr, mu, sizeof(double) * 3 * c.N, cudaMemcpyHostToDevice, c.stream));
  DevBuf<float> out;
  RBS_TRY(out.alloc((size_t)c.n * W.D));
  c.stats.launches += 1;
  k_targets<<<c.n, 128, sizeof(double) * 3 * W.np, c.stream>>>(c.d_offset.ptr, c.d_rot.ptr, W.An.ptr, W.nb, W.np,
                                                                c.d_vec[0].ptr, out.ptr, W.D);
  RBS_CUDA_TRY(cudaGetLastError());
  RBS_CUDA_TRY(cudaMemcpyAsync(coef, out.ptr, sizeof(float) * c.n * W.D, cudaMemcpyDeviceToHost, c.stream));
  RBS_CUDA_TRY(cudaStreamSynchronize(c.stream));
  return Status::Ok();
}

Status warm_mlp_host(Context& c, int rows, const float* X, const float* Yt, float* Y, float* grads, double* loss) {
  RBS_TRY(warm_prepare(c));
  WarmState& W = *c.warm;
  if (!W.have_weights) return Status::Err(RBS_ESTATE, "no weights");
  RBS_TRY(ensure_rows(c, rows));
  RBS_CUDA_TRY(cudaMemcpyAsync(W.x32.ptr, X, sizeof(float) * rows * kFeat, cudaMemcpyHostToDevice, c.stream));
  c.stats.launches += 1;
  k_to_bf16<<<256, 256, 0, c.stream>>>(W.x32.ptr, W.xb.ptr, (long long)rows * kFeat);
  RBS_TRY(mlp_forward(c, rows));
  if (Y) RBS_CUDA_TRY(cudaMemcpyAsync(Y, W.y.ptr, sizeof(float) * rows * W.D, cudaMemcpyDeviceToHost, c.stream));
  if (grads && Yt) {
    RBS_CUDA_TRY(cudaMemcpyAsync(W.t.ptr, Yt, sizeof(float) * rows * W.D, cudaMemcpyHostToDevice, c.stream));
    const float keep = W.out_scale;
    W.out_scale = 1.0f;  // gradients of the plain mean squared error against Yt
    Status st = mlp_backward(c, rows, loss);
    W.out_scale = keep;
    RBS_TRY(st);
    RBS_CUDA_TRY(cudaMemcpyAsync(grads, W.g.ptr, sizeof(float) * W.nparam, cudaMemcpyDeviceToHost, c.stream));
  }
  RBS_CUDA_TRY(cudaStreamSynchronize(c.stream));
  return Status::Ok();
}

void warm_release(Context& c) {
  delete c.warm;
  c.warm = nullptr;
}

}  // namespace rbs
