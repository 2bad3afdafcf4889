// Dense float64 helpers used by the geometry set-up: a tiled batched GEMM (singular-rule
// interpolation and self blocks) and a batched Gauss-Jordan inverse (block-diagonal preconditioner
// of Section 3.2).
#include <algorithm>

#include "common.cuh"

namespace rbs {

// C[b] = A[b] (M x K) * B[b] (K x N), row-major with leading dimensions; 64 x 64 tile per block,
// 256 threads, each thread a 4 x 4 sub-tile at rows ty + 16 i, columns tx + 16 j.
__global__ void __launch_bounds__(256) k_dgemm(int M, int N, int K, const double* __restrict__ A, long long lda,
                                               long long sA, const double* __restrict__ B, long long ldb,
                                               long long sB, double* __restrict__ C, long long ldc, long long sC) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ double As[BK][BM];
  __shared__ double Bs[BK][BN];
  A += sA * blockIdx.z;
  B += sB * blockIdx.z;
  C += sC * blockIdx.z;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const long long row0 = (long long)blockIdx.y * BM, col0 = (long long)blockIdx.x * BN;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int l = threadIdx.x; l < BM * BK; l += 256) {
      int r = l / BK, kk = l % BK;
      long long gr = row0 + r;
      int gk = k0 + kk;
      As[kk][r] = (gr < M && gk < K) ? A[gr * lda + gk] : 0.0;
    }
    for (int l = threadIdx.x; l < BK * BN; l += 256) {
      int kk = l / BN, cc = l % BN;
      int gk = k0 + kk;
      long long gc = col0 + cc;
      Bs[kk][cc] = (gk < K && gc < N) ? B[(long long)gk * ldb + gc] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    long long r = row0 + ty + 16 * i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      long long cidx = col0 + tx + 16 * j;
      if (cidx < N) C[r * ldc + cidx] = acc[i][j];
    }
  }
}

Status dgemm_batched(cudaStream_t s, int M, int N, int K, const double* A, long long lda, long long strideA,
                     const double* B, long long ldb, long long strideB, double* C, long long ldc, long long strideC,
                     int batch) {
  if (M <= 0 || N <= 0 || batch <= 0) return Status::Ok();
  if (batch > 65535) return Status::Err(RBS_EINVAL, "dgemm_batched: batch too large");
  dim3 grid(cdiv(N, 64), cdiv(M, 64), batch);
  k_dgemm<<<grid, 256, 0, s>>>(M, N, K, A, lda, strideA, B, ldb, strideB, C, ldc, strideC);
  RBS_CUDA_TRY(cudaGetLastError());
  return Status::Ok();
}

// In-place Gauss-Jordan inverse with partial pivoting, one block per n x n matrix.  Row k is the
// pivot row after the swap; column k of the working matrix accumulates the inverse's column, and
// the row swaps become column swaps of the result, undone at the end.  singular[b] is set to 1 when
// a pivot is exactly zero.
__global__ void __launch_bounds__(512) k_gauss_jordan(double* mats, int n, int* piv_all, int* singular) {
  extern __shared__ double sh[];
  double* col = sh;                       // n
  double* rv = col + n;                   // blockDim
  int* ri = (int*)(rv + blockDim.x);      // blockDim
  double* A = mats + (size_t)blockIdx.x * n * n;
  int* piv = piv_all + (size_t)blockIdx.x * n;
  const int tid = threadIdx.x, bd = blockDim.x;
  const int lane = tid % 32, warp = tid / 32, nw = bd / 32;
  for (int k = 0; k < n; ++k) {
    double best = -1.0;
    int bi = k;
    for (int i = k + tid; i < n; i += bd) {
      double v = fabs(A[(size_t)i * n + k]);
      if (v > best) {
        best = v;
        bi = i;
      }
    }
    rv[tid] = best;
    ri[tid] = bi;
    __syncthreads();
    for (int h = bd / 2; h > 0; h >>= 1) {
      if (tid < h) {
        double o = rv[tid + h];
        int oi = ri[tid + h];
        if (o > rv[tid] || (o == rv[tid] && oi < ri[tid])) {
          rv[tid] = o;
          ri[tid] = oi;
        }
      }
      __syncthreads();
    }
    const int p = ri[0];
    if (tid == 0) {
      piv[k] = p;
      if (rv[0] == 0.0) singular[blockIdx.x] = 1;
    }
    if (p != k)
      for (int j = tid; j < n; j += bd) {
        double t = A[(size_t)k * n + j];
        A[(size_t)k * n + j] = A[(size_t)p * n + j];
        A[(size_t)p * n + j] = t;
      }
    __syncthreads();
    const double d = 1.0 / A[(size_t)k * n + k];
    for (int i = tid; i < n; i += bd) col[i] = A[(size_t)i * n + k];
    __syncthreads();
    for (int j = tid; j < n; j += bd) A[(size_t)k * n + j] = (j == k) ? d : A[(size_t)k * n + j] * d;
    __syncthreads();
    for (int i = warp; i < n; i += nw) {
      if (i == k) continue;
      const double f = col[i];
      double* Ai = A + (size_t)i * n;
      const double* Ak = A + (size_t)k * n;
      for (int j = lane; j < n; j += 32) Ai[j] = ((j == k) ? 0.0 : Ai[j]) - f * Ak[j];
    }
    __syncthreads();
  }
  for (int k = n - 1; k >= 0; --k) {
    int p = piv[k];
    if (p != k)
      for (int i = tid; i < n; i += bd) {
        double t = A[(size_t)i * n + k];
        A[(size_t)i * n + k] = A[(size_t)i * n + p];
        A[(size_t)i * n + p] = t;
      }
    __syncthreads();
  }
}

Status invert_batched(Context& c, double* mats, int n, int count) {
  if (count <= 0) return Status::Ok();
  DevBuf<int> piv, sing;
  RBS_TRY(piv.alloc((size_t)n * count));
  RBS_TRY(sing.alloc(count));
  RBS_CUDA_TRY(cudaMemsetAsync(sing.ptr, 0, sizeof(int) * count, c.stream));
  const int threads = 512;
  size_t smem = sizeof(double) * (n + threads) + sizeof(int) * threads;
  if (smem > 48 * 1024) RBS_CUDA_TRY(cudaFuncSetAttribute(k_gauss_jordan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  for (int start = 0; start < count; start += 65535) {
    int cnt = std::min(65535, count - start);
    k_gauss_jordan<<<cnt, threads, smem, c.stream>>>(mats + (size_t)start * n * n, n, piv.ptr + (size_t)start * n,
                                                     sing.ptr + start);
    RBS_CUDA_TRY(cudaGetLastError());
  }
  std::vector<int> h(count);
  RBS_CUDA_TRY(cudaMemcpyAsync(h.data(), sing.ptr, sizeof(int) * count, cudaMemcpyDeviceToHost, c.stream));
  RBS_CUDA_TRY(cudaStreamSynchronize(c.stream));
  for (int b = 0; b < count; ++b)
    if (h[b]) return Status::Err(RBS_EINVAL, "preconditioner block is singular");
  return Status::Ok();
}

}  // namespace rbs
