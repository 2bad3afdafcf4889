// Self blocks of particles that share a body shape, applied as one GEMM on the tensor cores
// (Section 3.1, Eq. 38: the singular-quadrature blocks are computed once per shape in the body frame
// and rotated per particle; Section 4.2: their application is the dense apply of n matrices).
//
// For the n_g particles j of a shape group, with A the shape's body-frame block (3N_p x 3N_p: K0 or
// the preconditioner P0 of Section 3.2) and z_j = R_j^T x_j the body-frame input,
//     D[j, m] = sum_k Z[j, k] A[m, k],      y_j = R_j D[j, :]
// is a GEMM of M = n_g particles, N = 3N_p block rows and K = 3N_p, float16 or bfloat16 operands with
// float32 accumulation (the inner solve's arithmetic of RBS_PREC_MIXED_FP16 / _BF16).  A pack kernel
// writes Z row by row (one row per particle, zero-padded to a multiple of 64 columns; float16 rows are
// scaled by a power of two so they use the format's range); the GEMM kernel streams 128 x 64 tiles of
// Z and 240 x 64 tiles of A through a four-stage TMA pipeline with 128-byte swizzle into tcgen05 MMAs
// of 128 x 240 x 16, accumulating in tensor memory (two accumulators, so the epilogue of one tile
// overlaps the MMAs of the next), and its epilogue rotates each row back and writes y in float64.
// Warps: 0 issues the TMA loads, 1 issues the MMAs (and owns the tensor memory), 2-5 run the epilogue,
// one tensor-memory lane (one particle) per thread.  Every wait is bounded: a wait that runs out sets
// an error flag that the host reads, and the kernel drains its own copies and MMAs before it frees the
// tensor memory and returns.
#include <algorithm>
#include <cmath>
#include <cstring>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "umma.cuh"

namespace rbs {

namespace {

constexpr int kBM = 128, kBN = 240, kBK = 64, kStages = 4;
constexpr int kAccCols = 256, kTmemCols = 2 * kAccCols;
constexpr uint32_t kBytesA = kBM * kBK * 2, kBytesB = kBN * kBK * 2;
constexpr long long kSpin = 1LL << 24;
constexpr int kGemmThreads = 192;
// epilogue staging per epilogue warp: 32 rows x 48 float32 (row stride 49) and the rows' offsets,
// L moments and centres
constexpr int kEpiCols = 48, kEpiStride = 49;
static_assert(kBN % kEpiCols == 0 && kEpiCols % 16 == 0 && kEpiCols <= 64, "epilogue chunks");
constexpr size_t kEpiWarpBytes = 32 * kEpiStride * 4 + 32 * 8 + 32 * 6 * 8 + 32 * 3 * 8;
constexpr size_t kGemmSmem = 1024 + (size_t)kStages * (kBytesA + kBytesB) + 4 * kEpiWarpBytes + 256;

struct GemmEpi {
  int mode;              // kModePrecond, kModeKOnlySelf, kModeSelfKNoL or kModeSelfK
  int rows;              // particles of the group
  int np;                // nodes per particle
  const int* list;       // the group's particle ids
  const long long* offset;
  const double* rot;
  const double* centre;
  const double4* x;      // node positions (the L term)
  const double* in;      // input field (the 1/2 x term)
  const float* inv;      // per row: 1 / (row scale * block scale)
  const double* mom;     // per row: the six moments of L (kModeSelfK)
  double* out;
  double scale;
  int* err;
};

__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int* abort, long long limit) {
  for (long long i = 0; i < limit; ++i) {
    const bool done = umma::mbar_try_wait(bar, parity);
    if (__all_sync(0xffffffffu, done)) return true;
    if (__any_sync(0xffffffffu, *abort != 0)) return false;
  }
  return false;
}

__global__ void __launch_bounds__(kGemmThreads, 1)
    k_self_gemm(const __grid_constant__ CUtensorMap tmZ, const __grid_constant__ CUtensorMap tmA, int m_tiles,
                int n_tiles, int k_blocks, uint32_t idesc, GemmEpi ep) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = umma::smem_addr(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* gbase = smem_raw + (base - raw);
  const uint32_t sZ = base, sA = base + kStages * kBytesA;
  uint8_t* epi_base = gbase + kStages * (kBytesA + kBytesB);
  uint64_t* bars = reinterpret_cast<uint64_t*>(epi_base + 4 * kEpiWarpBytes);
  // barriers: full[0, S), empty[S, 2S), acc_full[2S, 2S + 2), acc_empty[2S + 2, 2S + 4), drain 2S + 4
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  auto bar = [&](int i) { return umma::smem_addr(bars + i); };
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles = m_tiles * n_tiles;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      umma::mbar_init(bar(s), 1);
      umma::mbar_init(bar(kStages + s), 1);
    }
    umma::mbar_init(bar(2 * kStages), 1);
    umma::mbar_init(bar(2 * kStages + 1), 1);
    umma::mbar_init(bar(2 * kStages + 2), 128);
    umma::mbar_init(bar(2 * kStages + 3), 128);
    umma::mbar_init(bar(2 * kStages + 4), 1);
    *abort_flag = 0;
    umma::fence_barrier_init();
  }
  if (warp == 0 && lane == 0) {
    umma::prefetch_tensormap(&tmZ);
    umma::prefetch_tensormap(&tmA);
  }
  if (warp == 1) {
    umma::tmem_alloc(umma::smem_addr(tmem_slot), kTmemCols);
    umma::tmem_relinquish();
  }
  umma::tc_fence_before();
  __syncthreads();
  umma::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // TMA producer
      int stage = 0;
      uint32_t phase = 0;
      bool used[kStages] = {};
      uint32_t last[kStages] = {};
      bool ok = true;
      for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
        const int mt = t / n_tiles, nt = t % n_tiles;
        for (int kb = 0; kb < k_blocks; ++kb) {
          if (!umma::mbar_wait(bar(kStages + stage), phase ^ 1u, abort_flag, kSpin)) {
            ok = false;
            break;
          }
          umma::mbar_arrive_expect_tx(bar(stage), kBytesA + kBytesB);
          umma::tma_load_2d(sZ + stage * kBytesA, &tmZ, bar(stage), kb * kBK, mt * kBM);
          umma::tma_load_2d(sA + stage * kBytesB, &tmA, bar(stage), kb * kBK, nt * kBN);
          used[stage] = true;
          last[stage] = phase;
          if (++stage == kStages) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok) {
        atomicExch(ep.err, 1);
        *abort_flag = 1;
      }
      // no copy of this block may still be in flight when it exits
      volatile int never = 0;
      for (int s = 0; s < kStages; ++s)
        if (used[s]) umma::mbar_wait(bar(s), last[s], &never, kSpin);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer
      int stage = 0, acc = 0;
      uint32_t phase = 0, aphase = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
        if (!umma::mbar_wait(bar(2 * kStages + 2 + acc), aphase ^ 1u, abort_flag, kSpin)) {
          ok = false;
          break;
        }
        umma::tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(acc * kAccCols);
        for (int kb = 0; kb < k_blocks; ++kb) {
          if (!umma::mbar_wait(bar(stage), phase, abort_flag, kSpin)) {
            ok = false;
            break;
          }
          umma::tc_fence_after();
          const uint64_t zd = umma::desc_k128(sZ + stage * kBytesA), ad = umma::desc_k128(sA + stage * kBytesB);
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk)
            umma::mma_f16(d, zd + 2 * kk, ad + 2 * kk, idesc, (kb | kk) != 0 ? 1u : 0u);
          umma::mma_commit(bar(kStages + stage));  // frees the stage when these MMAs are done
          if (++stage == kStages) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        umma::mma_commit(bar(2 * kStages + acc));  // the accumulator is complete
        if (++acc == 2) {
          acc = 0;
          aphase ^= 1u;
        }
      }
      if (!ok) {
        atomicExch(ep.err, 2);
        *abort_flag = 1;
      }
      // every MMA of this block has completed before the tensor memory is freed
      umma::mma_commit(bar(2 * kStages + 4));
      volatile int never = 0;
      umma::mbar_wait(bar(2 * kStages + 4), 0, &never, kSpin);
    }
  } else {
    // epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. 32 (w % 4) + 31, one particle per lane.
    // A chunk of 48 columns (16 nodes) is rotated to the lab frame in registers, staged in shared
    // memory, and written row by row, 32 and then 16 consecutive float64 per particle.
    const int q = warp & 3;
    const int r = q * 32 + lane;
    uint8_t* ew = epi_base + (warp - 2) * kEpiWarpBytes;
    float(*stage)[kEpiStride] = reinterpret_cast<float(*)[kEpiStride]>(ew);
    long long* s_off = reinterpret_cast<long long*>(ew + 32 * kEpiStride * 4);
    double(*s_mom)[6] = reinterpret_cast<double(*)[6]>(ew + 32 * kEpiStride * 4 + 32 * 8);
    double(*s_cen)[3] = reinterpret_cast<double(*)[3]>(ew + 32 * kEpiStride * 4 + 32 * 8 + 32 * 6 * 8);
    const bool half_x = ep.mode == kModeSelfK || ep.mode == kModeSelfKNoL;
    const bool with_L = ep.mode == kModeSelfK;
    int acc = 0;
    uint32_t aphase = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
      if (!warp_wait(bar(2 * kStages + acc), aphase, abort_flag, kSpin)) {
        ok = false;
        break;
      }
      umma::tc_fence_after();
      const int mt = t / n_tiles, nt = t % n_tiles;
      const int j = mt * kBM + r;
      const bool valid = j < ep.rows;
      const int row0 = mt * kBM + q * 32;  // this warp's first row
      float R[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};  // R_j / (row scale * block scale), float32
      __syncwarp();  // the previous tile's reads of the row parameters are done
      if (valid) {
        const int pid = ep.list[j];
        s_off[lane] = ep.offset[pid];
        const float inv = ep.inv[j];  // a power of two: exact in the product below
#pragma unroll
        for (int k = 0; k < 9; ++k) R[k] = (float)ep.rot[9 * pid + k] * inv;
        if (with_L) {
#pragma unroll
          for (int k = 0; k < 6; ++k) s_mom[lane][k] = ep.mom[6 * (long long)j + k];
#pragma unroll
          for (int k = 0; k < 3; ++k) s_cen[lane][k] = ep.centre[3 * pid + k];
        }
      }
      const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * kAccCols);
#pragma unroll 1
      for (int ch = 0; ch < kBN / kEpiCols; ++ch) {
        uint32_t raw[kEpiCols];
#pragma unroll
        for (int k = 0; k < kEpiCols / 16; ++k) umma::tmem_ld16_raw(taddr + kEpiCols * ch + 16 * k, raw + 16 * k);
        umma::tmem_wait_ld16(raw);
#pragma unroll
        for (int k = 1; k < kEpiCols / 16; ++k) umma::reg_fence16(raw + 16 * k);
        float v[kEpiCols];
#pragma unroll
        for (int k = 0; k < kEpiCols; ++k) v[k] = __uint_as_float(raw[k]);
        __syncwarp();  // the previous chunk's stores have read the stage
        if (valid) {
          // the lab-frame product in float32 (the 16-bit operands bound its accuracy far above float32
          // rounding; GB300's float64 rate would make this rotation the kernel's bottleneck)
#pragma unroll
          for (int u = 0; u < kEpiCols / 3; ++u) {
            const float b0 = v[3 * u], b1 = v[3 * u + 1], b2 = v[3 * u + 2];
            stage[lane][3 * u] = fmaf(R[0], b0, fmaf(R[1], b1, R[2] * b2));
            stage[lane][3 * u + 1] = fmaf(R[3], b0, fmaf(R[4], b1, R[5] * b2));
            stage[lane][3 * u + 2] = fmaf(R[6], b0, fmaf(R[7], b1, R[8] * b2));
          }
        }
        __syncwarp();
        // row by row: lane e writes entries e and 32 + e of the chunk (node e / 3, component e % 3), so
        // one row takes 32 and then 16 consecutive float64
        const bool plain = !half_x && !with_L && ep.scale == 1.0;
        const int nrows = min(32, ep.rows - row0);
#pragma unroll
        for (int h = 0; h < (kEpiCols + 31) / 32; ++h) {
          const int e = lane + 32 * h;
          const int node = nt * (kBN / 3) + ch * (kEpiCols / 3) + e / 3;
          const int comp = e % 3;
          if (e >= kEpiCols || node >= ep.np) continue;
          if (plain) {
#pragma unroll 8
            for (int rr = 0; rr < nrows; ++rr) ep.out[3 * (s_off[rr] + node) + comp] = f32_to_f64_bits(stage[rr][e]);
          } else {
            for (int rr = 0; rr < nrows; ++rr) {
              const long long gi = s_off[rr] + node;
              const float sv = stage[rr][e];
              double val = (double)sv;
              if (half_x) val += 0.5 * ep.in[3 * gi + comp];
              if (with_L) {
                const double4 pp = ep.x[gi];
                const double rx = pp.x - s_cen[rr][0], ry = pp.y - s_cen[rr][1], rz = pp.z - s_cen[rr][2];
                const double* m = s_mom[rr];
                val += comp == 0 ? m[0] + (m[4] * rz - m[5] * ry)
                                 : (comp == 1 ? m[1] + (m[5] * rx - m[3] * rz) : m[2] + (m[3] * ry - m[4] * rx));
              }
              ep.out[3 * gi + comp] = ep.scale * val;
            }
          }
        }
      }
      umma::tc_fence_before();
      umma::mbar_arrive(bar(2 * kStages + 2 + acc));
      if (++acc == 2) {
        acc = 0;
        aphase ^= 1u;
      }
    }
    if (!ok && lane == 0) {
      atomicExch(ep.err, 3);
      *abort_flag = 1;
    }
  }
  __syncthreads();
  if (warp == 1) {
    umma::tc_fence_after();
    umma::tmem_dealloc(tmem, kTmemCols);
  }
}

// Row j of Z: the body-frame input z = R^T x of particle list[j] in 16 bits (scaled by a power of two
// for float16), its inverse scale over the block's, the moments of L when asked, and aux = x for the
// preconditioner mode.  One block per particle.
__global__ void __launch_bounds__(256) k_gemm_pack(int rows, const int* __restrict__ list,
                                                   const long long* __restrict__ offset, int np, int Kp,
                                                   const double* __restrict__ rot, const double* __restrict__ centre,
                                                   const double4* __restrict__ xn, const double* __restrict__ in,
                                                   int bf16, float ascale, uint16_t* __restrict__ Z,
                                                   float* __restrict__ inv, int want_mom, double* __restrict__ mom,
                                                   double* __restrict__ aux) {
  __shared__ float red[8];
  __shared__ double redm[8][6];
  __shared__ float s_scale;
  const int j = blockIdx.x;
  if (j >= rows) return;
  const int pid = list[j];
  const long long o = offset[pid];
  const double* R = rot + 9 * pid;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float mx = 0.0f;
  double m[6] = {0, 0, 0, 0, 0, 0};
  const double cx = centre[3 * pid], cy = centre[3 * pid + 1], cz = centre[3 * pid + 2];
  for (int t = threadIdx.x; t < np; t += blockDim.x) {
    const double* xs = in + 3 * (o + t);
    const double a = xs[0], b = xs[1], c = xs[2];
    const double z0 = R[0] * a + R[3] * b + R[6] * c;
    const double z1 = R[1] * a + R[4] * b + R[7] * c;
    const double z2 = R[2] * a + R[5] * b + R[8] * c;
    mx = fmaxf(mx, fmaxf(fabsf((float)z0), fmaxf(fabsf((float)z1), fabsf((float)z2))));
    if (want_mom) {
      const double4 q = xn[o + t];
      const double rx = q.x - cx, ry = q.y - cy, rz = q.z - cz, w = q.w;
      m[0] += w * a;
      m[1] += w * b;
      m[2] += w * c;
      m[3] += w * (ry * c - rz * b);
      m[4] += w * (rz * a - rx * c);
      m[5] += w * (rx * b - ry * a);
    }
    if (aux) {
      aux[3 * (o + t)] = a;
      aux[3 * (o + t) + 1] = b;
      aux[3 * (o + t) + 2] = c;
    }
  }
  for (int d = 16; d > 0; d >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, d));
  if (want_mom)
    for (int k = 0; k < 6; ++k)
      for (int d = 16; d > 0; d >>= 1) m[k] += __shfl_xor_sync(0xffffffffu, m[k], d);
  if (lane == 0) {
    red[warp] = mx;
    for (int k = 0; k < 6; ++k) redm[warp][k] = m[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float a = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a = fmaxf(a, red[w]);
    // float16: the largest entry scaled into [2^8, 2^9); bfloat16 keeps float32's range
    int e = 0;
    frexpf(a, &e);
    const float sc = bf16 ? 1.0f : ldexpf(1.0f, 9 - e);
    s_scale = sc;
    inv[j] = 1.0f / (sc * ascale);
    if (want_mom)
      for (int k = 0; k < 6; ++k) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += redm[w][k];
        mom[6 * (long long)j + k] = s;
      }
  }
  __syncthreads();
  const float sc = s_scale;
  uint16_t* zr = Z + (long long)j * Kp;
  for (int t = threadIdx.x; t < np; t += blockDim.x) {
    const double* xs = in + 3 * (o + t);
    const double a = xs[0], b = xs[1], c = xs[2];
    const float z[3] = {(float)(R[0] * a + R[3] * b + R[6] * c), (float)(R[1] * a + R[4] * b + R[7] * c),
                        (float)(R[2] * a + R[5] * b + R[8] * c)};
    for (int q = 0; q < 3; ++q)
      zr[3 * t + q] = bf16 ? __bfloat16_as_ushort(__float2bfloat16_rn(z[q] * sc))
                           : __half_as_ushort(__float2half_rn(z[q] * sc));
  }
}

// The full body-frame block of an ellipsoid shape from its representative rows (the reflection
// symmetry A_{g(t), s} = D_g A_{t, g(s)} D_g of the grid), in 16 bits times ascale, rows 3 N_p with a
// row pitch of Kp entries (the padding stays zero).
__global__ void k_expand_block(int np, int p, int nphi, int Kp, const int* __restrict__ rep_of,
                               const int* __restrict__ g_of, const double* __restrict__ A, int bf16, double ascale,
                               uint16_t* __restrict__ out) {
  const long long dim = 3LL * np;
  const long long total = dim * dim;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int row = (int)(e / dim), col = (int)(e % dim);
    const int t = row / 3, a = row % 3, s = col / 3, b = col % 3;
    const int g = g_of[t];
    // g applied to node s: j -> p - j (bit 2), k -> -k (bit 1), k -> n_phi / 2 - k (bit 0), mod n_phi
    int js = s / nphi, ks = s % nphi;
    if (g & 4) js = p - js;
    if (g & 2) ks = ks == 0 ? 0 : nphi - ks;
    if (g & 1) ks = (nphi / 2 - ks + nphi) % nphi;
    const int gs = js * nphi + ks;
    const double sa = ((g >> a) & 1) ? -1.0 : 1.0, sb = ((g >> b) & 1) ? -1.0 : 1.0;
    const double v = sa * sb * A[(long long)(3 * rep_of[t] + a) * dim + 3 * gs + b] * ascale;
    out[(long long)row * Kp + col] = bf16 ? __bfloat16_as_ushort(__double2bfloat16(v)) : __half_as_ushort(__double2half(v));
  }
}

__global__ void k_absmax(const double* __restrict__ a, long long n, unsigned int* __restrict__ out) {
  float m = 0.0f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    m = fmaxf(m, (float)fabs(a[i]));
  for (int d = 16; d > 0; d >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, d));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));  // non-negative floats order as integers
}

template <typename T>
Status upload(DevBuf<T>& buf, const std::vector<T>& host, cudaStream_t s) {
  RBS_TRY(buf.alloc(std::max<size_t>(1, host.size())));
  if (!host.empty()) RBS_CUDA_TRY(cudaMemcpyAsync(buf.ptr, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  return Status::Ok();
}

__global__ void k_promote(const float* __restrict__ in, double* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}

Status promote_float(Context& c, const float* in, double* out, long long n) {
  k_promote<<<1024, 256, 0, c.stream>>>(in, out, n);
  RBS_CUDA_TRY(cudaGetLastError());
  return Status::Ok();
}

typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

Status encode_2d(CUtensorMap* map, bool bf16, void* base, long long inner, long long outer, long long pitch_bytes,
                 int box_inner, int box_outer) {
  static EncodeTiled fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    RBS_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    if (!p || q != cudaDriverEntryPointSuccess) return Status::Err(RBS_ECUDA, "cuTensorMapEncodeTiled unavailable");
    fn = reinterpret_cast<EncodeTiled>(p);
  }
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  const cuuint64_t strides[1] = {(cuuint64_t)pitch_bytes};
  const cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, base, dims,
                        strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return Status::Err(RBS_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return Status::Ok();
}

}  // namespace

Status build_self_gemm(Context& c) {
  c.gemm.clear();
  c.sym_rest.clear();
  c.d_sym_rest.release();
  if (!prec_16(c.opt.precision)) return Status::Ok();
  const bool bf16 = c.opt.precision == RBS_PREC_MIXED_BF16;
  cudaStream_t s = c.stream;
  std::vector<std::vector<int>> members(c.shapes.size());
  for (int i = 0; i < c.n; ++i) members[c.shape_of[i]].push_back(i);
  DevBuf<unsigned int> d_max;
  RBS_TRY(d_max.alloc(1));
  for (size_t k = 0; k < c.shapes.size(); ++k) {
    const Shape& sh = c.shapes[k];
    if (!sh.sym || (int)members[k].size() < kGemmMinParticles) {
      if (sh.sym) c.sym_rest.insert(c.sym_rest.end(), members[k].begin(), members[k].end());
      continue;
    }
    c.gemm.emplace_back(new GemmGroup());
    GemmGroup& G = *c.gemm.back();
    const Grid& g = *c.grids[sh.grid];
    G.shape = (int)k;
    G.np = sh.np;
    G.Kp = (3 * sh.np + 63) / 64 * 64;
    G.rows = (int)members[k].size();
    G.parts = members[k];
    RBS_TRY(upload(G.d_list, G.parts, s));
    RBS_TRY(G.K.alloc((size_t)3 * sh.np * G.Kp));
    RBS_TRY(G.P.alloc((size_t)3 * sh.np * G.Kp));
    RBS_TRY(G.Z.alloc((size_t)G.rows * G.Kp));
    RBS_TRY(G.inv.alloc(G.rows));
    RBS_TRY(G.mom.alloc((size_t)6 * G.rows));
    RBS_CUDA_TRY(cudaMemsetAsync(G.K.ptr, 0, sizeof(uint16_t) * G.K.n, s));
    RBS_CUDA_TRY(cudaMemsetAsync(G.P.ptr, 0, sizeof(uint16_t) * G.P.n, s));
    RBS_CUDA_TRY(cudaMemsetAsync(G.Z.ptr, 0, sizeof(uint16_t) * G.Z.n, s));
    const SymTables T = sym_tables(g);
    const long long rep_elems = (long long)sh.rows * 3 * sh.np;
    // K0 from the float32 copy's float64 source (d_blockK), P0 from the float64 preconditioner when it
    // still exists, else from its float32 copy promoted
    for (int which = 0; which < 2; ++which) {
      if (which == 1 && !c.opt.preconditioner) break;
      DevBuf<double> tmp;
      const double* src = nullptr;
      if (which == 0) {
        src = c.d_blockK.ptr + sh.block_off;
      } else {
        RBS_TRY(tmp.alloc(rep_elems));
        RBS_TRY(promote_float(c, c.d_precond32.ptr + sh.block_off, tmp.ptr, rep_elems));
        src = tmp.ptr;
      }
      float ascale = 1.0f;
      if (!bf16) {
        RBS_CUDA_TRY(cudaMemsetAsync(d_max.ptr, 0, sizeof(unsigned int), s));
        k_absmax<<<256, 256, 0, s>>>(src, rep_elems, d_max.ptr);
        unsigned int mb = 0;
        RBS_CUDA_TRY(cudaMemcpyAsync(&mb, d_max.ptr, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
        RBS_CUDA_TRY(cudaStreamSynchronize(s));
        float amax;
        std::memcpy(&amax, &mb, sizeof(float));
        int e = 0;
        std::frexp(amax, &e);
        ascale = std::ldexp(1.0f, 9 - e);
      }
      (which == 0 ? G.ascaleK : G.ascaleP) = ascale;
      k_expand_block<<<1024, 256, 0, s>>>(sh.np, g.p, g.nphi, G.Kp, T.rep_of, T.g_of, src, bf16 ? 1 : 0, ascale,
                                          which == 0 ? G.K.ptr : G.P.ptr);
      RBS_CUDA_TRY(cudaGetLastError());
      RBS_CUDA_TRY(cudaStreamSynchronize(s));
    }
    RBS_TRY(encode_2d(&G.tmZ, bf16, G.Z.ptr, G.Kp, G.rows, 2LL * G.Kp, kBK, kBM));
    RBS_TRY(encode_2d(&G.tmK, bf16, G.K.ptr, G.Kp, 3LL * sh.np, 2LL * G.Kp, kBK, kBN));
    RBS_TRY(encode_2d(&G.tmP, bf16, G.P.ptr, G.Kp, 3LL * sh.np, 2LL * G.Kp, kBK, kBN));
  }
  std::sort(c.sym_rest.begin(), c.sym_rest.end());
  RBS_TRY(upload(c.d_sym_rest, c.sym_rest, s));
  RBS_CUDA_TRY(cudaFuncSetAttribute(k_self_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem));
  if (!c.d_gemm_err.ptr) RBS_TRY(c.d_gemm_err.alloc(1));
  RBS_CUDA_TRY(cudaMemsetAsync(c.d_gemm_err.ptr, 0, sizeof(int), s));
  RBS_CUDA_TRY(cudaStreamSynchronize(s));
  return Status::Ok();
}

// The 16-bit self blocks of the shape groups by GEMM: modes kModePrecond (y = R P0 R^T x, aux = x),
// kModeKOnlySelf (R K0 R^T x), kModeSelfKNoL (+ x / 2) and kModeSelfK (+ L x), times scale.
Status apply_self_gemm(Context& c, int mode, const double* x, double* y, double* aux, double scale) {
  const bool bf16 = c.opt.precision == RBS_PREC_MIXED_BF16;
  const uint32_t idesc = umma::idesc_f16(bf16 ? 1 : 0, kBM, kBN);
  for (auto& gp : c.gemm) {
    GemmGroup& G = *gp;
    const bool pre = mode == kModePrecond;
    const float ascale = pre ? G.ascaleP : G.ascaleK;
    c.stats.launches += 2;
    k_gemm_pack<<<G.rows, 256, 0, c.stream>>>(G.rows, G.d_list.ptr, c.d_offset.ptr, G.np, G.Kp, c.d_rot.ptr,
                                              c.d_centre.ptr, c.d_x.ptr, x, bf16 ? 1 : 0, ascale, G.Z.ptr,
                                              G.inv.ptr, mode == kModeSelfK ? 1 : 0, G.mom.ptr, pre ? aux : nullptr);
    GemmEpi ep;
    ep.mode = mode;
    ep.rows = G.rows;
    ep.np = G.np;
    ep.list = G.d_list.ptr;
    ep.offset = c.d_offset.ptr;
    ep.rot = c.d_rot.ptr;
    ep.centre = c.d_centre.ptr;
    ep.x = c.d_x.ptr;
    ep.in = x;
    ep.inv = G.inv.ptr;
    ep.mom = G.mom.ptr;
    ep.out = y;
    ep.scale = scale;
    ep.err = c.d_gemm_err.ptr;
    const int m_tiles = (G.rows + kBM - 1) / kBM, n_tiles = (3 * G.np + kBN - 1) / kBN, k_blocks = G.Kp / kBK;
    const int grid = std::max(1, std::min(m_tiles * n_tiles, c.sm_count));
    const double flops = 2.0 * G.rows * (3.0 * G.np) * (3.0 * G.np);
    KernelTimer timer(c, RBS_KC_SELF_GEMM);
    k_self_gemm<<<grid, kGemmThreads, kGemmSmem, c.stream>>>(G.tmZ, pre ? G.tmP : G.tmK, m_tiles, n_tiles, k_blocks,
                                                            idesc, ep);
    RBS_CUDA_TRY(cudaGetLastError());
    timer.done(flops);
    c.stats.launches -= 1;  // counted with the pack kernel above
    G.flops += flops;
  }
  return Status::Ok();
}

// The GEMM kernel's error flag (a bounded wait that ran out): read and cleared.
Status check_self_gemm(Context& c) {
  if (c.gemm.empty() || !c.d_gemm_err.ptr) return Status::Ok();
  int e = 0;
  RBS_CUDA_TRY(cudaMemcpyAsync(&e, c.d_gemm_err.ptr, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  RBS_CUDA_TRY(cudaStreamSynchronize(c.stream));
  if (e) {
    RBS_CUDA_TRY(cudaMemsetAsync(c.d_gemm_err.ptr, 0, sizeof(int), c.stream));
    return Status::Err(RBS_ETIMEOUT, "self-block GEMM: a bounded wait ran out (role " + std::to_string(e) + ")");
  }
  return Status::Ok();
}

}  // namespace rbs
