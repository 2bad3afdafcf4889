// The mobility solve (Section 3's three steps; Algorithm 1 lines 3-5 without contact):
//   1. incident density rho (Eq. 19);
//   2. (1/2 I + K + L) mu = -(1/2 I + K) rho (Eq. 25) by GMRES (Section 3.2) with the right
//      block-diagonal preconditioner; in the mixed mode the operator of the inner GMRES is applied in
//      float32 and float64 iterative refinement recovers the float64 solution;
//   3. u = S[rho + mu] and the rigid velocities v (Eq. 41), omega (Eq. 42).
// The suspensions of a batch are solved together but converge separately: GMRES (gmres.cu) keeps a
// Krylov recursion per suspension, and the refinement of the mixed mode decides per suspension.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <mutex>

#include "common.cuh"

namespace rbs {

namespace {

// Incident density of Eq. 19 at every node.
__global__ void k_incident(long long N, const int* __restrict__ pid, const double4* __restrict__ x,
                           const double* __restrict__ centre, const double* __restrict__ area,
                           const double* __restrict__ tauinv, const double* __restrict__ FT, double* __restrict__ rho) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N; t += (long long)gridDim.x * blockDim.x) {
    const int i = pid[t];
    const double* f = FT + 6 * i;
    const double* Ti = tauinv + 9 * i;
    const double a0 = Ti[0] * f[3] + Ti[1] * f[4] + Ti[2] * f[5];
    const double a1 = Ti[3] * f[3] + Ti[4] * f[4] + Ti[5] * f[5];
    const double a2 = Ti[6] * f[3] + Ti[7] * f[4] + Ti[8] * f[5];
    const double4 p = x[t];
    const double rx = p.x - centre[3 * i], ry = p.y - centre[3 * i + 1], rz = p.z - centre[3 * i + 2];
    const double inva = 1.0 / area[i];
    rho[3 * t + 0] = f[0] * inva + (a1 * rz - a2 * ry);
    rho[3 * t + 1] = f[1] * inva + (a2 * rx - a0 * rz);
    rho[3 * t + 2] = f[2] * inva + (a0 * ry - a1 * rx);
  }
}

// Rigid velocities (Eqs. 41-42) from the surface velocity u, one block per particle; the result is
// divided by the viscosity.
__global__ void __launch_bounds__(256) k_rigid(const long long* __restrict__ offset, const double4* __restrict__ x,
                                               const double* __restrict__ centre, const double* __restrict__ area,
                                               const double* __restrict__ tauinv, const double* __restrict__ u,
                                               double inv_visc, double* __restrict__ vo) {
  __shared__ double red[8][6];
  const int i = blockIdx.x;
  const double cx = centre[3 * i], cy = centre[3 * i + 1], cz = centre[3 * i + 2];
  double m[6] = {0, 0, 0, 0, 0, 0};
  for (long long s = offset[i] + threadIdx.x; s < offset[i + 1]; s += blockDim.x) {
    const double4 p = x[s];
    const double rx = p.x - cx, ry = p.y - cy, rz = p.z - cz, w = p.w;
    const double a = u[3 * s], b = u[3 * s + 1], c = u[3 * s + 2];
    m[0] += w * a;
    m[1] += w * b;
    m[2] += w * c;
    m[3] += w * (ry * c - rz * b);
    m[4] += w * (rz * a - rx * c);
    m[5] += w * (rx * b - ry * a);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 6; ++q)
    for (int o = 16; o > 0; o >>= 1) m[q] += __shfl_xor_sync(0xffffffffu, m[q], o);
  if (lane == 0)
    for (int q = 0; q < 6; ++q) red[warp][q] = m[q];
  __syncthreads();
  if (threadIdx.x == 0) {
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
      for (int q = 0; q < 6; ++q) s[q] += red[w][q];
    const double* T = tauinv + 9 * i;
    const double ia = 1.0 / area[i];
    vo[6 * i + 0] = s[0] * ia * inv_visc;
    vo[6 * i + 1] = s[1] * ia * inv_visc;
    vo[6 * i + 2] = s[2] * ia * inv_visc;
    vo[6 * i + 3] = (T[0] * s[3] + T[1] * s[4] + T[2] * s[5]) * inv_visc;
    vo[6 * i + 4] = (T[3] * s[3] + T[4] * s[4] + T[5] * s[5]) * inv_visc;
    vo[6 * i + 5] = (T[6] * s[3] + T[7] * s[4] + T[8] * s[5]) * inv_visc;
  }
}

// y = a x + b y elementwise; x may be y (no restrict: the right-hand side's b = -b passes both)
__global__ void k_axpby(double* y, double a, const double* x, double b, long long n) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
    y[k] = a * x[k] + b * y[k];
}

// z = x + y
__global__ void k_add(double* __restrict__ z, const double* __restrict__ x, const double* __restrict__ y, long long n) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
    z[k] = x[k] + y[k];
}

}  // namespace

// ------------------------------------------------------------------------------------------
// Vector helpers and GMRES on the context stream.

static int vec_blocks(const Context& c, long long n) {
  return (int)std::min<long long>(std::max(1, 8 * c.sm_count), std::max<long long>(1, (n + 255) / 256));
}

// The operator inside GMRES: with the preconditioner, w = (1/2 I + K + L) P v = v + K_off P v
// (P the exact inverse of the particle-diagonal part), z = P v; without, w = A v.
static Status gmres_operator(Context& c, int prec, const double* v, double* w, double* z) {
  if (c.opt.preconditioner) {
    RBS_TRY(apply_blocks(c, kModePrecond, prec, v, z, w, 1.0));
    return apply_pairs(c, 0, prec, z, w);
  }
  return apply_operator(c, RBS_OP_A, prec, v, w);
}

// The mobility system's operator for the segmented GMRES: A = 1/2 I + K + L on 3N-vectors in
// arithmetic prec, right-preconditioned by the block-diagonal inverse when the context has one, one
// segment per suspension (A does not couple suspensions).  Its Arnoldi step may run as a graph.
static Status gmres(Context& c, int prec, const double* b, double* x, bool x_zero, const std::vector<double>& tol_abs,
                    int max_iters, SegResult& out) {
  LinOp op;
  op.n = 3 * c.N;
  op.graph_key = 2 * prec + (c.opt.preconditioner ? 1 : 0);
  op.apply_AP = [&c, prec](const double* v, double* w, double* z) { return gmres_operator(c, prec, v, w, z); };
  op.apply_A = [&c, prec](const double* xx, double* y) { return apply_operator(c, RBS_OP_A, prec, xx, y); };
  if (c.opt.preconditioner)
    op.apply_P = [&c, prec](const double* v, double* z, double* aux) {
      return apply_blocks(c, kModePrecond, prec, v, z, aux, 1.0);
    };
  return gmres_seg(c, op, c.seg3, b, x, x_zero, tol_abs, max_iters, out);
}

Status incident_density(Context& c, const double* FT_dev, double* rho) {
  c.stats.launches++;
  k_incident<<<vec_blocks(c, c.N), 256, 0, c.stream>>>(c.N, c.d_pid.ptr, c.d_x.ptr, c.d_centre.ptr, c.d_area.ptr,
                                                       c.d_tauinv.ptr, FT_dev, rho);
  RBS_CUDA_TRY(cudaGetLastError());
  return Status::Ok();
}

Status rigid_velocities(Context& c, const double* u, double* vo_dev) {
  c.stats.launches++;
  k_rigid<<<c.n, 256, 0, c.stream>>>(c.d_offset.ptr, c.d_x.ptr, c.d_centre.ptr, c.d_area.ptr, c.d_tauinv.ptr, u,
                                     1.0 / c.opt.viscosity, vo_dev);
  RBS_CUDA_TRY(cudaGetLastError());
  return Status::Ok();
}

// F, T: n x 3 each (host or device); FT interleaved on the device as n x 6.
__global__ void k_pack_ft(int n, const double* F, const double* T, double* FT) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int q = 0; q < 3; ++q) {
    FT[6 * i + q] = F[3 * i + q];
    FT[6 * i + 3 + q] = T[3 * i + q];
  }
}
__global__ void k_unpack_vo(int n, const double* vo, double* v, double* om) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int q = 0; q < 3; ++q) {
    v[3 * i + q] = vo[6 * i + q];
    om[3 * i + q] = vo[6 * i + 3 + q];
  }
}

// The relative error of a float32 operator application (f32_operator_error: 1e-5 for float32 pair
// sums with per-tile compensation, float32 blocks and interpolation, a bound on the measured relative
// L2 error of a few 1e-7 on the 1,000-ellipsoid p = 12 suspension, plus the treecode's model when it
// is on) decides when a refinement residual may be updated in float32.

// Float64-class residual and surface velocity of one iterate x, sharing one pass over the pairs:
// with sigma = rho + x,  r = b - A x = -(1/2 I + K) sigma - L x = L rho - A sigma  (Eq. 25, A the
// operator 1/2 I + K + L) and  u = S sigma  (the velocity of Section 2.3).
static Status residual_and_velocity(Context& c, int prec, const double* rho, const double* lrho, const double* x,
                                    double* sigma, double* r, double* u) {
  const long long n3 = 3 * c.N;
  const int nbk = vec_blocks(c, n3);
  c.stats.launches++;
  k_add<<<nbk, 256, 0, c.stream>>>(sigma, rho, x, n3);
  RBS_TRY(apply_blocks(c, kModeSelfK, prec, sigma, r, nullptr, 1.0));
  RBS_TRY(apply_blocks(c, kModeSelfS, prec, sigma, u, nullptr, 1.0));
  RBS_TRY(apply_pairs_both(c, prec, sigma, r, u));
  c.stats.launches++;
  k_axpby<<<nbk, 256, 0, c.stream>>>(r, 1.0, lrho, -1.0, n3);
  RBS_CUDA_TRY(cudaGetLastError());
  return Status::Ok();
}

// One mobility solve of the forces and torques in c.d_FT (n x 6, device) in the context's arithmetic:
// the scattered density in d_vec[2] and the rigid velocities in c.d_vo (n x 6).  `warm` allows the
// configured warm start.  Every suspension converges on its own right-hand side: its GMRES iterations
// are added to iters[s] and its final relative residual ||b_s - A mu_s|| / ||b_s|| goes to rel[s].
static Status solve_core(Context& c, double tol, bool warm, std::vector<int>& iters, std::vector<double>& rel,
                         int* refinements_out, bool* converged_out) {
  const long long n3 = 3 * c.N;
  const int nbk = vec_blocks(c, n3);
  const int S = c.seg3.S;
  double* rho = c.d_vec[0].ptr;
  double* b = c.d_vec[1].ptr;
  double* x = c.d_vec[2].ptr;
  double* r = c.d_vec[3].ptr;
  double* d = c.d_vec[7].ptr;
  iters.resize(S, 0);
  rel.assign(S, 0.0);
  // 1. incident density; right-hand side b = -(1/2 I + K) rho (Eq. 25): float64 for the float64 path;
  //    float32 for the mixed path, where b only seeds the first inner solve (every refinement residual
  //    below is formed from rho in float64-class arithmetic, so b's float32 error does not persist)
  RBS_TRY(incident_density(c, c.d_FT.ptr, rho));
  const bool mixed = prec_f32(c.opt.precision);
  const int hi = mixed ? c.opt.refine_precision : RBS_PREC_FP64;
  RBS_TRY(apply_operator(c, RBS_OP_HALF_K, mixed ? RBS_PREC_MIXED : RBS_PREC_FP64, rho, b));
  c.stats.launches++;
  k_axpby<<<nbk, 256, 0, c.stream>>>(b, 0.0, b, -1.0, n3);
  std::vector<double> bn;
  RBS_TRY(seg_norms_host(c, c.seg3, b, bn));
  double bmax = 0.0;
  for (double v : bn) bmax = std::max(bmax, v);
  int refinements = 0;
  bool converged = true;
  // initial guess: zero, the previous solution, or the learned warm start
  bool have_x0 = false;
  double* x0 = d;
  if (warm && bmax > 0.0 && c.opt.warm_start == RBS_WARM_PREVIOUS && c.have_prev && c.d_prev.n == (size_t)n3) {
    RBS_CUDA_TRY(cudaMemcpyAsync(x0, c.d_prev.ptr, sizeof(double) * n3, cudaMemcpyDeviceToDevice, c.stream));
    have_x0 = true;
  } else if (warm && bmax > 0.0 && c.opt.warm_start == RBS_WARM_LEARNED) {
    RBS_TRY(warm_guess(c, c.d_FT.ptr, x0));
    have_x0 = true;
  } else if (warm && bmax > 0.0 && c.opt.warm_start == RBS_WARM_LEARNED_DELTA) {
    // x0 = mu_prev + (net(now) - net(prev)): the network's guess for the current configuration, shifted
    // by its error at the last solved configuration; the network's guess alone without a last solve
    RBS_TRY(warm_guess(c, c.d_FT.ptr, x0));
    const bool have_pred = c.have_prev && c.d_prev.n == (size_t)n3 && c.d_pred_prev.n == (size_t)n3 && c.have_pred;
    if (c.d_pred_prev.n != (size_t)n3) RBS_TRY(c.d_pred_prev.alloc(n3));
    double* tmp = c.d_vec[5].ptr;
    if (have_pred) {
      // tmp = x0 - pred_prev + prev; pred_prev = x0
      c.stats.launches += 2;
      k_add<<<nbk, 256, 0, c.stream>>>(tmp, x0, c.d_prev.ptr, n3);
      k_axpby<<<nbk, 256, 0, c.stream>>>(tmp, -1.0, c.d_pred_prev.ptr, 1.0, n3);
      RBS_CUDA_TRY(cudaMemcpyAsync(c.d_pred_prev.ptr, x0, sizeof(double) * n3, cudaMemcpyDeviceToDevice, c.stream));
      RBS_CUDA_TRY(cudaMemcpyAsync(x0, tmp, sizeof(double) * n3, cudaMemcpyDeviceToDevice, c.stream));
    } else {
      RBS_CUDA_TRY(cudaMemcpyAsync(c.d_pred_prev.ptr, x0, sizeof(double) * n3, cudaMemcpyDeviceToDevice, c.stream));
      c.have_pred = true;
    }
    have_x0 = true;
  }
  double* sigma = c.d_vec[9].ptr;
  double* u = c.d_vec[1].ptr;  // b's storage once b has been used
  double* w = c.d_vec[4].ptr;
  bool u_done = false;
  // 2. the scattered density
  if (bmax == 0.0) {
    RBS_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * n3, c.stream));
  } else if (!mixed) {
    if (have_x0) RBS_CUDA_TRY(cudaMemcpyAsync(x, x0, sizeof(double) * n3, cudaMemcpyDeviceToDevice, c.stream));
    std::vector<double> tl(S);
    for (int s = 0; s < S; ++s) tl[s] = tol * bn[s];
    SegResult R;
    RBS_TRY(gmres(c, RBS_PREC_FP64, b, x, !have_x0, tl, c.opt.max_iters, R));
    for (int s = 0; s < S; ++s) {
      iters[s] += R.iters[s];
      rel[s] = bn[s] > 0.0 ? R.res[s] / bn[s] : 0.0;
      if (!R.conv[s]) converged = false;
    }
  } else {
    // Iterative refinement around float32 inner solves.  A float64-class pass gives the true
    // residual r = b - A x and, from the same pair sums, u = S[rho + x].  After a pass, a small
    // correction d may instead update r -= A d and u += S d in float32: the float32 operator's error
    // on d is f32_operator_error ||A d||, and these updates are taken only while that error, summed
    // since the last pass, stays below a tenth of the tolerance in every suspension the correction
    // touched.  Suspensions within tolerance after a float64-class pass take no further inner
    // iterations.
    double* lrho = c.d_vec[8].ptr;  // L rho (Eq. 26), float64
    RBS_TRY(apply_blocks(c, kModeL, RBS_PREC_FP64, rho, lrho, nullptr, 1.0));
    std::vector<double> rn = bn;
    if (have_x0) {
      // the first inner solve starts from the warm start's residual in float32 arithmetic, like a
      // zero start from b; the float64-class pass follows it
      RBS_CUDA_TRY(cudaMemcpyAsync(x, x0, sizeof(double) * n3, cudaMemcpyDeviceToDevice, c.stream));
      RBS_TRY(apply_operator(c, RBS_OP_A, RBS_PREC_MIXED, x, w));
      RBS_CUDA_TRY(cudaMemcpyAsync(r, b, sizeof(double) * n3, cudaMemcpyDeviceToDevice, c.stream));
      c.stats.launches++;
      k_axpby<<<nbk, 256, 0, c.stream>>>(r, -1.0, w, 1.0, n3);
      RBS_TRY(seg_norms_host(c, c.seg3, r, rn));
    } else {
      RBS_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * n3, c.stream));
      RBS_CUDA_TRY(cudaMemcpyAsync(r, b, sizeof(double) * n3, cudaMemcpyDeviceToDevice, c.stream));
    }
    // sigma accumulates the corrections applied in float32 since the last float64-class pass
    std::vector<double> pending(S, 0.0);
    std::vector<int> used(S, 0);
    const double ferr = f32_operator_error(c);
    converged = false;
    int used_max = 0;
    while (!converged && refinements < c.opt.max_refinements && used_max < c.opt.max_iters) {
      // each inner solve reduces a suspension's residual by inner_tol, or only as far as the final
      // tolerance needs (half of tol ||b_s||), whichever is looser; suspensions already within
      // tolerance after a float64-class pass are left out
      std::vector<double> tl(S);
      for (int s = 0; s < S; ++s) {
        if (u_done && rn[s] <= tol * bn[s]) {
          tl[s] = INFINITY;
        } else {
          const double need = rn[s] > 0.0 ? 0.5 * tol * bn[s] / rn[s] : 1.0;
          tl[s] = std::min(0.5, std::max(c.opt.inner_tol, need)) * rn[s];
        }
      }
      SegResult R;
      // the inner operator: float32 pair sums, self blocks in the context's inner arithmetic
      RBS_TRY(gmres(c, c.opt.precision, r, d, true, tl, c.opt.max_iters - used_max, R));
      int moved = 0;
      for (int s = 0; s < S; ++s) {
        iters[s] += R.iters[s];
        used[s] += R.iters[s];
        used_max = std::max(used_max, used[s]);
        moved = std::max(moved, R.iters[s]);
      }
      ++refinements;
      c.stats.launches++;
      k_axpby<<<nbk, 256, 0, c.stream>>>(x, 1.0, d, 1.0, n3);
      bool f32_ok = u_done;
      for (int s = 0; s < S && f32_ok; ++s)
        if (R.iters[s] > 0 && ferr * (pending[s] + rn[s]) > 0.1 * tol * bn[s]) f32_ok = false;
      if (f32_ok) {
        RBS_TRY(apply_operator(c, RBS_OP_A, RBS_PREC_MIXED, d, w));
        c.stats.launches += 2;
        k_axpby<<<nbk, 256, 0, c.stream>>>(r, -1.0, w, 1.0, n3);
        k_axpby<<<nbk, 256, 0, c.stream>>>(sigma, 1.0, d, 1.0, n3);
        for (int s = 0; s < S; ++s)
          if (R.iters[s] > 0) pending[s] += rn[s];
      } else {
        RBS_TRY(residual_and_velocity(c, hi, rho, lrho, x, sigma, r, u));
        u_done = true;
        RBS_CUDA_TRY(cudaMemsetAsync(sigma, 0, sizeof(double) * n3, c.stream));
        std::fill(pending.begin(), pending.end(), 0.0);
      }
      RBS_TRY(seg_norms_host(c, c.seg3, r, rn));
      converged = u_done;
      for (int s = 0; s < S; ++s)
        if (!(rn[s] <= tol * bn[s])) converged = false;
      if (moved == 0) break;  // the inner solves could not move
    }
    for (int s = 0; s < S; ++s) rel[s] = bn[s] > 0.0 ? rn[s] / bn[s] : 0.0;
    bool any_pending = false;
    for (double p : pending) any_pending = any_pending || p > 0.0;
    if (u_done && any_pending) {
      RBS_TRY(apply_operator(c, RBS_OP_S, RBS_PREC_MIXED, sigma, w));
      c.stats.launches++;
      k_axpby<<<nbk, 256, 0, c.stream>>>(u, 1.0, w, 1.0, n3);
    }
  }
  // 3. u = S[rho + mu] (already formed by the mixed path's float64-class passes) and the rigid velocities
  if (!u_done) {
    c.stats.launches++;
    k_add<<<nbk, 256, 0, c.stream>>>(sigma, rho, x, n3);
    RBS_TRY(apply_operator(c, RBS_OP_S, hi, sigma, u));
  }
  RBS_TRY(rigid_velocities(c, u, c.d_vo.ptr));
  RBS_CUDA_TRY(cudaGetLastError());
  *refinements_out = refinements;
  *converged_out = converged;
  return Status::Ok();
}

// ------------------------------------------------------------------------------------------
// Contact force algorithm (Section 3.4).  Candidates are near pairs i < j of one suspension whose
// bounding spheres come within the gap; for each, the closest pair of upsampled nodes decides.

// Closest pair of upsampled nodes of two particles, one block (256 threads) per candidate pair.
// Squared distances are formed with every product and sum rounded once (no fused multiply-add), and
// ties go to the first pair in node order (a * n_b + b smallest).
__global__ void __launch_bounds__(256) k_closest_nodes(const int2* __restrict__ pairs,
                                                       const long long* __restrict__ up_off,
                                                       const int* __restrict__ up_index,
                                                       const double4* __restrict__ up_x, double* __restrict__ d2_out,
                                                       long long* __restrict__ arg_out) {
  __shared__ double sd[256];
  __shared__ long long sk[256];
  const int2 pr = pairs[blockIdx.x];
  const int ua = up_index[pr.x], ub = up_index[pr.y];
  const long long oa = up_off[ua], ob = up_off[ub];
  const long long na = up_off[ua + 1] - oa, nb = up_off[ub + 1] - ob;
  double best = INFINITY;
  long long bk = LLONG_MAX;
  for (long long k = threadIdx.x; k < na * nb; k += blockDim.x) {
    const long long a = k / nb, b = k - (k / nb) * nb;
    const double4 p = up_x[oa + a], q = up_x[ob + b];
    const double dx = __dsub_rn(p.x, q.x), dy = __dsub_rn(p.y, q.y), dz = __dsub_rn(p.z, q.z);
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    if (d2 < best || (d2 == best && k < bk)) {
      best = d2;
      bk = k;
    }
  }
  sd[threadIdx.x] = best;
  sk[threadIdx.x] = bk;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      const double o = sd[threadIdx.x + h];
      const long long ok = sk[threadIdx.x + h];
      if (o < sd[threadIdx.x] || (o == sd[threadIdx.x] && ok < sk[threadIdx.x])) {
        sd[threadIdx.x] = o;
        sk[threadIdx.x] = ok;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    d2_out[blockIdx.x] = sd[0];
    arg_out[blockIdx.x] = sk[0];
  }
}

// Contacts of the current configuration into c.contacts (ascending (i, j)).
static Status find_contacts(Context& c) {
  c.contacts.clear();
  std::vector<int2> cand;
  for (const int2& pr : c.near_pairs) {
    if (pr.x >= pr.y) continue;
    const double dx = c.centres[3 * pr.x] - c.centres[3 * pr.y], dy = c.centres[3 * pr.x + 1] - c.centres[3 * pr.y + 1],
                 dz = c.centres[3 * pr.x + 2] - c.centres[3 * pr.y + 2];
    const double R = c.shapes[c.shape_of[pr.x]].radius + c.shapes[c.shape_of[pr.y]].radius;
    if (std::sqrt(dx * dx + dy * dy + dz * dz) < R + c.opt.contact_gap) cand.push_back(pr);
  }
  if (cand.empty()) return Status::Ok();
  std::sort(cand.begin(), cand.end(), [](int2 a, int2 b) { return a.x != b.x ? a.x < b.x : a.y < b.y; });
  DevBuf<int2> d_cand;
  DevBuf<double> d_d2;
  DevBuf<long long> d_arg;
  RBS_TRY(d_cand.alloc(cand.size()));
  RBS_TRY(d_d2.alloc(cand.size()));
  RBS_TRY(d_arg.alloc(cand.size()));
  RBS_CUDA_TRY(cudaMemcpyAsync(d_cand.ptr, cand.data(), sizeof(int2) * cand.size(), cudaMemcpyHostToDevice, c.stream));
  c.stats.launches++;
  k_closest_nodes<<<(unsigned)cand.size(), 256, 0, c.stream>>>(d_cand.ptr, c.d_up_off.ptr, c.d_up_index.ptr,
                                                              c.d_up_x.ptr, d_d2.ptr, d_arg.ptr);
  RBS_CUDA_TRY(cudaGetLastError());
  std::vector<double> d2(cand.size());
  std::vector<long long> arg(cand.size());
  RBS_CUDA_TRY(cudaMemcpyAsync(d2.data(), d_d2.ptr, sizeof(double) * d2.size(), cudaMemcpyDeviceToHost, c.stream));
  RBS_CUDA_TRY(cudaMemcpyAsync(arg.data(), d_arg.ptr, sizeof(long long) * arg.size(), cudaMemcpyDeviceToHost, c.stream));
  RBS_CUDA_TRY(cudaStreamSynchronize(c.stream));
  for (size_t q = 0; q < cand.size(); ++q) {
    if (!(std::sqrt(d2[q]) < c.opt.contact_gap)) continue;
    const int ua = c.up_index[cand[q].x], ub = c.up_index[cand[q].y];
    const long long nb = c.up_offset[ub + 1] - c.up_offset[ub];
    const long long a = arg[q] / nb, b = arg[q] % nb;
    double4 pa, pb;
    RBS_CUDA_TRY(cudaMemcpy(&pa, c.d_up_x.ptr + c.up_offset[ua] + a, sizeof(double4), cudaMemcpyDeviceToHost));
    RBS_CUDA_TRY(cudaMemcpy(&pb, c.d_up_x.ptr + c.up_offset[ub] + b, sizeof(double4), cudaMemcpyDeviceToHost));
    Context::Contact ct;
    ct.i = cand[q].x;
    ct.j = cand[q].y;
    ct.x[0] = 0.5 * (pa.x + pb.x);
    ct.x[1] = 0.5 * (pa.y + pb.y);
    ct.x[2] = 0.5 * (pa.z + pb.z);
    ct.f[0] = ct.f[1] = ct.f[2] = 0.0;
    c.contacts.push_back(ct);
  }
  return Status::Ok();
}

// Column 3 k + a of C (n x 6 forces and torques of a unit force along axis a at contact k) added,
// times s, into FT.
static void add_contact_column(const Context& c, int k, int a, double s, std::vector<double>& FT) {
  const Context::Contact& ct = c.contacts[k];
  double f[3] = {0.0, 0.0, 0.0};
  f[a] = s;
  for (int side = 0; side < 2; ++side) {
    const int p = side == 0 ? ct.i : ct.j;
    const double sg = side == 0 ? 1.0 : -1.0;
    const double r[3] = {ct.x[0] - c.centres[3 * p], ct.x[1] - c.centres[3 * p + 1], ct.x[2] - c.centres[3 * p + 2]};
    FT[6 * p + 0] += sg * f[0];
    FT[6 * p + 1] += sg * f[1];
    FT[6 * p + 2] += sg * f[2];
    FT[6 * p + 3] += sg * (r[1] * f[2] - r[2] * f[1]);
    FT[6 * p + 4] += sg * (r[2] * f[0] - r[0] * f[2]);
    FT[6 * p + 5] += sg * (r[0] * f[1] - r[1] * f[0]);
  }
}

// Velocity difference at contact k from the rigid velocities V (n x 6): v_i + w_i x r_i - v_j - w_j x r_j.
static void contact_slip(const Context& c, int k, const std::vector<double>& V, double out[3]) {
  const Context::Contact& ct = c.contacts[k];
  for (int q = 0; q < 3; ++q) out[q] = 0.0;
  for (int side = 0; side < 2; ++side) {
    const int p = side == 0 ? ct.i : ct.j;
    const double sg = side == 0 ? 1.0 : -1.0;
    const double r[3] = {ct.x[0] - c.centres[3 * p], ct.x[1] - c.centres[3 * p + 1], ct.x[2] - c.centres[3 * p + 2]};
    const double* v = &V[6 * p];
    out[0] += sg * (v[0] + v[4] * r[2] - v[5] * r[1]);
    out[1] += sg * (v[1] + v[5] * r[0] - v[3] * r[2]);
    out[2] += sg * (v[2] + v[3] * r[1] - v[4] * r[0]);
  }
}

// Dense solve of A x = y (m x m, row-major) by Gaussian elimination with partial pivoting.
static Status dense_solve(std::vector<double> A, std::vector<double>& y, int m) {
  for (int k = 0; k < m; ++k) {
    int piv = k;
    for (int r = k + 1; r < m; ++r)
      if (std::fabs(A[(size_t)r * m + k]) > std::fabs(A[(size_t)piv * m + k])) piv = r;
    if (!(std::fabs(A[(size_t)piv * m + k]) > 0.0)) return Status::Err(RBS_ENOTCONV, "contact system is singular");
    if (piv != k) {
      for (int q = 0; q < m; ++q) std::swap(A[(size_t)k * m + q], A[(size_t)piv * m + q]);
      std::swap(y[k], y[piv]);
    }
    for (int r = k + 1; r < m; ++r) {
      const double f = A[(size_t)r * m + k] / A[(size_t)k * m + k];
      for (int q = k; q < m; ++q) A[(size_t)r * m + q] -= f * A[(size_t)k * m + q];
      y[r] -= f * y[k];
    }
  }
  for (int k = m - 1; k >= 0; --k) {
    double acc = y[k];
    for (int q = k + 1; q < m; ++q) acc -= A[(size_t)k * m + q] * y[q];
    y[k] = acc / A[(size_t)k * m + k];
  }
  return Status::Ok();
}

// Contact correction of the solve just made (its forces in c.d_FT, velocities in c.d_vo): the
// columns M C from 3 n_c solves, the contact forces from (D M C) F_c = -D V_0, and a final solve with
// the forces and torques F + C F_c, which gives the corrected velocities and density together.
static Status contact_correction(Context& c, double tol) {
  RBS_TRY(find_contacts(c));
  c.stats.n_contacts = (int)c.contacts.size();
  const int nc = (int)c.contacts.size();
  if (nc == 0) return Status::Ok();
  const int n = c.n, m = 3 * nc;
  std::vector<double> V0(6 * (size_t)n), FT0(6 * (size_t)n);
  RBS_CUDA_TRY(cudaMemcpyAsync(V0.data(), c.d_vo.ptr, sizeof(double) * V0.size(), cudaMemcpyDeviceToHost, c.stream));
  RBS_CUDA_TRY(cudaMemcpyAsync(FT0.data(), c.d_FT.ptr, sizeof(double) * FT0.size(), cudaMemcpyDeviceToHost, c.stream));
  RBS_CUDA_TRY(cudaStreamSynchronize(c.stream));
  std::vector<double> DMC((size_t)m * m), rhs(m), Vk(6 * (size_t)n), FT(6 * (size_t)n);
  for (int col = 0; col < m; ++col) {
    std::fill(FT.begin(), FT.end(), 0.0);
    add_contact_column(c, col / 3, col % 3, 1.0, FT);
    RBS_CUDA_TRY(cudaMemcpyAsync(c.d_FT.ptr, FT.data(), sizeof(double) * FT.size(), cudaMemcpyHostToDevice, c.stream));
    int refs = 0;
    bool conv = false;
    std::vector<double> rel;
    RBS_TRY(solve_core(c, tol, false, c.susp_iters, rel, &refs, &conv));
    if (!conv) return Status::Err(RBS_ENOTCONV, "a contact column solve did not converge");
    RBS_CUDA_TRY(cudaMemcpyAsync(Vk.data(), c.d_vo.ptr, sizeof(double) * Vk.size(), cudaMemcpyDeviceToHost, c.stream));
    RBS_CUDA_TRY(cudaStreamSynchronize(c.stream));
    for (int k = 0; k < nc; ++k) {
      double s[3];
      contact_slip(c, k, Vk, s);
      for (int q = 0; q < 3; ++q) DMC[(size_t)(3 * k + q) * m + col] = s[q];
    }
  }
  for (int k = 0; k < nc; ++k) {
    double s[3];
    contact_slip(c, k, V0, s);
    for (int q = 0; q < 3; ++q) rhs[3 * k + q] = -s[q];
  }
  RBS_TRY(dense_solve(DMC, rhs, m));
  FT = FT0;
  for (int col = 0; col < m; ++col) add_contact_column(c, col / 3, col % 3, rhs[col], FT);
  for (int k = 0; k < nc; ++k)
    for (int q = 0; q < 3; ++q) c.contacts[k].f[q] = rhs[3 * k + q];
  RBS_CUDA_TRY(cudaMemcpyAsync(c.d_FT.ptr, FT.data(), sizeof(double) * FT.size(), cudaMemcpyHostToDevice, c.stream));
  int refs = 0;
  bool conv = false;
  RBS_TRY(solve_core(c, tol, false, c.susp_iters, c.susp_res, &refs, &conv));
  if (!conv) return Status::Err(RBS_ENOTCONV, "the contact-corrected solve did not converge");
  return Status::Ok();
}

Status mobility_solve(Context& c, const double* F, const double* T, double tol, double* v, double* om, double* density,
                      int* iters_out, bool device_io) {
  auto t0 = std::chrono::steady_clock::now();
  const long long n3 = 3 * c.N;
  const int n = c.n;
  double* x = c.d_vec[2].ptr;
  // forces and torques to the device (n x 6)
  if (device_io) {
    c.stats.launches++;
    k_pack_ft<<<cdiv(n, 128), 128, 0, c.stream>>>(n, F, T, c.d_FT.ptr);
  } else {
    // staged through the velocity buffer: F then T, then packed
    RBS_CUDA_TRY(cudaMemcpyAsync(c.d_vo.ptr, F, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, c.stream));
    RBS_CUDA_TRY(cudaMemcpyAsync(c.d_vo.ptr + 3 * n, T, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, c.stream));
    c.stats.launches++;
    k_pack_ft<<<cdiv(n, 128), 128, 0, c.stream>>>(n, c.d_vo.ptr, c.d_vo.ptr + 3 * n, c.d_FT.ptr);
  }
  RBS_CUDA_TRY(cudaGetLastError());
  int refinements = 0;
  bool converged = false;
  c.susp_iters.assign(c.seg3.S, 0);
  RBS_TRY(solve_core(c, tol, true, c.susp_iters, c.susp_res, &refinements, &converged));
  c.stats.n_contacts = 0;
  c.contacts.clear();
  if (converged && c.opt.contact_gap > 0.0) RBS_TRY(contact_correction(c, tol));
  int total_iters = 0;
  double rel = 0.0;
  for (int v : c.susp_iters) total_iters = std::max(total_iters, v);
  for (double v : c.susp_res) rel = std::max(rel, v);
  // keep the density for a previous-solution warm start and for recording training samples
  if (c.d_prev.n != (size_t)n3) RBS_TRY(c.d_prev.alloc(n3));
  RBS_CUDA_TRY(cudaMemcpyAsync(c.d_prev.ptr, x, sizeof(double) * n3, cudaMemcpyDeviceToDevice, c.stream));
  c.have_prev = true;
  if (device_io) {
    c.stats.launches++;
    k_unpack_vo<<<cdiv(n, 128), 128, 0, c.stream>>>(n, c.d_vo.ptr, v, om);
    if (density) RBS_CUDA_TRY(cudaMemcpyAsync(density, x, sizeof(double) * n3, cudaMemcpyDeviceToDevice, c.stream));
    RBS_CUDA_TRY(cudaStreamSynchronize(c.stream));
  } else {
    double* tmp = c.d_FT.ptr;  // reuse: n x 6 -> v (n x 3) then omega (n x 3)
    c.stats.launches++;
    k_unpack_vo<<<cdiv(n, 128), 128, 0, c.stream>>>(n, c.d_vo.ptr, tmp, tmp + 3 * n);
    RBS_CUDA_TRY(cudaMemcpyAsync(v, tmp, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c.stream));
    RBS_CUDA_TRY(cudaMemcpyAsync(om, tmp + 3 * n, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c.stream));
    if (density) RBS_CUDA_TRY(cudaMemcpyAsync(density, x, sizeof(double) * n3, cudaMemcpyDeviceToHost, c.stream));
    RBS_CUDA_TRY(cudaStreamSynchronize(c.stream));
  }
  RBS_CUDA_TRY(cudaGetLastError());
  RBS_TRY(check_self_gemm(c));
  if (iters_out) *iters_out = total_iters;
  c.stats.iterations = total_iters;
  c.stats.refinements = refinements;
  c.stats.residual = rel;
  c.stats.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (!converged)
    return Status::Err(RBS_ENOTCONV, "GMRES stopped at relative residual " + std::to_string(rel) + " after " +
                                         std::to_string(total_iters) + " iterations");
  return Status::Ok();
}

}  // namespace rbs

// ------------------------------------------------------------------------------------------
// Allocation-free rigid velocities.  Some callers may not allocate device memory when they call in:
// frameworks that reserve nearly all device memory for their own pool up front (so a cudaMalloc from a
// library they call would fail), real-time time-stepping loops that forbid allocator calls, and hosts
// that hand the library a fixed memory budget.  For them rbs_rigid_velocities_noalloc reads u and
// writes v and omega in caller buffers, and keeps its one intermediate (the interleaved n x 6 result of
// the per-particle reduction) in the fixed device array below instead of a context buffer.
namespace rbs {
namespace {

constexpr int kNoAllocMaxParticles = 65536;  // 65,536 x 6 float64 = 3 MiB per device
static __device__ __align__(256) double g_rigid_scratch[6 * kNoAllocMaxParticles];

std::mutex g_scratch_mutex;
double* g_scratch_addr[64] = {};  // device address of g_rigid_scratch, per device ordinal

// Host code may not pass g_rigid_scratch to a kernel directly (its name is a host-side stand-in);
// the device address is looked up once per device, with that device current.
Status rigid_scratch(int device, double** out) {
  if (device < 0 || device >= 64) return Status::Err(RBS_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    RBS_CUDA_TRY(cudaGetSymbolAddress(&p, g_rigid_scratch));
    g_scratch_addr[device] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[device];
  return Status::Ok();
}

}  // namespace
}  // namespace rbs

extern "C" int rbs_rigid_velocities_noalloc(rbs_ctx* h, const double* u_dev, double* v_dev, double* omega_dev) {
  if (!h) return RBS_EINVAL;
  rbs::Context& c = h->c;
  auto fail = [&](const rbs::Status& s) {
    c.err = s.msg;
    return s.code;
  };
  if (!c.have_geometry) return fail(rbs::Status::Err(RBS_ESTATE, "no geometry"));
  if (!u_dev || !v_dev || !omega_dev) return fail(rbs::Status::Err(RBS_EINVAL, "rigid_velocities_noalloc: null pointer"));
  if (c.n > rbs::kNoAllocMaxParticles)
    return fail(rbs::Status::Err(RBS_EINVAL, "rigid_velocities_noalloc: " + std::to_string(c.n) +
                                                 " particles exceed the fixed scratch limit of " +
                                                 std::to_string(rbs::kNoAllocMaxParticles)));
  // the work runs on the context's device; the caller's current device is put back before returning
  int prev_device = -1;
  cudaError_t e = cudaGetDevice(&prev_device);
  if (e != cudaSuccess) return fail(rbs::Status::Err(RBS_ECUDA, cudaGetErrorString(e)));
  auto restore = [&](int code) {
    if (prev_device >= 0 && prev_device != c.device) cudaSetDevice(prev_device);
    return code;
  };
  e = cudaSetDevice(c.device);
  if (e != cudaSuccess) return restore(fail(rbs::Status::Err(RBS_ECUDA, cudaGetErrorString(e))));
  double* scratch = nullptr;
  rbs::Status s = rbs::rigid_scratch(c.device, &scratch);
  if (!s.ok()) return restore(fail(s));
  // every scratch entry read below is written first by k_rigid, so nothing needs clearing
  rbs::k_rigid<<<c.n, 256, 0, c.stream>>>(c.d_offset.ptr, c.d_x.ptr, c.d_centre.ptr, c.d_area.ptr, c.d_tauinv.ptr,
                                         u_dev, 1.0 / c.opt.viscosity, scratch);
  rbs::k_unpack_vo<<<rbs::cdiv(c.n, 128), 128, 0, c.stream>>>(c.n, scratch, v_dev, omega_dev);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess)
    return restore(fail(rbs::Status::Err(RBS_ECUDA, std::string("rigid_velocities_noalloc: ") + cudaGetErrorString(e))));
  c.stats.launches += 2;
  c.err.clear();
  return restore(RBS_OK);
}
