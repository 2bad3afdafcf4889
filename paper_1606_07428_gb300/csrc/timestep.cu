// Rigid-body time stepping (Section 3.3, Eqs. 40 and 43; Algorithm 1): explicit Runge-Kutta steps of
// dc_i/dt = v_i and dq_i/dt = 1/2 (0, omega_i) q_i (Hamilton product) with the forces and torques held
// fixed; each stage is one mobility solve at the stage configuration, whose self blocks are the
// body-frame blocks rotated by R(q) (Eq. 38), followed by the contact correction of Section 3.4 when
// rbs_options.contact_gap > 0; with a magnetic field and mu_ratio != 1 in the options, each stage first
// adds the particles' magnetic forces and torques (Section 4.1.3).  Quaternions are renormalised after
// each step.
#include <vector>

#include "common.cuh"

namespace rbs {

namespace {

// k = (v, 1/2 (0, omega) q) for every particle; vo is n x 6, state and k are n x 7 (c, q).
__global__ void k_rk_rates(int n, const double* __restrict__ vo, const double* __restrict__ state, double* __restrict__ k) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* q = state + 7 * i + 3;
  const double wx = vo[6 * i + 3], wy = vo[6 * i + 4], wz = vo[6 * i + 5];
  double* o = k + 7 * i;
  o[0] = vo[6 * i + 0];
  o[1] = vo[6 * i + 1];
  o[2] = vo[6 * i + 2];
  // (0, w) (x) (q0, q1, q2, q3)
  o[3] = 0.5 * (-wx * q[1] - wy * q[2] - wz * q[3]);
  o[4] = 0.5 * (wx * q[0] + wy * q[3] - wz * q[2]);
  o[5] = 0.5 * (-wx * q[3] + wy * q[0] + wz * q[1]);
  o[6] = 0.5 * (wx * q[2] - wy * q[1] + wz * q[0]);
}

// out = base + dt * sum_s coef[s] k_s (n x 7 each); optionally renormalise the quaternion part.
__global__ void k_rk_combine(int n, const double* __restrict__ base, const double* __restrict__ ks, int nstage,
                             double c0, double c1, double c2, double c3, double dt, int normalize, double* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double coef[4] = {c0, c1, c2, c3};
  double v[7];
  for (int q = 0; q < 7; ++q) {
    double acc = base[7 * i + q];
    for (int s = 0; s < nstage; ++s) acc += dt * coef[s] * ks[(size_t)s * 7 * n + 7 * i + q];
    v[q] = acc;
  }
  if (normalize) {
    const double r = rsqrt(v[3] * v[3] + v[4] * v[4] + v[5] * v[5] + v[6] * v[6]);
    for (int q = 3; q < 7; ++q) v[q] *= r;
  }
  for (int q = 0; q < 7; ++q) out[7 * i + q] = v[q];
}

}  // namespace

Status advance(Context& c, const double* F, const double* T, double dt, int steps, int scheme, double tol, int* iters) {
  // Butcher tableaux (explicit): forward Euler, trapezoidal rule (Heun), classical RK4
  std::vector<std::vector<double>> A;
  std::vector<double> b;
  if (scheme == RBS_RK_EULER) {
    A = {{}};
    b = {1.0};
  } else if (scheme == RBS_RK_TRAPEZOID) {
    A = {{}, {1.0}};
    b = {0.5, 0.5};
  } else if (scheme == RBS_RK4) {
    A = {{}, {0.5}, {0.0, 0.5}, {0.0, 0.0, 1.0}};
    b = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
  } else {
    return Status::Err(RBS_EINVAL, "advance: unknown scheme");
  }
  const int n = c.n;
  const int S = (int)b.size();
  cudaStream_t s = c.stream;
  DevBuf<double> state0, stage, ks;
  RBS_TRY(state0.alloc((size_t)7 * n));
  RBS_TRY(stage.alloc((size_t)7 * n));
  RBS_TRY(ks.alloc((size_t)7 * n * S));
  std::vector<double> h(7 * (size_t)n);
  for (int i = 0; i < n; ++i) {
    double nq = 0.0;
    for (int q = 0; q < 4; ++q) nq += c.quats[4 * i + q] * c.quats[4 * i + q];
    nq = std::sqrt(nq);
    for (int q = 0; q < 3; ++q) h[7 * i + q] = c.centres[3 * i + q];
    for (int q = 0; q < 4; ++q) h[7 * i + 3 + q] = c.quats[4 * i + q] / nq;
  }
  RBS_CUDA_TRY(cudaMemcpyAsync(state0.ptr, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, s));
  std::vector<double> vtmp(3 * (size_t)n), otmp(3 * (size_t)n), cen(3 * (size_t)n), qu(4 * (size_t)n);
  const bool magnetic = c.opt.mu_ratio != 1.0 && (c.opt.magnetic_field[0] != 0.0 || c.opt.magnetic_field[1] != 0.0 ||
                                                  c.opt.magnetic_field[2] != 0.0);
  std::vector<double> Fm(magnetic ? 3 * (size_t)n : 0), Tm(magnetic ? 3 * (size_t)n : 0);
  int total = 0;
  const int nb = cdiv(n, 128);
  for (int step = 0; step < steps; ++step) {
    for (int st = 0; st < S; ++st) {
      double cf[4] = {0, 0, 0, 0};
      for (size_t k = 0; k < A[st].size(); ++k) cf[k] = A[st][k];
      c.stats.launches += 1;
      k_rk_combine<<<nb, 128, 0, s>>>(n, state0.ptr, ks.ptr, st, cf[0], cf[1], cf[2], cf[3], dt, 0, stage.ptr);
      RBS_CUDA_TRY(cudaGetLastError());
      RBS_CUDA_TRY(cudaMemcpyAsync(h.data(), stage.ptr, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
      RBS_CUDA_TRY(cudaStreamSynchronize(s));
      for (int i = 0; i < n; ++i) {
        for (int q = 0; q < 3; ++q) cen[3 * i + q] = h[7 * i + q];
        for (int q = 0; q < 4; ++q) qu[4 * i + q] = h[7 * i + 3 + q];
      }
      RBS_TRY(update_configuration(c, cen.data(), qu.data()));
      int its = 0;
      const double* Fs = F;
      const double* Ts = T;
      if (magnetic) {
        // the magnetic force and torque of the stage configuration (Section 4.1.3) join the applied ones
        int mits = 0;
        RBS_TRY(c.mag.d_FT.alloc(6 * (size_t)n));
        RBS_TRY(magnetic_forces(c, c.opt.magnetic_field, c.opt.mu_ratio, tol, c.mag.d_FT.ptr, nullptr, &mits));
        std::vector<double> ftm(6 * (size_t)n);
        RBS_CUDA_TRY(cudaMemcpyAsync(ftm.data(), c.mag.d_FT.ptr, sizeof(double) * ftm.size(), cudaMemcpyDeviceToHost, s));
        RBS_CUDA_TRY(cudaStreamSynchronize(s));
        for (int i = 0; i < n; ++i)
          for (int q = 0; q < 3; ++q) {
            Fm[3 * i + q] = F[3 * i + q] + ftm[6 * i + q];
            Tm[3 * i + q] = T[3 * i + q] + ftm[6 * i + 3 + q];
          }
        Fs = Fm.data();
        Ts = Tm.data();
      }
      RBS_TRY(mobility_solve(c, Fs, Ts, tol, vtmp.data(), otmp.data(), nullptr, &its, false));
      total += its;
      if (c.opt.warm_record) {
        std::vector<double> ft(6 * (size_t)n);
        for (int i = 0; i < n; ++i)
          for (int q = 0; q < 3; ++q) {
            ft[6 * i + q] = Fs[3 * i + q];
            ft[6 * i + 3 + q] = Ts[3 * i + q];
          }
        DevBuf<double> dft;
        RBS_TRY(dft.alloc(ft.size()));
        RBS_CUDA_TRY(cudaMemcpyAsync(dft.ptr, ft.data(), sizeof(double) * ft.size(), cudaMemcpyHostToDevice, s));
        RBS_TRY(warm_record(c, dft.ptr, c.d_prev.ptr));
      }
      c.stats.launches += 1;
      k_rk_rates<<<nb, 128, 0, s>>>(n, c.d_vo.ptr, stage.ptr, ks.ptr + (size_t)st * 7 * n);
      RBS_CUDA_TRY(cudaGetLastError());
    }
    c.stats.launches += 1;
    k_rk_combine<<<nb, 128, 0, s>>>(n, state0.ptr, ks.ptr, S, b[0], S > 1 ? b[1] : 0.0, S > 2 ? b[2] : 0.0,
                                    S > 3 ? b[3] : 0.0, dt, 1, state0.ptr);
    RBS_CUDA_TRY(cudaGetLastError());
  }
  RBS_CUDA_TRY(cudaMemcpyAsync(h.data(), state0.ptr, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
  RBS_CUDA_TRY(cudaStreamSynchronize(s));
  for (int i = 0; i < n; ++i) {
    for (int q = 0; q < 3; ++q) cen[3 * i + q] = h[7 * i + q];
    for (int q = 0; q < 4; ++q) qu[4 * i + q] = h[7 * i + 3 + q];
  }
  RBS_TRY(update_configuration(c, cen.data(), qu.data()));
  if (iters) *iters = total;
  return Status::Ok();
}

}  // namespace rbs
