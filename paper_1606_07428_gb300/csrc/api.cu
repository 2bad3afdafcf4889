// The C ABI of include/rbs.h: argument checks, host <-> device copies and dispatch.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>

#include "common.cuh"

using rbs::Context;
using rbs::Status;

namespace {

int finish(Context& c, const Status& s) {
  c.err = s.ok() ? std::string() : s.msg;
  return s.code;
}

Status enter(Context& c) {
  RBS_CUDA_TRY(cudaSetDevice(c.device));
  return Status::Ok();
}

bool finite_all(const double* a, long long n) {
  for (long long i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

}  // namespace

namespace rbs {

Status Context::time_begin(int cls, Timed* t) {
  t->cls = cls;
  for (cudaEvent_t* e : {&t->a, &t->b}) {
    if (!free_events.empty()) {
      *e = free_events.back();
      free_events.pop_back();
    } else {
      RBS_CUDA_TRY(cudaEventCreate(e));
    }
  }
  RBS_CUDA_TRY(cudaEventRecord(t->a, stream));
  return Status::Ok();
}

Status Context::time_end(Timed* t, double units) {
  RBS_CUDA_TRY(cudaEventRecord(t->b, stream));
  t->units = units;
  pending.push_back(*t);
  if (pending.size() > 4096) return harvest();
  return Status::Ok();
}

Status Context::harvest() {
  for (const Timed& t : pending) {
    RBS_CUDA_TRY(cudaEventSynchronize(t.b));
    float ms = 0.0f;
    RBS_CUDA_TRY(cudaEventElapsedTime(&ms, t.a, t.b));
    stats.kernel_ms[t.cls] += ms;
    free_events.push_back(t.a);
    free_events.push_back(t.b);
  }
  pending.clear();
  return Status::Ok();
}

Context::~Context() {
  warm_release(*this);
  for (const Timed& t : pending) {
    free_events.push_back(t.a);
    free_events.push_back(t.b);
  }
  for (cudaEvent_t e : free_events) cudaEventDestroy(e);
  for (Grid* g : grids) delete g;
  grids.clear();
  if (h_pinned) cudaFreeHost(h_pinned);
  h_pinned = nullptr;
}
}  // namespace rbs

extern "C" {

void rbs_default_options(rbs_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = RBS_PREC_FP64;
  o->restart = 50;
  o->max_iters = 500;
  o->preconditioner = 1;
  o->near_delta = 1.0;
  o->p_up_factor = 2;
  o->p_self_factor = 2;
  o->viscosity = 1.0;
  o->inner_tol = 1e-5;
  o->max_refinements = 20;
  o->device = 0;
  o->stream = nullptr;
  o->timing = 0;
  o->refine_precision = RBS_PREC_DF;
  o->warm_start = RBS_WARM_ZERO;
  o->pair_variant = 0;
  o->warm_record = 0;
  o->contact_gap = 0.0;
  o->magnetic_field[0] = o->magnetic_field[1] = o->magnetic_field[2] = 0.0;
  o->mu_ratio = 1.0;
  o->far_field = RBS_FAR_DIRECT;
  o->tree_theta = 0.5;
  o->tree_degree = 7;
  o->tree_df_theta = 0.4;
  o->tree_df_degree = 12;
  o->graphs = 1;
}

int rbs_create(const rbs_options* opt, rbs_ctx** out) {
  if (!out) return RBS_EINVAL;
  *out = nullptr;
  rbs_options o;
  if (opt)
    o = *opt;
  else
    rbs_default_options(&o);
  if (o.restart < 1 || o.restart > 500 || o.max_iters < 1 || o.p_up_factor < 1 || o.p_up_factor > 4 ||
      o.p_self_factor < 1 || o.p_self_factor > 4 || !(o.viscosity > 0) || !(o.near_delta >= 0) ||
      !(o.inner_tol > 0 && o.inner_tol < 1) || o.max_refinements < 1 ||
      (o.precision != RBS_PREC_FP64 && !rbs::prec_f32(o.precision)) ||
      (o.refine_precision != RBS_PREC_FP64 && o.refine_precision != RBS_PREC_DF) || o.warm_start < 0 ||
      (o.pair_variant != 0 && o.pair_variant != 1 && o.pair_variant != 2 && o.pair_variant != 4 &&
       o.pair_variant != 9 && o.pair_variant != 10 && o.pair_variant != 12) ||
      o.warm_start > 3 || !(o.contact_gap >= 0.0) || !(o.mu_ratio > 0.0) ||
      !std::isfinite(o.magnetic_field[0]) || !std::isfinite(o.magnetic_field[1]) || !std::isfinite(o.magnetic_field[2]) ||
      (o.far_field != RBS_FAR_DIRECT && o.far_field != RBS_FAR_TREECODE && o.far_field != RBS_FAR_TREECODE_DF) ||
      !(o.tree_theta > 0.0 && o.tree_theta < 1.0) || o.tree_degree < 2 || o.tree_degree > 10 ||
      !(o.tree_df_theta > 0.0 && o.tree_df_theta < 1.0) || o.tree_df_degree < 2 || o.tree_df_degree > 12 ||
      (o.graphs != 0 && o.graphs != 1))
    return RBS_EINVAL;
  rbs_ctx* h = new rbs_ctx();
  Context& c = h->c;
  c.opt = o;
  c.device = o.device;
  c.stream = (cudaStream_t)o.stream;
  Status s = enter(c);
  if (s.ok()) {
    cudaError_t e = cudaDeviceGetAttribute(&c.sm_count, cudaDevAttrMultiProcessorCount, c.device);
    if (e == cudaSuccess) e = cudaMallocHost(&c.h_pinned, 64 * sizeof(double));
    if (e != cudaSuccess) s = Status::Err(RBS_ECUDA, std::string("device set-up: ") + cudaGetErrorString(e));
  }
  if (!s.ok()) {
    delete h;
    return s.code;
  }
  *out = h;
  return RBS_OK;
}

void rbs_destroy(rbs_ctx* h) {
  if (!h) return;
  cudaSetDevice(h->c.device);
  cudaStreamSynchronize(h->c.stream);
  delete h;
}

namespace {

// Checks shared by both geometry entry points: grids, orientations and suspension ids.
Status check_particles(int n, const int* p, const int* nphi, const double* centres, const double* quats,
                       const int* suspension_id) {
  if (!finite_all(centres, 3LL * n) || !finite_all(quats, 4LL * n))
    return Status::Err(RBS_EINVAL, "set_geometry: non-finite input");
  for (int i = 0; i < n; ++i) {
    if (p[i] < 2 || p[i] > 32) return Status::Err(RBS_EINVAL, "set_geometry: p must be in [2, 32]");
    int nf = nphi ? nphi[i] : 2 * p[i];
    if (nf < 2 * p[i] || nf % 2 != 0 || nf > 4 * p[i] + 4)
      return Status::Err(RBS_EINVAL, "set_geometry: nphi must be even and in [2p, 4p + 4]");
    const double* q = quats + 4 * i;
    double qn = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    if (!(qn > 1e-12)) return Status::Err(RBS_EINVAL, "set_geometry: zero quaternion");
    if (suspension_id && i > 0 && suspension_id[i] != suspension_id[i - 1]) {
      for (int k = 0; k < i - 1; ++k)
        if (suspension_id[k] == suspension_id[i])
          return Status::Err(RBS_EINVAL, "set_geometry: particles of one suspension must be contiguous");
    }
  }
  return Status::Ok();
}

void store_particles(Context& c, int n, const int* p, const int* nphi, const double* centres, const double* quats,
                     const int* suspension_id) {
  c.have_geometry = false;
  c.n = n;
  c.centres.assign(centres, centres + 3LL * n);
  c.quats.assign(quats, quats + 4LL * n);
  c.p.assign(p, p + n);
  c.nphi.resize(n);
  for (int i = 0; i < n; ++i) c.nphi[i] = nphi ? nphi[i] : 2 * p[i];
  c.sid.assign(n, 0);
  if (suspension_id) c.sid.assign(suspension_id, suspension_id + n);
}

}  // namespace

int rbs_set_geometry(rbs_ctx* h, int n, const double* semi_axes, const int* p, const int* nphi, const double* centres,
                     const double* quats, const int* suspension_id) {
  if (!h) return RBS_EINVAL;
  Context& c = h->c;
  if (n < 1 || !semi_axes || !p || !centres || !quats)
    return finish(c, Status::Err(RBS_EINVAL, "set_geometry: null array or n < 1"));
  if (!finite_all(semi_axes, 3LL * n)) return finish(c, Status::Err(RBS_EINVAL, "set_geometry: non-finite input"));
  for (int i = 0; i < n; ++i)
    if (!(semi_axes[3 * i] > 0 && semi_axes[3 * i + 1] > 0 && semi_axes[3 * i + 2] > 0))
      return finish(c, Status::Err(RBS_EINVAL, "set_geometry: semi-axes must be positive"));
  Status s = check_particles(n, p, nphi, centres, quats, suspension_id);
  if (!s.ok()) return finish(c, s);
  s = enter(c);
  if (!s.ok()) return finish(c, s);
  store_particles(c, n, p, nphi, centres, quats, suspension_id);
  c.axes.assign(semi_axes, semi_axes + 3LL * n);
  c.cs_of.clear();
  c.cs_pg.clear();
  c.cs_off.clear();
  c.cs_coef.clear();
  return finish(c, rbs::build_geometry(c));
}

int rbs_set_geometry_sh(rbs_ctx* h, int n, int nshape, const int* shape_pg, const double* shape_coef,
                        const int* shape_of, const int* p, const int* nphi, const double* centres, const double* quats,
                        const int* suspension_id) {
  if (!h) return RBS_EINVAL;
  Context& c = h->c;
  if (n < 1 || nshape < 1 || !shape_pg || !shape_coef || !shape_of || !p || !centres || !quats)
    return finish(c, Status::Err(RBS_EINVAL, "set_geometry_sh: null array, n < 1 or nshape < 1"));
  std::vector<long long> off(nshape);
  long long total = 0;
  for (int k = 0; k < nshape; ++k) {
    if (shape_pg[k] < 1 || shape_pg[k] > RBS_MAX_SHAPE_DEGREE)
      return finish(c, Status::Err(RBS_EINVAL, "set_geometry_sh: shape degree must be in [1, RBS_MAX_SHAPE_DEGREE]"));
    off[k] = total;
    total += 3LL * (shape_pg[k] + 1) * (shape_pg[k] + 1);
  }
  if (!finite_all(shape_coef, total))
    return finish(c, Status::Err(RBS_EINVAL, "set_geometry_sh: non-finite coefficient"));
  for (int i = 0; i < n; ++i)
    if (shape_of[i] < 0 || shape_of[i] >= nshape)
      return finish(c, Status::Err(RBS_EINVAL, "set_geometry_sh: shape_of out of range"));
  Status s = check_particles(n, p, nphi, centres, quats, suspension_id);
  if (!s.ok()) return finish(c, s);
  s = enter(c);
  if (!s.ok()) return finish(c, s);
  store_particles(c, n, p, nphi, centres, quats, suspension_id);
  c.axes.assign(3LL * n, 0.0);
  c.cs_of.assign(shape_of, shape_of + n);
  c.cs_pg.assign(shape_pg, shape_pg + nshape);
  c.cs_off = off;
  c.cs_coef.assign(shape_coef, shape_coef + total);
  return finish(c, rbs::build_geometry(c));
}

long long rbs_total_nodes(const rbs_ctx* h) { return (h && h->c.have_geometry) ? h->c.N : 0; }

int rbs_get_surface(rbs_ctx* h, double* x, double* normal, double* weight) {
  if (!h) return RBS_EINVAL;
  Context& c = h->c;
  if (!c.have_geometry) return finish(c, Status::Err(RBS_ESTATE, "no geometry"));
  Status s = enter(c);
  if (!s.ok()) return finish(c, s);
  std::vector<double4> hx(c.N), hn(c.N);
  cudaError_t e = cudaMemcpyAsync(hx.data(), c.d_x.ptr, sizeof(double4) * c.N, cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hn.data(), c.d_nrm.ptr, sizeof(double4) * c.N, cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) return finish(c, Status::Err(RBS_ECUDA, std::string("get_surface: ") + cudaGetErrorString(e)));
  for (long long t = 0; t < c.N; ++t) {
    if (x) {
      x[3 * t] = hx[t].x;
      x[3 * t + 1] = hx[t].y;
      x[3 * t + 2] = hx[t].z;
    }
    if (normal) {
      normal[3 * t] = hn[t].x;
      normal[3 * t + 1] = hn[t].y;
      normal[3 * t + 2] = hn[t].z;
    }
    if (weight) weight[t] = hx[t].w;
  }
  return finish(c, Status::Ok());
}

static int solve_common(rbs_ctx* h, const double* F, const double* T, double tol, double* v, double* omega,
                        double* density, int* iterations, bool device_io) {
  if (!h) return RBS_EINVAL;
  Context& c = h->c;
  if (!c.have_geometry) return finish(c, Status::Err(RBS_ESTATE, "mobility_solve before set_geometry"));
  if (!F || !T || !v || !omega) return finish(c, Status::Err(RBS_EINVAL, "mobility_solve: null array"));
  if (!(tol > 0 && tol < 1)) return finish(c, Status::Err(RBS_EINVAL, "mobility_solve: tol must be in (0, 1)"));
  if (!device_io && (!finite_all(F, 3LL * c.n) || !finite_all(T, 3LL * c.n)))
    return finish(c, Status::Err(RBS_EINVAL, "mobility_solve: non-finite force or torque"));
  Status s = enter(c);
  if (!s.ok()) return finish(c, s);
  int its = 0;
  s = rbs::mobility_solve(c, F, T, tol, v, omega, density, &its, device_io);
  if (iterations && (s.ok() || s.code == RBS_ENOTCONV))
    for (int k = 0; k < c.seg3.S; ++k) iterations[k] = k < (int)c.susp_iters.size() ? c.susp_iters[k] : 0;
  return finish(c, s);
}

int rbs_suspension_count(const rbs_ctx* h) {
  if (!h) return RBS_EINVAL;
  return h->c.have_geometry ? h->c.seg3.S : 0;
}

int rbs_get_suspension_results(rbs_ctx* h, int* iterations, double* residual) {
  if (!h) return RBS_EINVAL;
  Context& c = h->c;
  if (!c.have_geometry) return finish(c, Status::Err(RBS_ESTATE, "no geometry"));
  const int S = c.seg3.S;
  for (int k = 0; k < S; ++k) {
    if (iterations) iterations[k] = k < (int)c.susp_iters.size() ? c.susp_iters[k] : 0;
    if (residual) residual[k] = k < (int)c.susp_res.size() ? c.susp_res[k] : 0.0;
  }
  return finish(c, Status::Ok());
}

int rbs_mobility_solve(rbs_ctx* h, const double* F, const double* T, double tol, double* v, double* omega,
                       double* density, int* iterations) {
  return solve_common(h, F, T, tol, v, omega, density, iterations, false);
}

int rbs_mobility_solve_device(rbs_ctx* h, const double* F_dev, const double* T_dev, double tol, double* v_dev,
                              double* omega_dev, double* density_dev, int* iterations) {
  return solve_common(h, F_dev, T_dev, tol, v_dev, omega_dev, density_dev, iterations, true);
}

int rbs_advance(rbs_ctx* h, const double* F, const double* T, double dt, int steps, int scheme, double tol,
                int* iterations) {
  if (!h) return RBS_EINVAL;
  Context& c = h->c;
  if (!c.have_geometry) return finish(c, Status::Err(RBS_ESTATE, "advance before set_geometry"));
  if (!F || !T) return finish(c, Status::Err(RBS_EINVAL, "advance: null force or torque"));
  if (!(dt > 0) || !std::isfinite(dt) || steps < 0 || !(tol > 0 && tol < 1))
    return finish(c, Status::Err(RBS_EINVAL, "advance: need dt > 0, steps >= 0, 0 < tol < 1"));
  if (!finite_all(F, 3LL * c.n) || !finite_all(T, 3LL * c.n))
    return finish(c, Status::Err(RBS_EINVAL, "advance: non-finite force or torque"));
  Status s = enter(c);
  if (!s.ok()) return finish(c, s);
  return finish(c, rbs::advance(c, F, T, dt, steps, scheme, tol, iterations));
}

int rbs_warmstart_record(rbs_ctx* h, const double* F, const double* T) {
  if (!h) return RBS_EINVAL;
  Context& c = h->c;
  if (!c.have_geometry || !c.have_prev) return finish(c, Status::Err(RBS_ESTATE, "warmstart_record needs a solved density"));
  if (!F || !T) return finish(c, Status::Err(RBS_EINVAL, "warmstart_record: null force or torque"));
  Status s = enter(c);
  if (!s.ok()) return finish(c, s);
  std::vector<double> ft(6 * (size_t)c.n);
  for (int i = 0; i < c.n; ++i)
    for (int q = 0; q < 3; ++q) {
      ft[6 * i + q] = F[3 * i + q];
      ft[6 * i + 3 + q] = T[3 * i + q];
    }
  cudaError_t e = cudaMemcpyAsync(c.d_FT.ptr, ft.data(), sizeof(double) * ft.size(), cudaMemcpyHostToDevice, c.stream);
  if (e != cudaSuccess) return finish(c, Status::Err(RBS_ECUDA, cudaGetErrorString(e)));
  return finish(c, rbs::warm_record(c, c.d_FT.ptr, c.d_prev.ptr));
}

int rbs_warmstart_train(rbs_ctx* h, int epochs, int batch, double lr, unsigned seed, double* loss) {
  if (!h) return RBS_EINVAL;
  Context& c = h->c;
  if (!c.have_geometry) return finish(c, Status::Err(RBS_ESTATE, "no geometry"));
  if (epochs < 0 || batch < 1 || !(lr > 0)) return finish(c, Status::Err(RBS_EINVAL, "warmstart_train: bad arguments"));
  Status s = enter(c);
  if (!s.ok()) return finish(c, s);
  return finish(c, rbs::warm_train(c, epochs, batch, lr, seed, loss));
}

int rbs_warmstart_weights(rbs_ctx* h, float* out, const float* in, long long* count, float* scale) {
  if (!h) return RBS_EINVAL;
  Context& c = h->c;
  if (!c.have_geometry) return finish(c, Status::Err(RBS_ESTATE, "no geometry"));
  Status s = enter(c);
  if (!s.ok()) return finish(c, s);
  return finish(c, rbs::warm_weights(c, out, in, count, scale));
}

int rbs_warmstart_features(rbs_ctx* h, const double* F, const double* T, float* X) {
  if (!h) return RBS_EINVAL;
  Context& c = h->c;
  if (!c.have_geometry) return finish(c, Status::Err(RBS_ESTATE, "no geometry"));
  if (!F || !T || !X) return finish(c, Status::Err(RBS_EINVAL, "warmstart_features: null array"));
  Status s = enter(c);
  if (!s.ok()) return finish(c, s);
  return finish(c, rbs::warm_features_host(c, F, T, X));
}

int rbs_warmstart_targets(rbs_ctx* h, const double* mu, float* coef) {
  if (!h) return RBS_EINVAL;
  Context& c = h->c;
  if (!c.have_geometry) return finish(c, Status::Err(RBS_ESTATE, "no geometry"));
  if (!mu || !coef) return finish(c, Status::Err(RBS_EINVAL, "warmstart_targets: null array"));
  Status s = enter(c);
  if (!s.ok()) return finish(c, s);
  return finish(c, rbs::warm_targets_host(c, mu, coef));
}

int rbs_warmstart_mlp(rbs_ctx* h, int rows, const float* X, const float* Yt, float* Y, float* grads, double* loss) {
  if (!h) return RBS_EINVAL;
  Context& c = h->c;
  if (!c.have_geometry) return finish(c, Status::Err(RBS_ESTATE, "no geometry"));
  if (rows < 1 || !X) return finish(c, Status::Err(RBS_EINVAL, "warmstart_mlp: bad arguments"));
  Status s = enter(c);
  if (!s.ok()) return finish(c, s);
  return finish(c, rbs::warm_mlp_host(c, rows, X, Yt, Y, grads, loss));
}

int rbs_get_state(rbs_ctx* h, double* centres, double* quats) {
  if (!h) return RBS_EINVAL;
  Context& c = h->c;
  if (!c.have_geometry) return finish(c, Status::Err(RBS_ESTATE, "no geometry"));
  for (int i = 0; i < 3 * c.n && centres; ++i) centres[i] = c.centres[i];
  for (int i = 0; i < 4 * c.n && quats; ++i) quats[i] = c.quats[i];
  return finish(c, Status::Ok());
}

int rbs_incident_density(rbs_ctx* h, const double* F, const double* T, double* rho) {
  if (!h) return RBS_EINVAL;
  Context& c = h->c;
  if (!c.have_geometry) return finish(c, Status::Err(RBS_ESTATE, "no geometry"));
  if (!F || !T || !rho) return finish(c, Status::Err(RBS_EINVAL, "incident_density: null array"));
  Status s = enter(c);
  if (!s.ok()) return finish(c, s);
  std::vector<double> ft(6 * (size_t)c.n);
  for (int i = 0; i < c.n; ++i)
    for (int q = 0; q < 3; ++q) {
      ft[6 * i + q] = F[3 * i + q];
      ft[6 * i + 3 + q] = T[3 * i + q];
    }
  cudaError_t e = cudaMemcpyAsync(c.d_FT.ptr, ft.data(), sizeof(double) * ft.size(), cudaMemcpyHostToDevice, c.stream);
  if (e != cudaSuccess) return finish(c, Status::Err(RBS_ECUDA, cudaGetErrorString(e)));
  s = rbs::incident_density(c, c.d_FT.ptr, c.d_vec[0].ptr);
  if (!s.ok()) return finish(c, s);
  e = cudaMemcpyAsync(rho, c.d_vec[0].ptr, sizeof(double) * 3 * c.N, cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) return finish(c, Status::Err(RBS_ECUDA, cudaGetErrorString(e)));
  return finish(c, Status::Ok());
}

int rbs_rigid_velocities(rbs_ctx* h, const double* u, double* v, double* omega) {
  if (!h) return RBS_EINVAL;
  Context& c = h->c;
  if (!c.have_geometry) return finish(c, Status::Err(RBS_ESTATE, "no geometry"));
  if (!u || !v || !omega) return finish(c, Status::Err(RBS_EINVAL, "rigid_velocities: null array"));
  Status s = enter(c);
  if (!s.ok()) return finish(c, s);
  cudaError_t e = cudaMemcpyAsync(c.d_vec[0].ptr, u, sizeof(double) * 3 * c.N, cudaMemcpyHostToDevice, c.stream);
  if (e != cudaSuccess) return finish(c, Status::Err(RBS_ECUDA, cudaGetErrorString(e)));
  s = rbs::rigid_velocities(c, c.d_vec[0].ptr, c.d_vo.ptr);
  if (!s.ok()) return finish(c, s);
  std::vector<double> vo(6 * (size_t)c.n);
  e = cudaMemcpyAsync(vo.data(), c.d_vo.ptr, sizeof(double) * vo.size(), cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) return finish(c, Status::Err(RBS_ECUDA, cudaGetErrorString(e)));
  for (int i = 0; i < c.n; ++i)
    for (int q = 0; q < 3; ++q) {
      v[3 * i + q] = vo[6 * i + q];
      omega[3 * i + q] = vo[6 * i + 3 + q];
    }
  return finish(c, Status::Ok());
}

int rbs_apply_operator_device(rbs_ctx* h, int op, int precision, const double* x_dev, double* y_dev) {
  if (!h) return RBS_EINVAL;
  Context& c = h->c;
  if (!c.have_geometry) return finish(c, Status::Err(RBS_ESTATE, "no geometry"));
  if (!x_dev || !y_dev || x_dev == y_dev) return finish(c, Status::Err(RBS_EINVAL, "apply_operator: bad buffers"));
  if (precision != RBS_PREC_FP64 && !rbs::prec_f32(precision) && precision != RBS_PREC_DF)
    return finish(c, Status::Err(RBS_EINVAL, "apply_operator: bad precision"));
  if (rbs::prec_16(precision) && c.opt.precision != precision)
    return finish(c, Status::Err(RBS_EINVAL, "apply_operator: 16-bit self blocks need a context of that precision"));
  Status s = enter(c);
  if (!s.ok()) return finish(c, s);
  s = rbs::apply_operator(c, op, precision, x_dev, y_dev);
  if (s.ok()) {
    cudaError_t e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) s = Status::Err(RBS_ECUDA, cudaGetErrorString(e));
  }
  if (s.ok()) s = rbs::check_self_gemm(c);
  return finish(c, s);
}

int rbs_apply_operator(rbs_ctx* h, int op, int precision, const double* x, double* y) {
  if (!h) return RBS_EINVAL;
  Context& c = h->c;
  if (!c.have_geometry) return finish(c, Status::Err(RBS_ESTATE, "no geometry"));
  if (!x || !y) return finish(c, Status::Err(RBS_EINVAL, "apply_operator: null array"));
  Status s = enter(c);
  if (!s.ok()) return finish(c, s);
  cudaError_t e = cudaMemcpyAsync(c.d_vec[0].ptr, x, sizeof(double) * 3 * c.N, cudaMemcpyHostToDevice, c.stream);
  if (e != cudaSuccess) return finish(c, Status::Err(RBS_ECUDA, cudaGetErrorString(e)));
  int rc = rbs_apply_operator_device(h, op, precision, c.d_vec[0].ptr, c.d_vec[1].ptr);
  if (rc != RBS_OK) return rc;
  e = cudaMemcpyAsync(y, c.d_vec[1].ptr, sizeof(double) * 3 * c.N, cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) return finish(c, Status::Err(RBS_ECUDA, cudaGetErrorString(e)));
  return finish(c, Status::Ok());
}

int rbs_get_stats(rbs_ctx* h, rbs_stats* out) {
  if (!h || !out) return RBS_EINVAL;
  Context& c = h->c;
  Status s = enter(c);
  if (s.ok()) s = c.harvest();
  if (!s.ok()) return finish(c, s);
  *out = c.stats;
  for (int k = 0; k < 5; ++k) out->pair_variant[k] = c.tuned[k];
  for (int k = 0; k < 2; ++k)  // the float32 sums run in the treecode kernel when it is on
    if (c.tree.active) out->pair_variant[k] = c.tree.nt[k] ? rbs::kPacked + c.tree.nt[k] : 0;
  for (int k = 0; k < 3; ++k)  // and the double-float ones in the double-float treecode kernel
    if (c.tree_df.active) out->pair_variant[2 + k] = c.tree_df.nt[k];
  return RBS_OK;
}

int rbs_reset_stats(rbs_ctx* h) {
  if (!h) return RBS_EINVAL;
  Context& c = h->c;
  Status s = enter(c);
  if (s.ok()) s = c.harvest();
  if (!s.ok()) return finish(c, s);
  c.stats.launches = 0;
  for (int k = 0; k < RBS_KC_COUNT; ++k) {
    c.stats.kernel_ms[k] = 0.0;
    c.stats.kernel_count[k] = 0;
    c.stats.kernel_units[k] = 0.0;
  }
  return RBS_OK;
}

int rbs_magnetic_forces(rbs_ctx* h, const double* H0, double mu_ratio, double tol, double* F, double* T, double* q,
                        int* iterations) {
  if (!h) return RBS_EINVAL;
  Context& c = h->c;
  if (!H0 || !F || !T) return finish(c, Status::Err(RBS_EINVAL, "magnetic_forces: null array"));
  if (!c.have_geometry) return finish(c, Status::Err(RBS_ESTATE, "no geometry"));
  if (!finite_all(H0, 3) || !(mu_ratio > 0.0) || !(tol > 0.0 && tol < 1.0))
    return finish(c, Status::Err(RBS_EINVAL, "magnetic_forces: bad field, permeability ratio or tolerance"));
  Status s = enter(c);
  if (!s.ok()) return finish(c, s);
  s = c.mag.d_FT.alloc(6 * (size_t)c.n);
  int its = 0;
  if (s.ok()) s = rbs::magnetic_forces(c, H0, mu_ratio, tol, c.mag.d_FT.ptr, q, &its);
  if (s.ok()) {
    std::vector<double> ft(6 * (size_t)c.n);
    cudaError_t e = cudaMemcpyAsync(ft.data(), c.mag.d_FT.ptr, sizeof(double) * ft.size(), cudaMemcpyDeviceToHost,
                                    c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) s = Status::Err(RBS_ECUDA, std::string("magnetic_forces: ") + cudaGetErrorString(e));
    for (int i = 0; s.ok() && i < c.n; ++i)
      for (int k = 0; k < 3; ++k) {
        F[3 * i + k] = ft[6 * i + k];
        T[3 * i + k] = ft[6 * i + 3 + k];
      }
  }
  if (iterations) *iterations = its;
  return finish(c, s);
}

int rbs_apply_laplace(rbs_ctx* h, int kind, const double* x, double* y) {
  if (!h) return RBS_EINVAL;
  Context& c = h->c;
  if (!x || !y || (kind != 0 && kind != 1)) return finish(c, Status::Err(RBS_EINVAL, "apply_laplace: bad arguments"));
  if (!c.have_geometry) return finish(c, Status::Err(RBS_ESTATE, "no geometry"));
  Status s = enter(c);
  if (!s.ok()) return finish(c, s);
  rbs::DevBuf<double> dx, dy;
  s = dx.alloc(c.N);
  if (s.ok()) s = dy.alloc(c.N);
  cudaError_t e = cudaSuccess;
  if (s.ok()) e = cudaMemcpyAsync(dx.ptr, x, sizeof(double) * c.N, cudaMemcpyHostToDevice, c.stream);
  if (s.ok() && e == cudaSuccess) s = rbs::laplace_operator(c, kind, dx.ptr, dy.ptr);
  if (s.ok() && e == cudaSuccess) e = cudaMemcpyAsync(y, dy.ptr, sizeof(double) * c.N, cudaMemcpyDeviceToHost, c.stream);
  if (s.ok() && e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (s.ok() && e != cudaSuccess) s = Status::Err(RBS_ECUDA, std::string("apply_laplace: ") + cudaGetErrorString(e));
  return finish(c, s);
}

int rbs_get_contacts(rbs_ctx* h, int max, int* pairs, double* points, double* forces) {
  if (!h || max < 0) return RBS_EINVAL;
  const Context& c = h->c;
  const int nc = (int)c.contacts.size();
  for (int k = 0; k < std::min(nc, max); ++k) {
    const Context::Contact& ct = c.contacts[k];
    if (pairs) {
      pairs[2 * k] = ct.i;
      pairs[2 * k + 1] = ct.j;
    }
    for (int q = 0; q < 3; ++q) {
      if (points) points[3 * k + q] = ct.x[q];
      if (forces) forces[3 * k + q] = ct.f[q];
    }
  }
  return nc;
}

const char* rbs_last_error(const rbs_ctx* h) {
  if (!h) return "null context";
  return h->c.err.c_str();
}

int rbs_treecode_plan(int n, const int* nodes, const double* centres, const double* radius, const double* node_box,
                      const int* suspension_id, double theta, int degree, double near_delta, int sm_count,
                      long long* out) {
  if (n < 1 || !nodes || !centres || !radius || !node_box || !out || !(theta > 0.0 && theta < 1.0) || degree < 2 ||
      degree > 12 || !(near_delta >= 0.0) || sm_count < 1)
    return RBS_EINVAL;
  std::vector<long long> offset(n + 1, 0);
  std::vector<int> sid(n, 0);
  for (int i = 0; i < n; ++i) {
    if (nodes[i] < 1 || !(radius[i] >= 0.0)) return RBS_EINVAL;
    offset[i + 1] = offset[i] + nodes[i];
    if (suspension_id) sid[i] = suspension_id[i];
  }
  const rbs::PlanInput in{n, offset.data(), centres, radius, sid.data(), node_box, near_delta, sm_count};
  rbs::TreePlan plan;
  const rbs::Status s = rbs::plan_treecode(in, theta, degree, plan);
  if (!s.ok()) return s.code;
  out[0] = plan.direct_pairs;
  out[1] = plan.proxy_pairs;
  out[2] = plan.n_cells;
  out[3] = (long long)plan.items.size();
  out[4] = (long long)plan.segs.size();
  out[5] = plan.tmax;
  return RBS_OK;
}

int rbs_grid_symmetry(int p, int nphi, int* rep_of, int* g_of, int* irrep_dim) {
  if (p < 2 || p > 32 || nphi < 2 * p || (nphi & 1)) return RBS_EINVAL;
  std::vector<int> r, g;
  int dims[8], nrep = 0;
  const rbs::Status s = rbs::grid_symmetry_host(p, nphi, r, g, dims, &nrep);
  if (!s.ok()) return s.code;
  const size_t np = (size_t)(p + 1) * nphi;
  for (size_t t = 0; t < np; ++t) {
    if (rep_of) rep_of[t] = r[t];
    if (g_of) g_of[t] = g[t];
  }
  if (irrep_dim)
    for (int c = 0; c < 8; ++c) irrep_dim[c] = dims[c];
  return nrep;
}

int rbs_near_plan(int n, const double* centres, const double* radius, const double* rmin, const int* suspension_id,
                  double near_delta, int max_pairs, int* pairs) {
  if (n < 1 || !centres || !radius || !rmin || !(near_delta >= 0.0) || max_pairs < 0 || (max_pairs > 0 && !pairs))
    return RBS_EINVAL;
  std::vector<int> sid(n, 0);
  if (suspension_id)
    for (int i = 0; i < n; ++i) sid[i] = suspension_id[i];
  std::vector<int2> out;
  const rbs::Status s = rbs::plan_near(n, centres, radius, rmin, sid.data(), near_delta, out);
  if (!s.ok()) return s.code;
  for (size_t k = 0; k < out.size() && k < (size_t)max_pairs; ++k) {
    pairs[2 * k] = out[k].x;
    pairs[2 * k + 1] = out[k].y;
  }
  return (int)std::min<size_t>(out.size(), (size_t)INT_MAX);
}

}  // extern "C"
