// Restarted, right-preconditioned GMRES (Section 3.2) over independent segments of the unknowns.
//
// The unknowns are split into S contiguous segments that the operator does not couple (the
// suspensions of a batch: particles of different suspensions do not interact).  Every segment runs
// its own Krylov recursion inside one shared sweep: the operator is applied to all segments' basis
// vectors at once, while the Gram-Schmidt coefficients, the Hessenberg matrix, the Givens rotations,
// the residual estimate and the stopping decision are kept per segment.  A segment whose residual
// estimate reaches its own tolerance stops contributing (its next basis vector is zero, and the
// operator maps zero to zero), so small suspensions converge on their own norm instead of on the
// union's.
//
// One Arnoldi step (basis gather, operator, two-pass classical Gram-Schmidt, norm, Givens, scaling)
// is a fixed sequence of kernels whose step index lives in device memory.  For the mobility operator
// the steps of a restart cycle run as one CUDA graph: a conditional WHILE node whose body is the
// captured step, re-entered by the device as long as some segment is active, so a cycle costs one
// graph launch and no host round trip per iteration.  The first step on a configuration runs eagerly
// (it also lets the autotuners pick their variants before capture); contexts that cannot build the
// graph run the same kernels eagerly with one host read per step.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace rbs {

namespace {

constexpr int kThreads = 256;
constexpr long long kChunk = 4096;  // elements per chunk; chunks never straddle a segment
constexpr int kDotBlocksX = 2048;

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
  __syncthreads();
  return s;  // valid in thread 0
}

// partial[i * nch + c] = V_i . w over chunk c, for i < nv; nv = ctrl[0] + nv_add, or nv_fixed when
// ctrl is null.
__global__ void __launch_bounds__(kThreads) k_seg_dot(const double* __restrict__ V, long long ldv,
                                                      const int* __restrict__ ctrl, int nv_add, int nv_fixed,
                                                      const double* __restrict__ w, const SegChunk* __restrict__ ch,
                                                      int nch, double* __restrict__ partial) {
  __shared__ double red[kThreads / 32];
  const int i = blockIdx.y;
  const int nv = ctrl ? ctrl[0] + nv_add : nv_fixed;
  if (i >= nv) return;
  const double* v = V + ldv * i;
  for (int c = blockIdx.x; c < nch; c += gridDim.x) {
    const SegChunk q = ch[c];
    double acc = 0.0;
    for (long long e = q.b + threadIdx.x; e < q.e; e += kThreads) acc = fma(v[e], w[e], acc);
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) partial[(long long)i * nch + c] = acc;
  }
}

// Sums the chunk partials of segment s = blockIdx.x for vector i = blockIdx.y.  Gram-Schmidt mode
// (H != null): coef[i * S + s] = the sum when segment s is active, else 0, and the same value is added
// to the Hessenberg entry H_s(i, k), k = ctrl[0].  Norm mode (H null): out[s] = the sum (i = 0).
__global__ void __launch_bounds__(kThreads) k_seg_reduce(const double* __restrict__ partial, int nch,
                                                         const int* __restrict__ c0, int S,
                                                         const int* __restrict__ ctrl, int nv_add, int nv_fixed,
                                                         const int* __restrict__ active, double* __restrict__ coef,
                                                         double* __restrict__ H, int ld, long long hs,
                                                         double* __restrict__ out) {
  __shared__ double red[kThreads / 32];
  const int s = blockIdx.x, i = blockIdx.y;
  const int nv = ctrl ? ctrl[0] + nv_add : nv_fixed;
  if (i >= nv) return;
  double acc = 0.0;
  for (int c = c0[s] + threadIdx.x; c < c0[s + 1]; c += kThreads) acc += partial[(long long)i * nch + c];
  acc = block_sum(acc, red);
  if (threadIdx.x != 0) return;
  if (H) {
    const double v = active[s] ? acc : 0.0;
    coef[(long long)i * S + s] = v;
    if (active[s]) H[hs * s + (long long)ctrl[0] * ld + i] += v;
  } else {
    out[s] = acc;
  }
}

// w = alpha w + sign * sum_{i < nv} coef[i * S + seg] V_i on every chunk; nv = ctrl[0] + nv_add, or
// nv_fixed when ctrl is null.
__global__ void __launch_bounds__(kThreads) k_seg_combine(double* __restrict__ w, double alpha,
                                                          const double* __restrict__ V, long long ldv,
                                                          const int* __restrict__ ctrl, int nv_add, int nv_fixed,
                                                          const double* __restrict__ coef, int S, double sign,
                                                          const SegChunk* __restrict__ ch, int nch) {
  extern __shared__ double sc[];
  const int nv = ctrl ? ctrl[0] + nv_add : nv_fixed;
  for (int c = blockIdx.x; c < nch; c += gridDim.x) {
    const SegChunk q = ch[c];
    for (int i = threadIdx.x; i < nv; i += kThreads) sc[i] = sign * coef[(long long)i * S + q.seg];
    __syncthreads();
    for (long long e = q.b + threadIdx.x; e < q.e; e += kThreads) {
      double acc = (alpha == 0.0) ? 0.0 : alpha * w[e];
      for (int i = 0; i < nv; ++i) acc = fma(sc[i], V[ldv * i + e], acc);
      w[e] = acc;
    }
    __syncthreads();
  }
}

// out = V + ldv * (ctrl ? ctrl[0] + 1 : 0):  out = w / den[seg] on the chunks of active segments with
// den > 0, and 0 elsewhere.
__global__ void __launch_bounds__(kThreads) k_seg_scale(double* __restrict__ V, long long ldv,
                                                        const int* __restrict__ ctrl, const double* __restrict__ w,
                                                        const double* __restrict__ den,
                                                        const int* __restrict__ active,
                                                        const SegChunk* __restrict__ ch, int nch) {
  double* out = V + ldv * (ctrl ? ctrl[0] + 1 : 0);
  for (int c = blockIdx.x; c < nch; c += gridDim.x) {
    const SegChunk q = ch[c];
    const double d = den[q.seg];
    const bool on = active[q.seg] && d > 0.0;
    const double f = on ? 1.0 / d : 0.0;
    for (long long e = q.b + threadIdx.x; e < q.e; e += kThreads) out[e] = on ? w[e] * f : 0.0;
  }
}

// vin = V_k, k = ctrl[0].
__global__ void k_seg_gather(double* __restrict__ vin, const double* __restrict__ V, long long ldv,
                             const int* __restrict__ ctrl, long long n) {
  const double* v = V + ldv * ctrl[0];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    vin[e] = v[e];
}

// Start of a restart cycle from beta2[s] = ||r_s||^2: the least-squares right-hand side g_s =
// (beta_s, 0, ...), the residual estimate, and which segments iterate (not yet within tolerance, with
// iterations left).  ctrl = (k = 0, active count, NaN seen, max_iters).
__global__ void k_seg_cycle_init(int S, const double* __restrict__ beta2, const double* __restrict__ tol,
                                 double* __restrict__ g, int gs, double* __restrict__ res, int* __restrict__ active,
                                 int* __restrict__ conv, int* __restrict__ kdone, const int* __restrict__ iters,
                                 int max_iters, int* __restrict__ ctrl) {
  __shared__ int cnt[kThreads / 32], bad[kThreads / 32];
  int na = 0, nan = 0;
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    const double beta = sqrt(beta2[s]);
    res[s] = beta;
    kdone[s] = 0;
    double* gg = g + (long long)gs * s;
    for (int q = 0; q < gs; ++q) gg[q] = 0.0;
    gg[0] = beta;
    const bool ok = beta <= tol[s];
    conv[s] = ok ? 1 : 0;
    const bool isnan_ = !(beta == beta);
    nan += isnan_ ? 1 : 0;
    const int a = (!ok && !isnan_ && iters[s] < max_iters) ? 1 : 0;
    active[s] = a;
    na += a;
  }
  for (int o = 16; o > 0; o >>= 1) {
    na += __shfl_xor_sync(0xffffffffu, na, o);
    nan += __shfl_xor_sync(0xffffffffu, nan, o);
  }
  if ((threadIdx.x & 31) == 0) {
    cnt[threadIdx.x >> 5] = na;
    bad[threadIdx.x >> 5] = nan;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int a = 0, b = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
      a += cnt[q];
      b += bad[q];
    }
    ctrl[0] = 0;
    ctrl[1] = a;
    ctrl[2] = b;
    ctrl[3] = max_iters;
  }
}

// Givens step on column k = ctrl[0] of every active segment's Hessenberg matrix (column-major,
// leading dimension ld, hs entries per segment).  On entry wn2[s] = ||w_s||^2 after the
// orthogonalisation; hn[s] receives the new basis norm.  A segment stops when its residual estimate
// |g_s(k + 1)| is within tol[s] (converged) or is not a number, or when it has used ctrl[3]
// iterations.  ctrl[1] = the number of segments still active; ctrl[2] counts NaN estimates.
__global__ void k_seg_givens(int S, double* __restrict__ H, int ld, long long hs, double* __restrict__ cs,
                             double* __restrict__ sn, double* __restrict__ g, int gs, const double* __restrict__ wn2,
                             double* __restrict__ hn, const double* __restrict__ tol, double* __restrict__ res,
                             int* __restrict__ active, int* __restrict__ conv, int* __restrict__ kdone,
                             int* __restrict__ iters, int* __restrict__ ctrl) {
  __shared__ int cnt[kThreads / 32], bad[kThreads / 32];
  const int k = ctrl[0];
  const int max_iters = ctrl[3];
  int na = 0, nan = 0;
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    if (!active[s]) continue;
    double* col = H + hs * s + (long long)k * ld;
    double* c_ = cs + (long long)gs * s;
    double* s_ = sn + (long long)gs * s;
    double* gg = g + (long long)gs * s;
    const double h = sqrt(wn2[s]);
    hn[s] = h;
    col[k + 1] = h;
    for (int i = 0; i < k; ++i) {
      const double a = col[i], b = col[i + 1];
      col[i] = c_[i] * a + s_[i] * b;
      col[i + 1] = -s_[i] * a + c_[i] * b;
    }
    const double a = col[k], b = col[k + 1];
    const double den = hypot(a, b);
    const double cr = den > 0.0 ? a / den : 1.0, sr = den > 0.0 ? b / den : 0.0;
    c_[k] = cr;
    s_[k] = sr;
    col[k] = den;
    col[k + 1] = 0.0;
    gg[k + 1] = -sr * gg[k];
    gg[k] = cr * gg[k];
    const double r = fabs(gg[k + 1]);
    res[s] = r;
    iters[s] += 1;
    kdone[s] = k + 1;
    if (!(r > tol[s])) {
      active[s] = 0;
      if (r == r) {
        conv[s] = 1;
      } else {
        ++nan;
      }
    } else if (iters[s] >= max_iters) {
      active[s] = 0;
    }
    na += active[s];
  }
  for (int o = 16; o > 0; o >>= 1) {
    na += __shfl_xor_sync(0xffffffffu, na, o);
    nan += __shfl_xor_sync(0xffffffffu, nan, o);
  }
  if ((threadIdx.x & 31) == 0) {
    cnt[threadIdx.x >> 5] = na;
    bad[threadIdx.x >> 5] = nan;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int a_ = 0, b_ = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
      a_ += cnt[q];
      b_ += bad[q];
    }
    ctrl[1] = a_;
    ctrl[2] += b_;
  }
}

// End of an Arnoldi step: k += 1; with a graph condition, re-enter the loop body while a segment is
// active and the basis has room.
__global__ void k_seg_step_end(int* __restrict__ ctrl, int m, cudaGraphConditionalHandle handle, int use_handle) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int k = ctrl[0] + 1;
  ctrl[0] = k;
  if (use_handle) cudaGraphSetConditional(handle, (ctrl[1] > 0 && k < m) ? 1u : 0u);
}

// y_s = R_s^{-1} g_s for the kdone[s] x kdone[s] triangle of each segment, stored as y[i * S + s]
// (zero beyond kdone[s], up to m).
__global__ void k_seg_trisolve(int S, const double* __restrict__ H, int ld, long long hs,
                               const double* __restrict__ g, int gs, const int* __restrict__ kdone, int m,
                               double* __restrict__ y) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x) {
    const double* Hs = H + hs * s;
    const double* gg = g + (long long)gs * s;
    const int k = kdone[s];
    for (int i = m - 1; i >= k; --i) y[(long long)i * S + s] = 0.0;
    for (int i = k - 1; i >= 0; --i) {
      double acc = gg[i];
      for (int j = i + 1; j < k; ++j) acc -= Hs[(long long)j * ld + i] * y[(long long)j * S + s];
      y[(long long)i * S + s] = acc / Hs[(long long)i * ld + i];
    }
  }
}

__global__ void k_axpby_g(double* __restrict__ y, double a, const double* __restrict__ x, double b, long long n) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
    y[k] = a * x[k] + b * y[k];
}

int grid_for(const Context& c, long long n) {
  return (int)std::min<long long>(std::max(1, 8 * c.sm_count), std::max<long long>(1, (n + 255) / 256));
}

}  // namespace

// ------------------------------------------------------------------------------------------

Status SegSet::build(const std::vector<long long>& offsets, cudaStream_t s) {
  off = offsets;
  S = (int)off.size() - 1;
  n = off.back();
  std::vector<SegChunk> ch;
  std::vector<int> c0(S + 1, 0);
  for (int q = 0; q < S; ++q) {
    c0[q] = (int)ch.size();
    for (long long b = off[q]; b < off[q + 1]; b += kChunk) {
      SegChunk k;
      k.b = b;
      k.e = std::min(off[q + 1], b + kChunk);
      k.seg = q;
      k.pad = 0;
      ch.push_back(k);
    }
  }
  c0[S] = (int)ch.size();
  nch = (int)ch.size();
  RBS_TRY(d_chunks.alloc(std::max<size_t>(1, ch.size())));
  RBS_TRY(d_c0.alloc(c0.size()));
  if (!ch.empty())
    RBS_CUDA_TRY(cudaMemcpyAsync(d_chunks.ptr, ch.data(), sizeof(SegChunk) * ch.size(), cudaMemcpyHostToDevice, s));
  RBS_CUDA_TRY(cudaMemcpyAsync(d_c0.ptr, c0.data(), sizeof(int) * c0.size(), cudaMemcpyHostToDevice, s));
  RBS_CUDA_TRY(cudaStreamSynchronize(s));  // host vectors go out of scope
  return Status::Ok();
}

void GmresGraphs::release() {
  for (int k = 0; k < kSlots; ++k) {
    if (slot[k].exec) cudaGraphExecDestroy(slot[k].exec);
    slot[k] = Slot();
  }
  if (cap_stream) cudaStreamDestroy(cap_stream);
  cap_stream = nullptr;
}

// Device workspace of the segmented GMRES for S segments of n elements, restart m: reallocated (which
// invalidates captured graphs) only when it grows.
static Status ensure_work(Context& c, const SegSet& sg, long long n, int m) {
  GmresWork& g = c.gw;
  const int S = sg.S;
  const int ld = m + 1, gs = m + 2;
  const long long hs = (long long)ld * (m + 1);
  bool grown = false;
  auto need = [&](DevBuf<double>& b, size_t cnt) -> Status {
    if (b.n < cnt) {
      RBS_TRY(b.alloc(cnt));
      grown = true;
    }
    return Status::Ok();
  };
  auto need_i = [&](DevBuf<int>& b, size_t cnt) -> Status {
    if (b.n < cnt) {
      RBS_TRY(b.alloc(cnt));
      grown = true;
    }
    return Status::Ok();
  };
  RBS_TRY(need(g.H, (size_t)S * hs));
  RBS_TRY(need(g.cs, (size_t)S * gs));
  RBS_TRY(need(g.sn, (size_t)S * gs));
  RBS_TRY(need(g.g, (size_t)S * gs));
  RBS_TRY(need(g.y, (size_t)S * (m + 1)));
  RBS_TRY(need(g.coef, (size_t)S * (m + 1)));
  RBS_TRY(need(g.partial, (size_t)std::max(1, sg.nch) * (m + 1)));
  RBS_TRY(need(g.segd, (size_t)6 * S));  // tol, res, hn, wn2, beta2, spare
  RBS_TRY(need_i(g.segi, (size_t)4 * S + 8));  // active, conv, kdone, iters, then ctrl
  RBS_TRY(need(g.vin, (size_t)n));
  RBS_TRY(need(g.V, (size_t)(m + 1) * n));
  RBS_TRY(need(g.w, (size_t)n));
  RBS_TRY(need(g.z, (size_t)n));
  RBS_TRY(need(g.r, (size_t)n));
  if (g.host_cap < (size_t)6 * S + 8) {
    if (g.host) cudaFreeHost(g.host);
    g.host = nullptr;
    g.hint = g.hctrl = nullptr;
    g.host_cap = 0;
    const size_t nd = (size_t)6 * S + 8, ni = (size_t)4 * S + 8;
    void* p = nullptr;
    RBS_CUDA_TRY(cudaMallocHost(&p, sizeof(double) * nd + sizeof(int) * ni));
    g.host = static_cast<double*>(p);
    g.hint = reinterpret_cast<int*>(g.host + nd);
    g.hctrl = g.hint + 4 * (size_t)S;
    g.host_cap = nd;
  }
  if (grown) ++g.version;
  return Status::Ok();
}

// Per-segment squared norms (or dot products) of vectors of sg.n elements into the device array out
// (S doubles).
Status seg_dot(Context& c, const SegSet& sg, const double* a, const double* b, double* out) {
  GmresWork& g = c.gw;
  dim3 gd(std::min(std::max(1, sg.nch), kDotBlocksX), 1);
  c.stats.launches += 2;
  k_seg_dot<<<gd, kThreads, 0, c.stream>>>(a, 0, nullptr, 0, 1, b, sg.d_chunks.ptr, sg.nch, g.partial.ptr);
  k_seg_reduce<<<dim3(sg.S, 1), kThreads, 0, c.stream>>>(g.partial.ptr, sg.nch, sg.d_c0.ptr, sg.S, nullptr, 0, 1,
                                                         nullptr, nullptr, nullptr, 0, 0, out);
  RBS_CUDA_TRY(cudaGetLastError());
  return Status::Ok();
}

Status seg_norms_host(Context& c, const SegSet& sg, const double* v, std::vector<double>& out) {
  RBS_TRY(ensure_work(c, sg, sg.n, c.opt.restart));
  double* dv = c.gw.segd.ptr + 5 * (size_t)sg.S;
  RBS_TRY(seg_dot(c, sg, v, v, dv));
  RBS_CUDA_TRY(cudaMemcpyAsync(c.gw.host, dv, sizeof(double) * sg.S, cudaMemcpyDeviceToHost, c.stream));
  RBS_CUDA_TRY(cudaStreamSynchronize(c.stream));
  out.assign(c.gw.host, c.gw.host + sg.S);
  for (double& x : out) x = std::sqrt(x);
  return Status::Ok();
}

// One Arnoldi step for every active segment (k = ctrl[0] on the device).
static Status arnoldi_step(Context& c, const LinOp& op, const SegSet& sg, int m, cudaGraphConditionalHandle handle,
                           bool use_handle) {
  GmresWork& g = c.gw;
  const long long n = sg.n;
  const int S = sg.S, ld = m + 1, gs = m + 2;
  const long long hs = (long long)ld * (m + 1);
  int* active = g.segi.ptr;
  int* conv = active + S;
  int* kdone = conv + S;
  int* iters = kdone + S;
  int* ctrl = iters + S;
  double* tol = g.segd.ptr;
  double* res = tol + S;
  double* hn = res + S;
  double* wn2 = hn + S;
  const int nb = grid_for(c, n);
  c.stats.launches += 1;
  k_seg_gather<<<nb, 256, 0, c.stream>>>(g.vin.ptr, g.V.ptr, n, ctrl, n);
  RBS_TRY(op.apply_AP(g.vin.ptr, g.w.ptr, g.z.ptr));
  const dim3 gdot(std::min(std::max(1, sg.nch), kDotBlocksX), m + 1);
  const dim3 gred(S, m + 1);
  const int gcomb = std::min(std::max(1, sg.nch), 8 * std::max(1, c.sm_count));
  for (int pass = 0; pass < 2; ++pass) {
    c.stats.launches += 3;
    k_seg_dot<<<gdot, kThreads, 0, c.stream>>>(g.V.ptr, n, ctrl, 1, 0, g.w.ptr, sg.d_chunks.ptr, sg.nch,
                                                g.partial.ptr);
    k_seg_reduce<<<gred, kThreads, 0, c.stream>>>(g.partial.ptr, sg.nch, sg.d_c0.ptr, S, ctrl, 1, 0, active,
                                                   g.coef.ptr, g.H.ptr, ld, hs, nullptr);
    k_seg_combine<<<gcomb, kThreads, sizeof(double) * (m + 1), c.stream>>>(g.w.ptr, 1.0, g.V.ptr, n, ctrl, 1, 0,
                                                                           g.coef.ptr, S, -1.0, sg.d_chunks.ptr,
                                                                           sg.nch);
  }
  RBS_TRY(seg_dot(c, sg, g.w.ptr, g.w.ptr, wn2));
  c.stats.launches += 3;
  k_seg_givens<<<1, kThreads, 0, c.stream>>>(S, g.H.ptr, ld, hs, g.cs.ptr, g.sn.ptr, g.g.ptr, gs, wn2, hn, tol, res,
                                             active, conv, kdone, iters, ctrl);
  k_seg_scale<<<gcomb, kThreads, 0, c.stream>>>(g.V.ptr, n, ctrl, g.w.ptr, hn, active, sg.d_chunks.ptr, sg.nch);
  k_seg_step_end<<<1, 32, 0, c.stream>>>(ctrl, m, handle, use_handle ? 1 : 0);
  RBS_CUDA_TRY(cudaGetLastError());
  return Status::Ok();
}

// Captures the Arnoldi step of op into a graph whose WHILE node repeats it while the device says so.
// Failure to capture or instantiate leaves the slot marked failed (the solver then runs eagerly).
static Status build_step_graph(Context& c, const LinOp& op, const SegSet& sg, int m, GmresGraphs::Slot& slot) {
  GmresGraphs& G = c.graphs;
  if (!G.cap_stream) RBS_CUDA_TRY(cudaStreamCreateWithFlags(&G.cap_stream, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  RBS_CUDA_TRY(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle handle{};
  cudaError_t e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
  cudaGraphNode_t node = nullptr;
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = handle;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
  cudaGraph_t body = (e == cudaSuccess) ? np.conditional.phGraph_out[0] : nullptr;
  const long long launches0 = c.stats.launches;
  long long count0[RBS_KC_COUNT];
  double units0[RBS_KC_COUNT];
  for (int k = 0; k < RBS_KC_COUNT; ++k) {
    count0[k] = c.stats.kernel_count[k];
    units0[k] = c.stats.kernel_units[k];
  }
  Status st = Status::Ok();
  if (e == cudaSuccess) {
    cudaStream_t saved = c.stream;
    e = cudaStreamBeginCaptureToGraph(G.cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      c.stream = G.cap_stream;
      c.capturing = true;
      st = arnoldi_step(c, op, sg, m, handle, true);
      c.capturing = false;
      c.stream = saved;
      cudaGraph_t out = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(G.cap_stream, &out);
      if (e == cudaSuccess) e = e2;
    }
  }
  slot.launches_per_step = c.stats.launches - launches0;
  c.stats.launches = launches0;
  for (int k = 0; k < RBS_KC_COUNT; ++k) {
    c.stats.kernel_count[k] = count0[k];
    c.stats.kernel_units[k] = units0[k];
  }
  cudaGraphExec_t exec = nullptr;
  if (e == cudaSuccess && st.ok()) e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess || !st.ok() || !exec) {
    if (exec) cudaGraphExecDestroy(exec);
    cudaGetLastError();  // capture failures are not sticky; the eager path takes over
    slot.failed = true;
    return Status::Ok();
  }
  if (slot.exec) cudaGraphExecDestroy(slot.exec);
  slot.exec = exec;
  slot.failed = false;
  return Status::Ok();
}

Status gmres_seg(Context& c, const LinOp& op, const SegSet& sg, const double* b, double* x, bool x_zero,
                 const std::vector<double>& tol_abs, int max_iters, SegResult& out) {
  const long long n = op.n;
  const int S = sg.S;
  const int m = c.opt.restart;
  if (sg.n != n || (int)tol_abs.size() != S) return Status::Err(RBS_EINVAL, "gmres: segment layout mismatch");
  RBS_TRY(ensure_work(c, sg, n, m));
  GmresWork& g = c.gw;
  g.max_iters = std::max(0, max_iters);
  const int ld = m + 1, gs = m + 2;
  const long long hs = (long long)ld * (m + 1);
  int* active = g.segi.ptr;
  int* conv = active + S;
  int* kdone = conv + S;
  int* iters = kdone + S;
  int* ctrl = iters + S;
  double* tol = g.segd.ptr;
  double* res = tol + S;
  double* beta2 = res + 3 * S;
  const int nb = grid_for(c, n);
  const int gcomb = std::min(std::max(1, sg.nch), 8 * std::max(1, c.sm_count));
  double* r = g.r.ptr;

  // tolerances in, iteration counts zeroed
  for (int s = 0; s < S; ++s) g.host[s] = tol_abs[s];
  RBS_CUDA_TRY(cudaMemcpyAsync(tol, g.host, sizeof(double) * S, cudaMemcpyHostToDevice, c.stream));
  RBS_CUDA_TRY(cudaMemsetAsync(iters, 0, sizeof(int) * S, c.stream));
  if (x_zero) RBS_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * n, c.stream));

  // graph slot of this operator, valid for the configuration and workspace it was captured with
  GmresGraphs::Slot* slot = nullptr;
  if (op.graph_key >= 0 && op.graph_key < GmresGraphs::kSlots && c.opt.graphs) {
    slot = &c.graphs.slot[op.graph_key];
    if (slot->config != c.config_version || slot->work != g.version || slot->S != S || slot->m != m) {
      if (slot->exec) cudaGraphExecDestroy(slot->exec);
      *slot = GmresGraphs::Slot();
      slot->config = c.config_version;
      slot->work = g.version;
      slot->S = S;
      slot->m = m;
    }
    if (slot->failed) slot = nullptr;
  }

  bool first = true;
  int cycles = 0;
  while (true) {
    // r = b - A x (x = 0 on the first cycle of a zero start)
    if (first && x_zero) {
      RBS_CUDA_TRY(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, c.stream));
    } else {
      RBS_TRY(op.apply_A(x, r));
      c.stats.launches++;
      k_axpby_g<<<nb, 256, 0, c.stream>>>(r, 1.0, b, -1.0, n);
    }
    first = false;
    RBS_TRY(seg_dot(c, sg, r, r, beta2));
    c.stats.launches += 1;
    k_seg_cycle_init<<<1, kThreads, 0, c.stream>>>(S, beta2, tol, g.g.ptr, gs, res, active, conv, kdone, iters,
                                                   g.max_iters, ctrl);
    RBS_CUDA_TRY(cudaMemcpyAsync(g.hctrl, ctrl, sizeof(int) * 3, cudaMemcpyDeviceToHost, c.stream));
    RBS_CUDA_TRY(cudaStreamSynchronize(c.stream));
    if (g.hctrl[2] > 0) return Status::Err(RBS_ENOTCONV, "GMRES produced NaN");
    if (g.hctrl[1] == 0) break;
    ++cycles;
    RBS_CUDA_TRY(cudaMemsetAsync(g.H.ptr, 0, sizeof(double) * (size_t)S * hs, c.stream));
    c.stats.launches++;
    k_seg_scale<<<gcomb, kThreads, 0, c.stream>>>(g.V.ptr, n, nullptr, r, res, active, sg.d_chunks.ptr, sg.nch);
    int k_host = 0;
    bool cont = true;
    if (slot && !slot->exec) {
      // the first step on this configuration runs eagerly (autotuners settle), then the graph is captured
      RBS_TRY(arnoldi_step(c, op, sg, m, cudaGraphConditionalHandle{}, false));
      RBS_CUDA_TRY(cudaMemcpyAsync(g.hctrl, ctrl, sizeof(int) * 3, cudaMemcpyDeviceToHost, c.stream));
      RBS_CUDA_TRY(cudaStreamSynchronize(c.stream));
      k_host = g.hctrl[0];
      cont = g.hctrl[1] > 0 && k_host < m && g.hctrl[2] == 0;
      RBS_TRY(build_step_graph(c, op, sg, m, *slot));
      if (slot->failed) slot = nullptr;
    }
    if (cont && slot && slot->exec) {
      KernelTimer timer(c, RBS_KC_GMRES_GRAPH);
      RBS_CUDA_TRY(cudaGraphLaunch(slot->exec, c.stream));
      timer.done(0.0, 1);
      RBS_CUDA_TRY(cudaMemcpyAsync(g.hctrl, ctrl, sizeof(int) * 3, cudaMemcpyDeviceToHost, c.stream));
      RBS_CUDA_TRY(cudaStreamSynchronize(c.stream));
      const int steps = g.hctrl[0] - k_host;
      c.stats.launches += slot->launches_per_step * steps;
      c.stats.kernel_units[RBS_KC_GMRES_GRAPH] += steps;
      k_host = g.hctrl[0];
    } else {
      while (cont) {
        RBS_TRY(arnoldi_step(c, op, sg, m, cudaGraphConditionalHandle{}, false));
        RBS_CUDA_TRY(cudaMemcpyAsync(g.hctrl, ctrl, sizeof(int) * 3, cudaMemcpyDeviceToHost, c.stream));
        RBS_CUDA_TRY(cudaStreamSynchronize(c.stream));
        k_host = g.hctrl[0];
        cont = g.hctrl[1] > 0 && k_host < m && g.hctrl[2] == 0;
      }
    }
    if (g.hctrl[2] > 0) return Status::Err(RBS_ENOTCONV, "GMRES produced NaN");
    // x += P (V y), per segment
    c.stats.launches += 1;
    k_seg_trisolve<<<cdiv(S, 128), 128, 0, c.stream>>>(S, g.H.ptr, ld, hs, g.g.ptr, gs, kdone, m, g.y.ptr);
    if (op.apply_P) {
      c.stats.launches++;
      k_seg_combine<<<gcomb, kThreads, sizeof(double) * (m + 1), c.stream>>>(g.w.ptr, 0.0, g.V.ptr, n, nullptr, 0,
                                                                             k_host, g.y.ptr, S, 1.0,
                                                                             sg.d_chunks.ptr, sg.nch);
      RBS_TRY(op.apply_P(g.w.ptr, g.z.ptr, r));
      c.stats.launches++;
      k_axpby_g<<<nb, 256, 0, c.stream>>>(x, 1.0, g.z.ptr, 1.0, n);
    } else {
      c.stats.launches++;
      k_seg_combine<<<gcomb, kThreads, sizeof(double) * (m + 1), c.stream>>>(x, 1.0, g.V.ptr, n, nullptr, 0, k_host,
                                                                             g.y.ptr, S, 1.0, sg.d_chunks.ptr,
                                                                             sg.nch);
    }
    RBS_CUDA_TRY(cudaGetLastError());
    // every segment within its tolerance (by the estimate) or out of iterations: done
    RBS_CUDA_TRY(cudaMemcpyAsync(g.hint, active + S, sizeof(int) * 3 * S, cudaMemcpyDeviceToHost, c.stream));
    RBS_CUDA_TRY(cudaStreamSynchronize(c.stream));
    bool more = false;
    for (int s = 0; s < S; ++s)
      if (!g.hint[s] && g.hint[2 * S + s] < g.max_iters) more = true;
    if (!more) break;
  }
  // results
  RBS_CUDA_TRY(cudaMemcpyAsync(g.hint, active + S, sizeof(int) * 3 * S, cudaMemcpyDeviceToHost, c.stream));
  RBS_CUDA_TRY(cudaMemcpyAsync(g.host, res, sizeof(double) * S, cudaMemcpyDeviceToHost, c.stream));
  RBS_CUDA_TRY(cudaStreamSynchronize(c.stream));
  out.iters.assign(S, 0);
  out.res.assign(S, 0.0);
  out.conv.assign(S, 0);
  for (int s = 0; s < S; ++s) {
    out.conv[s] = (char)(g.hint[s] != 0);
    out.iters[s] = g.hint[2 * S + s];
    out.res[s] = g.host[s];
  }
  out.cycles = cycles;
  return Status::Ok();
}

// Single-system GMRES (one segment spanning op.n elements).
Status gmres_op(Context& c, const LinOp& op, const double* b, double* x, bool x_zero, double tol_abs, int max_iters,
                int* iters, double* res_out, bool* converged) {
  if (c.seg_single.S != 1 || c.seg_single.n != op.n) RBS_TRY(c.seg_single.build({0, op.n}, c.stream));
  SegResult r;
  RBS_TRY(gmres_seg(c, op, c.seg_single, b, x, x_zero, {tol_abs}, max_iters, r));
  *iters = r.iters[0];
  *res_out = r.res[0];
  *converged = r.conv[0] != 0;
  return Status::Ok();
}

}  // namespace rbs
