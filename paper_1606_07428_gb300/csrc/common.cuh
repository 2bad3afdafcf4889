// Internal declarations shared by the translation units of the rbs library.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <memory>
#include <cstdint>
#include <functional>
#include <map>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/rbs.h"

namespace rbs {

struct WarmState;

// Arithmetic classes of the precision codes: float32 pair sums (the mixed modes), and self blocks
// stored in 16 bits (float16 or bfloat16) for the inner solve.
inline bool prec_f32(int prec) {
  return prec == RBS_PREC_MIXED || prec == RBS_PREC_MIXED_FP16 || prec == RBS_PREC_MIXED_BF16;
}
inline bool prec_16(int prec) { return prec == RBS_PREC_MIXED_FP16 || prec == RBS_PREC_MIXED_BF16; }

constexpr double kPi = 3.14159265358979323846;

// Status carried through the host code: RBS_OK or a negative code plus a message.
struct Status {
  int code = RBS_OK;
  std::string msg;
  bool ok() const { return code == RBS_OK; }
  static Status Ok() { return Status(); }
  static Status Err(int c, const std::string& m) {
    Status s;
    s.code = c;
    s.msg = m;
    return s;
  }
};

#define RBS_CUDA_TRY(call)                                                                   \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) {                                                                 \
      return ::rbs::Status::Err(e_ == cudaErrorMemoryAllocation ? RBS_ENOMEM : RBS_ECUDA,    \
                                std::string(#call) + ": " + cudaGetErrorString(e_));         \
    }                                                                                        \
  } while (0)

#define RBS_TRY(expr)              \
  do {                             \
    ::rbs::Status s_ = (expr);     \
    if (!s_.ok()) return s_;       \
  } while (0)

// A device allocation owned by the context.
template <typename T>
struct DevBuf {
  T* ptr = nullptr;
  size_t n = 0;
  Status alloc(size_t count) {
    release();
    if (count == 0) return Status::Ok();
    RBS_CUDA_TRY(cudaMalloc(&ptr, count * sizeof(T)));
    n = count;
    return Status::Ok();
  }
  void release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    n = 0;
  }
  ~DevBuf() { release(); }
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
};

// One parametric grid (p, n_phi) and everything derived from it alone (Section 3, Eq. 33).
struct Grid {
  int p = 0, nphi = 0, np = 0;  // np = (p + 1) * nphi nodes
  int mmax = 0, nbasis = 0;     // retained real harmonics: n <= p, |m| <= min(n, mmax)
  int ps = 0, nrot = 0;         // singular rule order and its point count (ps + 1) * (2 ps + 2)
  int pup = 0, nphi_up = 0, nup = 0;  // upsampled grid for near sources
  std::vector<double> t, lam;         // Gauss-Legendre nodes (ascending) and weights, p + 1
  std::vector<double> t_up, lam_up;   // the same for the upsampled grid
  DevBuf<double> d_t, d_lam, d_t_up, d_lam_up;
  DevBuf<double> d_interp;  // (p + 1) x nrot x np: singular-rule interpolation, target (j, 0)
  DevBuf<double> d_rotpts;  // (p + 1) x nrot x 4: rotated-rule points (x, y, z, weight)
  DevBuf<double> d_up;      // nup x np: interpolation to the upsampled grid
  DevBuf<double> d_an;      // nbasis x np: analysis (grid values -> coefficients)
  DevBuf<double> d_yg;      // np x nbasis: basis values at the grid nodes
  DevBuf<float> d_up32;

  // Reflection symmetry of the grid (reflections x -> -x, y -> -y, z -> -z map nodes to nodes, since
  // the Gauss-Legendre nodes are symmetric and n_phi is even).  Representative nodes are
  // (j, k) with j <= p / 2 and k <= n_phi / 4: nrep = nj * nk of them, one per orbit.
  int nj = 0, nk = 0, nrep = 0;
  std::vector<int> rep_of, g_of;        // per node: its orbit's representative and a reflection taking the representative to it
  std::vector<int> orbit, stab;         // per representative: orbit size, bit mask of the reflections fixing it
  std::vector<int> orb_node, orb_g;     // per representative: its orbit's nodes and the reflection reaching each (8 slots)
  std::vector<int> irrep_pos;           // 8 x 3 nrep: position of (representative, component) in each irrep's basis, or -1
  int irrep_dim[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int dmax = 0;                         // largest irrep dimension
  DevBuf<int> d_sym;                    // device copy of the tables above and each irrep's basis list (see sym_tables)
};

// Offsets of the grid's symmetry tables inside Grid::d_sym.
struct SymTables {
  const int *rep_of, *g_of, *orbit, *orb_node, *orb_g, *irrep_pos, *irrep_list;
};
SymTables sym_tables(const Grid& g);

// One distinct body shape: an ellipsoid (semi-axes) or an input coefficient surface, on one
// (p, n_phi) grid.
struct Shape {
  int kind = 0;  // 0 ellipsoid, 1 coefficient surface
  double a = 0, b = 0, c = 0;
  int cs = -1;   // coefficient surface: index among the inputs
  double radius = 0, rmin = 0;  // largest / smallest centroid distance (near criterion, overlap test)
  int grid = 0;
  int np = 0;
  bool sym = false;      // an ellipsoid: blocks stored as the rows of the representative nodes only
  int rows = 0;          // stored rows: 3 nrep (sym) or 3 np
  size_t block_off = 0;  // offset (in elements) of its rows x 3np blocks in the block arrays
};

// Magnetostatic coupling state (magnetic.cu): scalar self blocks, the preconditioner for the last
// eta, differentiation matrices per grid, and work vectors; built on first use per geometry.
struct MagState {
  bool built = false;
  double eta = 0.0;
  std::vector<long long> block_off;
  DevBuf<long long> d_block_off;
  DevBuf<double> d_blockK, d_blockS, d_precond;
  std::vector<DevBuf<double>*> d_Dt, d_Dp;
  DevBuf<const double*> d_Dt_ptr, d_Dp_ptr, d_upU;
  DevBuf<int> d_grid_of;
  DevBuf<double> d_q, d_b, d_phi, d_hn, d_f, d_qup, d_FT;
  DevBuf<float2> d_wq;
  void release();
  MagState() = default;
  ~MagState();
  MagState(const MagState&) = delete;
  MagState& operator=(const MagState&) = delete;
};

// Barycentric Lagrange treecode for the float32 smooth pair sums (treecode.cu), rebuilt with the
// geometry when rbs_options.far_field is RBS_FAR_TREECODE.
struct TreeItem {  // one work item of the treecode pair sum
  int t0, t1;      // target nodes [t0, t1), all on one particle
  int s0, s1;      // source segments [s0, s1) of that particle's list
  int nmask;       // leading sources of the item that may lie on the target's own particle
  int pad0, pad1, pad2;
};
struct TreeState {
  bool active = false;
  bool df = false;           // sources in the double-float layout (the treecode of the double-float passes)
  int degree = 0, npx = 0;   // interpolation degree and (degree + 1)^3 proxy points per cluster
  int n_cells = 0;           // clusters with proxy points
  int tmax = 0;              // largest target count of a work item
  int nt[3] = {0, 0, 0};     // targets per thread chosen for (traction, Stokeslet, both), 0: not yet
  double theta = 0.0;
  long long n_src = 0;       // sources: N nodes, then n_cells * npx proxy points
  std::vector<TreeItem> items;
  std::vector<int2> segs;    // (first source, count): contiguous runs of the source arrays
  std::vector<int4> charge_items;  // (cluster, first, end) over d_order: the particles of one charge block
  DevBuf<TreeItem> d_items;
  DevBuf<int2> d_segs;
  DevBuf<int4> d_charge_items;
  DevBuf<int> d_order;       // particles in tree order
  DevBuf<double> d_box;      // per cluster with proxies: box midpoint (3), 1 / half-width (3)
  DevBuf<float> d_cheb;      // Chebyshev points, then barycentric weights (degree + 1 each)
  DevBuf<double> d_cheb64;   // the same in float64 (double-float layout)
  // sources for the pair kernel: positions as float32 hi + lo (w of hi: particle id bits, -3 for a
  // proxy point) and float32 weighted density (nodes) or cluster charge (proxy points).  In the
  // double-float layout: positions as exact three-float splits hi + x3m + lo, weighted densities and
  // charges as float32 pairs q + wl, and the charges accumulated in float64 (q64, 3 per proxy point)
  DevBuf<float4> d_hi, d_lo, d_q;
  DevBuf<float4> d_x3m, d_wl;
  DevBuf<double> d_q64;
  long long direct_pairs = 0, proxy_pairs = 0, charge_work = 0;
  void release();
};

// Contiguous segments of a vector (the suspensions of a batch) for the segmented GMRES (gmres.cu):
// element offsets, and chunks of at most 4,096 elements that never straddle a segment.
struct SegChunk {
  long long b, e;
  int seg, pad;
};
struct SegSet {
  int S = 0, nch = 0;
  long long n = 0;
  std::vector<long long> off;  // S + 1 element offsets
  DevBuf<SegChunk> d_chunks;
  DevBuf<int> d_c0;            // S + 1: first chunk of each segment
  Status build(const std::vector<long long>& offsets, cudaStream_t s);
};
// Per-segment outcome of a segmented GMRES solve.
struct SegResult {
  std::vector<int> iters;
  std::vector<double> res;   // final residual estimate (absolute)
  std::vector<char> conv;
  int cycles = 0;
};
// Device workspace of the segmented GMRES (Krylov basis, per-segment Hessenberg matrices, rotations,
// coefficients, flags) and pinned host mirrors of its per-segment outputs.
struct GmresWork {
  DevBuf<double> H, cs, sn, g, y, coef, partial, segd, vin, V, w, z, r;
  DevBuf<int> segi;
  double* host = nullptr;  // host_cap doubles, then 4 S + 8 ints (hint), the last 8 of them hctrl
  int* hint = nullptr;
  int* hctrl = nullptr;
  size_t host_cap = 0;
  int max_iters = 0;
  long long version = 0;  // bumped when a buffer is reallocated (captured graphs hold its pointers)
  GmresWork() = default;
  ~GmresWork() {
    if (host) cudaFreeHost(host);
  }
  GmresWork(const GmresWork&) = delete;
  GmresWork& operator=(const GmresWork&) = delete;
};
// Captured Arnoldi-step graphs (a WHILE conditional node around one step), one slot per operator and
// arithmetic, each valid for the configuration and workspace it was captured with.
struct GmresGraphs {
  static constexpr int kSlots = 16;
  struct Slot {
    cudaGraphExec_t exec = nullptr;
    long long config = -1, work = -1;
    int S = 0, m = 0;
    bool failed = false;
    long long launches_per_step = 0;
  };
  Slot slot[kSlots];
  cudaStream_t cap_stream = nullptr;
  void release();
  GmresGraphs() = default;
  ~GmresGraphs() { release(); }
  GmresGraphs(const GmresGraphs&) = delete;
  GmresGraphs& operator=(const GmresGraphs&) = delete;
};

// Particles sharing one ellipsoid shape whose 16-bit self blocks are applied as a GEMM on the tensor
// cores (selfgemm.cu): the full body-frame blocks K0 and P0 (3 N_p rows, row pitch Kp, 16-bit, scaled
// by ascale), the packed body-frame inputs Z (one row per particle), and their TMA descriptors.
constexpr int kGemmMinParticles = 64;
struct GemmGroup {
  int shape = 0, np = 0, Kp = 0, rows = 0;
  std::vector<int> parts;
  DevBuf<int> d_list;
  DevBuf<uint16_t> K, P, Z;
  DevBuf<float> inv;
  DevBuf<double> mom;
  float ascaleK = 1.0f, ascaleP = 1.0f;
  CUtensorMap tmZ, tmK, tmP;
  double flops = 0.0;  // tensor-core flops issued since creation
};

struct Context {
  rbs_options opt{};
  cudaStream_t stream = nullptr;
  std::string err;
  int device = 0;
  int sm_count = 0;

  // geometry (host)
  int n = 0;
  long long N = 0;  // total nodes
  std::vector<double> axes, centres, quats, rot;  // rot: n x 9 row-major R
  std::vector<int> p, nphi, sid, shape_of;
  std::vector<long long> offset;  // n + 1
  std::vector<Grid*> grids;
  std::vector<Shape> shapes;
  size_t block_elems = 0;  // sum over shapes of (3 np)^2
  double particle_block_entries = 0;  // sum over particles of (3 np)^2 (entries read per block apply)
  double near_pair_nodes = 0;         // sum over near pairs of np_i (nup_j + np_j)
  bool have_geometry = false;

  // per-particle device data
  std::vector<int> grid_of;
  DevBuf<long long> d_gtab_off, d_gtab_up_off;  // per particle: its grid's (t, lambda) in d_gtab
  DevBuf<double> d_gtab, d_axes;
  DevBuf<int> d_p, d_nphi, d_pup;
  DevBuf<double> d_centre, d_rot, d_area, d_tauinv;  // n x 3, n x 9, n, n x 9
  DevBuf<int> d_shape, d_nodes;                      // n: shape id, node count
  DevBuf<long long> d_offset;                        // n + 1
  // per-node device data
  DevBuf<double4> d_x;  // lab position, w = quadrature weight
  // the same positions as unevaluated float32 sums hi + lo (w of hi: the particle id's bits), the
  // normals in float32, and a float32 weighted density w mu per node rebuilt by each packed float32
  // pair sum
  DevBuf<float4> d_xhi, d_xlo, d_wmu32, d_nrm32;
  // for the double-float kernels: positions as exact sums of three float32 numbers (hi has the
  // particle id's bits in w), normals and the per-pass weighted density as hi + lo float32 pairs
  DevBuf<float4> d_x3h, d_x3m, d_x3l, d_nrmh, d_nrml, d_wmuh, d_wmul;
  DevBuf<double4> d_nrm;  // lab normal, w = unused
  DevBuf<int> d_pid;
  // coefficient surfaces of rbs_set_geometry_sh (empty: every particle is an ellipsoid): per
  // particle its input surface, per input surface its degree and first coefficient
  std::vector<int> cs_of, cs_pg;
  std::vector<long long> cs_off;
  std::vector<double> cs_coef;
  // shape-level device data (per distinct shape): kind, semi-axes, degree, coefficient offset
  // (into d_sh_coef, -1 for none) and the centroid shift of a coefficient surface
  DevBuf<int> d_sh_kind, d_sh_pg;
  DevBuf<double> d_sh_axes, d_sh_coef, d_sh_shift;
  DevBuf<long long> d_sh_coef_off;
  DevBuf<double> d_blockK, d_blockS, d_precond;  // body-frame 3np x 3np per shape, float64
  DevBuf<float> d_blockK32, d_precond32;
  // 16-bit copies (float16 or bfloat16 bits, as the context's precision says) of K0 and P0 for the
  // inner solve of RBS_PREC_MIXED_FP16 / RBS_PREC_MIXED_BF16
  DevBuf<uint16_t> d_blockK16, d_precond16;
  DevBuf<long long> d_block_off;  // nshape

  // near-field data
  std::vector<int2> near_pairs;   // (target particle, source particle)
  DevBuf<int2> d_near;
  std::vector<int> up_index;      // per particle: index into upsampled-source list or -1
  std::vector<long long> up_offset;  // per upsampled source particle: first upsampled node
  std::vector<int> up_particle;
  long long n_up_nodes = 0;
  DevBuf<double4> d_up_x;          // upsampled lab nodes (x, y, z, weight)
  DevBuf<long long> d_up_off;      // per upsampled source particle
  DevBuf<int> d_up_particle, d_up_index;
  DevBuf<double> d_up_mu;          // upsampled densities, n_up_nodes x 3

  // particle-block work lists: particles whose shape stores every row, as (particle, first node,
  // end node, 0) items of 24 nodes; particles whose shape stores representative rows, one per block
  std::vector<int4> bwork;
  DevBuf<int4> d_bwork;
  std::vector<int> sym_list;
  DevBuf<int> d_sym_list;
  // 16-bit modes: shape groups applied by GEMM, and the other ellipsoids (sym_rest)
  std::vector<std::unique_ptr<GemmGroup>> gemm;
  std::vector<int> sym_rest;
  DevBuf<int> d_sym_rest;
  DevBuf<int> d_gemm_err;
  int max_np_sym = 0;
  int max_np = 0;
  int max_np_shape = 0;
  // per upsampled-source particle: interpolation matrix of its grid (float64 and float32)
  DevBuf<const double*> d_upU;
  DevBuf<const float*> d_upU32;

  std::map<const void*, int> resident;  // kernel -> resident blocks per SM
  // chosen targets per thread: (float32, double-float) x (K, S), then the fused double-float K + S
  int tuned[5] = {0, 0, 0, 0, 0};
  float tune_ms[5] = {0, 0, 0, 0, 0};

  // smooth pair-sum work list: (target begin, target end, source begin, source end)
  std::vector<longlong4> work;
  DevBuf<longlong4> d_work;

  // scratch vectors (3N doubles each) and GMRES workspace
  DevBuf<double> d_vec[10];
  DevBuf<double> d_partials;
  DevBuf<double> d_FT;  // forces and torques, n x 6
  DevBuf<double> d_vo;  // velocities, n x 6
  double* h_pinned = nullptr;

  // segmented GMRES: the suspensions as segments of 3N-vectors, a one-segment set for single systems,
  // the workspace and the captured step graphs; config_version counts configuration rebuilds
  SegSet seg3, seg_single;
  GmresWork gw;
  GmresGraphs graphs;
  long long config_version = 0;
  bool capturing = false;  // kernels are being captured into a graph: no timing events
  // per-suspension outcome of the last mobility solve: iterations and relative residuals
  std::vector<int> susp_iters;
  std::vector<double> susp_res;

  // contacts of the last mobility solve (Section 3.4): particles i < j, point x*, force f on i
  struct Contact {
    int i, j;
    double x[3], f[3];
  };
  std::vector<Contact> contacts;

  MagState mag;  // magnetostatic coupling (magnetic.cu)
  TreeState tree;     // treecode for the float32 smooth sums (treecode.cu)
  TreeState tree_df;  // treecode for the double-float smooth sums (RBS_FAR_TREECODE_DF)

  rbs_stats stats{};
  WarmState* warm = nullptr;       // learned warm start (warmstart.cu)
  DevBuf<double> d_prev;           // last solved density (previous-solution warm start)
  bool have_prev = false;
  DevBuf<double> d_pred_prev;      // the network's guess at the last solve (RBS_WARM_LEARNED_DELTA)
  bool have_pred = false;
  // kernel timing: (class, start, stop, units) of launches not yet harvested
  struct Timed {
    int cls;
    cudaEvent_t a, b;
    double units;
  };
  std::vector<Timed> pending;
  std::vector<cudaEvent_t> free_events;
  Status time_begin(int cls, Timed* t);
  Status time_end(Timed* t, double units);
  Status harvest();

  Context() = default;
  ~Context();
  Context(const Context&) = delete;
  Context& operator=(const Context&) = delete;
};

// A linear operator for gmres_op on device vectors of length n: w = A P v (z = P v), y = A x, and the
// right preconditioner z = P v (empty: none; aux is scratch of length n).
struct LinOp {
  long long n = 0;
  int graph_key = -1;  // >= 0: the Arnoldi step of this operator may run as a captured graph (slot)
  std::function<Status(const double* v, double* w, double* z)> apply_AP;
  std::function<Status(const double* x, double* y)> apply_A;
  std::function<Status(const double* v, double* z, double* aux)> apply_P;
};
Status gmres_op(Context& c, const LinOp& op, const double* b, double* x, bool x_zero, double tol_abs, int max_iters,
                int* iters, double* res_out, bool* converged);
// GMRES for every segment of sg at once (the operator must not couple segments): segment s stops when
// its residual estimate is within tol_abs[s] or after max_iters iterations.
Status gmres_seg(Context& c, const LinOp& op, const SegSet& sg, const double* b, double* x, bool x_zero,
                 const std::vector<double>& tol_abs, int max_iters, SegResult& out);
// Per-segment dot products a . b into the device array out (S doubles); per-segment norms to the host.
Status seg_dot(Context& c, const SegSet& sg, const double* a, const double* b, double* out);
Status seg_norms_host(Context& c, const SegSet& sg, const double* v, std::vector<double>& out);

// ---- magnetostatic coupling (magnetic.cu)
// Net magnetic force and torque (n x 6 interleaved, device) of the current geometry in the uniform
// field H0 with permeability ratio mu / mu0; q_out (host, total_nodes, may be NULL) receives q.
Status magnetic_forces(Context& c, const double H0[3], double mu_ratio, double tol, double* FT_dev, double* q_out,
                       int* iters);
// y = K^L x (kind 0) or S^L x (kind 1), scalar fields on the nodes (device).
Status laplace_operator(Context& c, int kind, const double* x, double* y);

// ---- treecode (treecode.cu)
// Host inputs of the treecode plan: per particle its first node (offset, n + 1 entries), centre,
// bounding radius, suspension id and node bounding box (lo x, y, z, hi x, y, z).
struct PlanInput {
  int n;
  const long long* offset;
  const double* centres;
  const double* radius;
  const int* sid;
  const double* pbox;
  double near_delta;
  int sm_count;  // sizes the work split (about 96 items per SM)
};
// The plan: tree, interaction lists as source segments (nodes first, then (degree + 1)^3 proxy points
// per accepted cluster), work items, cluster boxes, proxy positions and charge blocks.
struct TreePlan {
  std::vector<TreeItem> items;
  std::vector<int2> segs;
  std::vector<int4> charge_items;
  std::vector<int> corder;
  std::vector<double> box, proxy;
  int n_cells = 0, tmax = 0;
  long long n_src = 0, direct_pairs = 0, proxy_pairs = 0, charge_work = 0;
};
// Host only: no device work (also usable without a GPU).
Status plan_treecode(const PlanInput& in, double theta, int degree, TreePlan& plan);
// Builds (or clears) the treecode of the current geometry; called after the near-pair lists.
Status build_far_field(Context& c);
// y += the treecode's float32 smooth pair sum of kind (0 traction, 1 Stokeslet) for density x, with
// nt targets per thread (1, 2 or 4; 0: the fastest, timed once per geometry).
Status apply_tree(Context& c, int kind, const double* x, double* y, int nt);
// The same for the double-float passes: y += kind 0 or 1 sum; kind 2: y += traction, y2 += Stokeslet.
Status apply_tree_df(Context& c, int kind, const double* x, double* y, double* y2);
// Relative error assumed for a float32 operator application: rounding plus, with the treecode,
// its approximation model C(theta) rho^-n.
double f32_operator_error(const Context& c);

// ---- setup (setup.cu)
Status build_geometry(Context& c);
Status place_particles(Context& c);
Status build_near(Context& c);
// Host only: the reflection-symmetry tables of a (p, n_phi) grid (see rbs_grid_symmetry).
Status grid_symmetry_host(int p, int nphi, std::vector<int>& rep_of, std::vector<int>& g_of, int irrep_dim[8],
                          int* nrep);
// Host only: the near pairs of centres with bounding radii R and inscribed radii rmin (see build_near).
Status plan_near(int n, const double* centres, const double* R, const double* rmin, const int* sid, double delta,
                 std::vector<int2>& out);
Status update_configuration(Context& c, const double* centres, const double* quats);
void gauss_legendre_newton(int n, std::vector<double>& t, std::vector<double>& w);

// ---- self blocks by tensor-core GEMM (selfgemm.cu)
Status build_self_gemm(Context& c);
Status apply_self_gemm(Context& c, int mode, const double* x, double* y, double* aux, double scale);
Status check_self_gemm(Context& c);

// ---- dense kernels (linalg.cu)
Status dgemm_batched(cudaStream_t s, int M, int N, int K, const double* A, long long lda, long long strideA,
                     const double* B, long long ldb, long long strideB, double* C, long long ldc, long long strideC,
                     int batch);
Status invert_batched(Context& c, double* mats, int n, int count);

// ---- operator pieces (operators.cu)
// Particle-block kernel modes.
// Pair-kernel variant code: targets per thread, plus kPacked for the packed-float32 kernels.
constexpr int kPacked = 8;

enum BlockMode {
  kModeSelfK = 0,      // y = 1/2 x + R K0 R^T x + L x      (system operator, self part)
  kModeSelfKNoL = 1,   // y = 1/2 x + R K0 R^T x            (right-hand-side operator, self part)
  kModeSelfS = 2,      // y = R S0 R^T x
  kModeKOnlySelf = 3,  // y = R K0 R^T x
  kModeL = 4,          // y = L x
  kModePrecond = 5,    // y = R P0 R^T x, and copy x to aux
  kModeZero = 6,       // y = 0
};
Status apply_blocks(Context& c, int mode, int prec, const double* x, double* y, double* aux, double scale);
Status apply_pairs(Context& c, int kind, int prec, const double* x, double* y);  // y += off-diagonal kind (0 K, 1 S)
// yK += off-diagonal K x and yS += off-diagonal S x in one pass over the pairs (double-float)
Status apply_pairs_both(Context& c, int prec, const double* x, double* yK, double* yS);
Status apply_operator(Context& c, int op, int prec, const double* x, double* y);

// ---- solver (solver.cu)
Status mobility_solve(Context& c, const double* F, const double* T, double tol, double* v, double* om,
                      double* density, int* iters, bool device_io);
Status incident_density(Context& c, const double* FT_dev, double* rho);
Status rigid_velocities(Context& c, const double* u, double* vo_dev);

// ---- learned warm start (warmstart.cu)
Status warm_prepare(Context& c);
Status warm_guess(Context& c, const double* FT_dev, double* mu0);
Status warm_record(Context& c, const double* FT_dev, const double* mu);
Status warm_train(Context& c, int epochs, int batch, double lr, unsigned seed, double* final_loss);
Status warm_weights(Context& c, float* out, const float* in, long long* count, float* scale_inout);
Status warm_features_host(Context& c, const double* F, const double* T, float* X);
Status warm_targets_host(Context& c, const double* mu, float* coef);
Status warm_mlp_host(Context& c, int rows, const float* X, const float* Yt, float* Y, float* grads, double* loss);
void warm_release(Context& c);

// ---- time stepping (timestep.cu)
Status advance(Context& c, const double* F, const double* T, double dt, int steps, int scheme, double tol, int* iters);

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// Shared memory of the reflection-symmetric block kernel (one CTA of kSymWarps warps per particle):
// a ring of block-row copies (lane_bytes a lane), the eight reflected inputs z_g with row stride
// sym_zstride, and, for float32 arithmetic, the row sums of every node until the block-wide finish.
constexpr int kSymWarps = 8;
__host__ __device__ constexpr int sym_lane_bytes(int ts_bytes) { return ts_bytes == 8 ? 96 : 192; }
// at least 64 ceil(3 N_p / 64) entries and an odd number of 16-byte units, so that the eight rows
// read at one column offset fall in distinct shared-memory banks
__host__ __device__ inline int sym_zstride(int dim, int tb_bytes) { return (dim + 63) / 64 * 64 + 16 / tb_bytes; }
__host__ __device__ inline long long sym_smem_bytes(int np, int ts_bytes, int tb_bytes) {
  return (long long)kSymWarps * 32 * sym_lane_bytes(ts_bytes) + 8LL * sym_zstride(3 * np, tb_bytes) * tb_bytes +
         (tb_bytes == 4 ? 3LL * np * tb_bytes : 0);
}

// Conversions between float64 and float32 from the IEEE 754 bit fields on the integer pipe (GB300's
// float64 pipe, 2 operations per clock per SM, would bound kernels that only widen or narrow): the
// exponent is re-biased by 1023 - 127 and the significand widened or truncated.  Finite values of the
// float32 range only; magnitudes below 2^-126 give signed zero, and narrowing truncates (an error
// below one float32 ulp).
__device__ __forceinline__ double f32_to_f64_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned hi = (u & 0x80000000u) | (e ? (((e + 896u) << 20) | ((u & 0x7fffffu) >> 3)) : 0u);
  const unsigned lo = e ? (u << 29) : 0u;
  return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ float f64_to_f32_trunc(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const int e = (int)((hi >> 20) & 0x7ffu) - 896;
  if (e <= 0) return __uint_as_float(hi & 0x80000000u);
  return __uint_as_float((hi & 0x80000000u) | ((unsigned)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}

// Brackets one timed launch: records events only when timing is on; always counts the launch.
struct KernelTimer {
  Context& c;
  Context::Timed t{};
  bool on;
  KernelTimer(Context& ctx, int cls) : c(ctx), on(ctx.opt.timing != 0 && !ctx.capturing) {
    t.cls = cls;
    if (on && !c.time_begin(cls, &t).ok()) on = false;
  }
  void done(double units, int launches = 1) {
    c.stats.launches += launches;
    c.stats.kernel_count[t.cls] += launches;
    c.stats.kernel_units[t.cls] += units;
    if (on) c.time_end(&t, units);
  }
};

}  // namespace rbs

struct rbs_ctx {
  rbs::Context c;
};
