"""Thin Python binding of the C ABI in include/rbs.h (argument marshalling only).

Every function named rbs_* calls the C function of the same name in librbs.so; all arithmetic of the
method runs in the library's CUDA kernels.  Host arrays are numpy float64 / int32; the *_device
variants take torch CUDA tensors (or raw device addresses).  Loading fails loudly when the library
has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librbs.so")

RBS_OK = 0
RBS_EINVAL = -1
RBS_EOVERLAP = -2
RBS_ENOTCONV = -3
RBS_ECUDA = -4
RBS_ENOMEM = -5
RBS_ETIMEOUT = -6
RBS_ESTATE = -7

RBS_PREC_FP64 = 0
RBS_PREC_MIXED = 1
RBS_PREC_MIXED_FP16 = 2
RBS_PREC_DF = 3
RBS_PREC_MIXED_BF16 = 4

RBS_OP_A = 0
RBS_OP_HALF_K = 1
RBS_OP_S = 2
RBS_OP_K_OFF = 3
RBS_OP_K_SELF = 4
RBS_OP_S_OFF = 5
RBS_OP_S_SELF = 6
RBS_OP_L = 7

# every symbol include/rbs.h declares
EXPORTS = [
    "rbs_default_options", "rbs_create", "rbs_destroy", "rbs_set_geometry", "rbs_total_nodes",
    "rbs_get_surface", "rbs_mobility_solve", "rbs_mobility_solve_device", "rbs_incident_density",
    "rbs_rigid_velocities", "rbs_apply_operator", "rbs_apply_operator_device", "rbs_get_stats",
    "rbs_reset_stats", "rbs_last_error", "rbs_rigid_velocities_noalloc", "rbs_advance", "rbs_get_state",
    "rbs_warmstart_record", "rbs_warmstart_train", "rbs_warmstart_weights", "rbs_warmstart_features",
    "rbs_warmstart_targets", "rbs_warmstart_mlp", "rbs_set_geometry_sh", "rbs_get_contacts",
    "rbs_magnetic_forces", "rbs_apply_laplace", "rbs_treecode_plan", "rbs_near_plan",
    "rbs_grid_symmetry", "rbs_suspension_count", "rbs_get_suspension_results",
]

RBS_MAX_SHAPE_DEGREE = 24

RBS_WARM_ZERO = 0
RBS_WARM_PREVIOUS = 1
RBS_WARM_LEARNED = 2
RBS_WARM_LEARNED_DELTA = 3

RBS_RK_EULER = 1
RBS_RK_TRAPEZOID = 2
RBS_RK4 = 4


class rbs_options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("restart", ctypes.c_int),
        ("max_iters", ctypes.c_int),
        ("preconditioner", ctypes.c_int),
        ("near_delta", ctypes.c_double),
        ("p_up_factor", ctypes.c_int),
        ("p_self_factor", ctypes.c_int),
        ("viscosity", ctypes.c_double),
        ("inner_tol", ctypes.c_double),
        ("max_refinements", ctypes.c_int),
        ("device", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("timing", ctypes.c_int),
        ("refine_precision", ctypes.c_int),
        ("pair_variant", ctypes.c_int),
        ("warm_start", ctypes.c_int),
        ("warm_record", ctypes.c_int),
        ("contact_gap", ctypes.c_double),
        ("magnetic_field", ctypes.c_double * 3),
        ("mu_ratio", ctypes.c_double),
        ("far_field", ctypes.c_int),
        ("tree_theta", ctypes.c_double),
        ("tree_degree", ctypes.c_int),
        ("tree_df_theta", ctypes.c_double),
        ("tree_df_degree", ctypes.c_int),
        ("graphs", ctypes.c_int),
    ]


RBS_FAR_DIRECT = 0
RBS_FAR_TREECODE = 1
RBS_FAR_TREECODE_DF = 2


RBS_KC_PAIR_K32 = 0
RBS_KC_PAIR_S32 = 1
RBS_KC_PAIR_K64 = 2
RBS_KC_PAIR_S64 = 3
RBS_KC_BLOCKS = 4
RBS_KC_NEAR = 5
RBS_KC_PAIR_KDF = 6
RBS_KC_PAIR_SDF = 7
RBS_KC_PAIR_KSDF = 8
RBS_KC_TREE = 9
RBS_KC_GMRES_GRAPH = 10
RBS_KC_SELF_GEMM = 11
RBS_KC_BLOCKS_F64 = 12
RBS_KC_COUNT = 13
KERNEL_CLASSES = ["pair_traction_f32", "pair_stokeslet_f32", "pair_traction_f64", "pair_stokeslet_f64",
                  "particle_blocks", "near_correction", "pair_traction_df", "pair_stokeslet_df", "pair_both_df",
                  "tree_charges", "gmres_graph", "self_gemm", "particle_blocks_f64"]


class rbs_stats(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int),
        ("refinements", ctypes.c_int),
        ("residual", ctypes.c_double),
        ("setup_ms", ctypes.c_double),
        ("solve_ms", ctypes.c_double),
        ("total_nodes", ctypes.c_longlong),
        ("n_particles", ctypes.c_int),
        ("n_shapes", ctypes.c_int),
        ("near_pairs", ctypes.c_longlong),
        ("far_pairs", ctypes.c_longlong),
        ("launches", ctypes.c_longlong),
        ("kernel_ms", ctypes.c_double * RBS_KC_COUNT),
        ("kernel_count", ctypes.c_longlong * RBS_KC_COUNT),
        ("kernel_units", ctypes.c_double * RBS_KC_COUNT),
        ("n_contacts", ctypes.c_int),
        ("pair_variant", ctypes.c_int * 5),
        ("tree_pairs", ctypes.c_longlong),
        ("tree_proxy_pairs", ctypes.c_longlong),
        ("tree_cells", ctypes.c_int),
        ("tree_df_pairs", ctypes.c_longlong),
        ("tree_df_proxy_pairs", ctypes.c_longlong),
        ("tree_df_cells", ctypes.c_int),
    ]


class RbsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rbs error {code}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load librbs.so (built by paper_1606_07428_gb300.build); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first (python -m paper_1606_07428_gb300.build)")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    D = ctypes.c_double
    I = ctypes.c_int
    sig = {
        "rbs_default_options": (None, [ctypes.POINTER(rbs_options)]),
        "rbs_create": (I, [ctypes.POINTER(rbs_options), ctypes.POINTER(P)]),
        "rbs_destroy": (None, [P]),
        "rbs_set_geometry": (I, [P, I, P, P, P, P, P, P]),
        "rbs_set_geometry_sh": (I, [P, I, I, P, P, P, P, P, P, P, P]),
        "rbs_get_contacts": (I, [P, I, P, P, P]),
        "rbs_magnetic_forces": (I, [P, P, D, D, P, P, P, P]),
        "rbs_apply_laplace": (I, [P, I, P, P]),
        "rbs_total_nodes": (ctypes.c_longlong, [P]),
        "rbs_get_surface": (I, [P, P, P, P]),
        "rbs_mobility_solve": (I, [P, P, P, D, P, P, P, P]),
        "rbs_mobility_solve_device": (I, [P, P, P, D, P, P, P, P]),
        "rbs_incident_density": (I, [P, P, P, P]),
        "rbs_rigid_velocities": (I, [P, P, P, P]),
        "rbs_rigid_velocities_noalloc": (I, [P, P, P, P]),
        "rbs_advance": (I, [P, P, P, D, I, I, D, P]),
        "rbs_get_state": (I, [P, P, P]),
        "rbs_warmstart_record": (I, [P, P, P]),
        "rbs_warmstart_train": (I, [P, I, I, D, ctypes.c_uint, P]),
        "rbs_warmstart_weights": (I, [P, P, P, P, P]),
        "rbs_warmstart_features": (I, [P, P, P, P]),
        "rbs_warmstart_targets": (I, [P, P, P]),
        "rbs_warmstart_mlp": (I, [P, I, P, P, P, P, P]),
        "rbs_apply_operator": (I, [P, I, I, P, P]),
        "rbs_apply_operator_device": (I, [P, I, I, P, P]),
        "rbs_get_stats": (I, [P, ctypes.POINTER(rbs_stats)]),
        "rbs_reset_stats": (I, [P]),
        "rbs_last_error": (ctypes.c_char_p, [P]),
        "rbs_treecode_plan": (I, [I, P, P, P, P, P, D, I, D, I, P]),
        "rbs_near_plan": (I, [I, P, P, P, P, D, I, P]),
        "rbs_grid_symmetry": (I, [I, I, P, P, P]),
        "rbs_suspension_count": (I, [P]),
        "rbs_get_suspension_results": (I, [P, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a) -> int | None:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return int(a)


def _f64(a, shape=None) -> np.ndarray:
    out = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        out = out.reshape(shape)
    return out


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def rbs_default_options() -> rbs_options:
    o = rbs_options()
    load().rbs_default_options(ctypes.byref(o))
    return o


def _check(ctx, rc: int, allow=()):
    if rc != RBS_OK and rc not in allow:
        msg = load().rbs_last_error(ctx).decode() if ctx else ""
        raise RbsError(rc, msg)
    return rc


def rbs_create(options: rbs_options | None = None, **kw) -> int:
    o = options or rbs_default_options()
    for k, v in kw.items():
        setattr(o, k, v)
    h = ctypes.c_void_p()
    rc = load().rbs_create(ctypes.byref(o), ctypes.byref(h))
    if rc != RBS_OK:
        raise RbsError(rc, "rbs_create failed")
    return h.value


def rbs_destroy(ctx) -> None:
    load().rbs_destroy(ctx)


def rbs_set_geometry(ctx, semi_axes, p, nphi, centres, quats, suspension_id=None) -> None:
    semi_axes = _f64(semi_axes, (-1, 3))
    n = semi_axes.shape[0]
    p = _i32(np.broadcast_to(p, (n,)))
    nphi = None if nphi is None else _i32(np.broadcast_to(nphi, (n,)))
    centres = _f64(centres, (n, 3))
    quats = _f64(quats, (n, 4))
    sid = None if suspension_id is None else _i32(suspension_id)
    _check(ctx, load().rbs_set_geometry(ctx, n, _ptr(semi_axes), _ptr(p), _ptr(nphi), _ptr(centres), _ptr(quats),
                                        _ptr(sid)))


def rbs_set_geometry_sh(ctx, shapes, shape_of, p, nphi, centres, quats, suspension_id=None) -> None:
    """shapes: list of (coef (3, (pg + 1)^2) in the library's basis order, pg); shape_of: n indices."""
    shape_of = _i32(shape_of)
    n = shape_of.shape[0]
    pg = _i32([int(g) for _, g in shapes])
    coef = _f64(np.concatenate([np.asarray(c, dtype=np.float64).reshape(3, (int(g) + 1) ** 2).ravel()
                                for c, g in shapes]), (-1,))
    p = _i32(np.broadcast_to(p, (n,)))
    nphi = None if nphi is None else _i32(np.broadcast_to(nphi, (n,)))
    centres = _f64(centres, (n, 3))
    quats = _f64(quats, (n, 4))
    sid = None if suspension_id is None else _i32(suspension_id)
    _check(ctx, load().rbs_set_geometry_sh(ctx, n, len(shapes), _ptr(pg), _ptr(coef), _ptr(shape_of), _ptr(p),
                                           _ptr(nphi), _ptr(centres), _ptr(quats), _ptr(sid)))


def rbs_treecode_plan(nodes, centres, radius, node_box, suspension_id=None, theta=0.5, degree=7, near_delta=1.0,
                      sm_count=152) -> dict:
    """Host-only treecode plan (no GPU): direct and proxy pair counts, clusters, work items, segments
    and the largest work item's target count."""
    nodes = _i32(nodes)
    n = nodes.shape[0]
    centres = _f64(centres, (n, 3))
    radius = _f64(radius, (n,))
    node_box = _f64(node_box, (n, 6))
    sid = None if suspension_id is None else _i32(suspension_id)
    out = np.zeros(6, np.int64)
    _check(None, load().rbs_treecode_plan(n, _ptr(nodes), _ptr(centres), _ptr(radius), _ptr(node_box), _ptr(sid),
                                          float(theta), int(degree), float(near_delta), int(sm_count), _ptr(out)))
    keys = ["direct_pairs", "proxy_pairs", "cells", "items", "segments", "tmax"]
    return {k: int(v) for k, v in zip(keys, out)}


def rbs_near_plan(centres, radius, rmin, suspension_id=None, near_delta=1.0) -> np.ndarray:
    """Host-only near pairs (n_pairs, 2) int32, as a context builds them (no GPU)."""
    centres = _f64(centres, (-1, 3))
    n = centres.shape[0]
    radius = _f64(radius, (n,))
    rmin = _f64(rmin, (n,))
    sid = None if suspension_id is None else _i32(suspension_id)
    cnt = _check(None, load().rbs_near_plan(n, _ptr(centres), _ptr(radius), _ptr(rmin), _ptr(sid), float(near_delta),
                                            0, None), allow=range(0, 1 << 31))
    pairs = np.zeros((cnt, 2), np.int32)
    if cnt:
        _check(None, load().rbs_near_plan(n, _ptr(centres), _ptr(radius), _ptr(rmin), _ptr(sid), float(near_delta),
                                          cnt, _ptr(pairs)), allow=range(0, 1 << 31))
    return pairs


def rbs_grid_symmetry(p: int, nphi: int):
    """Host-only symmetry tables of a grid: (representatives, rep_of, g_of, irrep_dim)."""
    np_ = (p + 1) * nphi
    rep_of = np.zeros(np_, np.int32)
    g_of = np.zeros(np_, np.int32)
    dims = np.zeros(8, np.int32)
    nrep = _check(None, load().rbs_grid_symmetry(int(p), int(nphi), _ptr(rep_of), _ptr(g_of), _ptr(dims)),
                  allow=range(0, 1 << 31))
    return nrep, rep_of, g_of, dims


def rbs_get_contacts(ctx):
    """The last solve's contacts: (pairs (n_c, 2) int32, points (n_c, 3), forces on the first particle
    (n_c, 3))."""
    n = _check(ctx, load().rbs_get_contacts(ctx, 0, None, None, None), allow=range(0, 1 << 30))
    pairs = np.zeros((n, 2), np.int32)
    points = np.zeros((n, 3))
    forces = np.zeros((n, 3))
    if n:
        _check(ctx, load().rbs_get_contacts(ctx, n, _ptr(pairs), _ptr(points), _ptr(forces)), allow=range(0, 1 << 30))
    return pairs, points, forces


def rbs_magnetic_forces(ctx, H0, mu_ratio, tol, n, total_nodes=None):
    """Magnetic force and torque (n x 3 each) per particle in the uniform field H0; with total_nodes
    also the single-layer density q."""
    H0 = _f64(H0, (3,))
    F = np.zeros((n, 3))
    T = np.zeros((n, 3))
    q = None if total_nodes is None else np.zeros(total_nodes)
    its = ctypes.c_int(0)
    _check(ctx, load().rbs_magnetic_forces(ctx, _ptr(H0), float(mu_ratio), float(tol), _ptr(F), _ptr(T), _ptr(q),
                                           ctypes.byref(its)))
    return F, T, q, its.value


def rbs_apply_laplace(ctx, kind, x):
    x = _f64(x, (-1,))
    y = np.zeros_like(x)
    _check(ctx, load().rbs_apply_laplace(ctx, int(kind), _ptr(x), _ptr(y)))
    return y


def rbs_total_nodes(ctx) -> int:
    return int(load().rbs_total_nodes(ctx))


def rbs_get_surface(ctx):
    N = rbs_total_nodes(ctx)
    x = np.zeros((N, 3))
    nrm = np.zeros((N, 3))
    w = np.zeros(N)
    _check(ctx, load().rbs_get_surface(ctx, _ptr(x), _ptr(nrm), _ptr(w)))
    return x, nrm, w


def rbs_suspension_count(ctx) -> int:
    return _check(ctx, load().rbs_suspension_count(ctx), allow=range(0, 1 << 31))


def rbs_get_suspension_results(ctx):
    """Per-suspension outcome of the last solve: (iterations int32 array, relative residuals)."""
    S = rbs_suspension_count(ctx)
    its = np.zeros(S, np.int32)
    res = np.zeros(S)
    _check(ctx, load().rbs_get_suspension_results(ctx, _ptr(its), _ptr(res)))
    return its, res


def rbs_mobility_solve(ctx, F, T, tol, want_density=False, allow_notconv=False, per_suspension=False):
    """Returns (v, omega, density or None, iterations): iterations is the per-suspension int32 array
    the C call fills when per_suspension is set, else its largest entry."""
    F = _f64(F, (-1, 3))
    T = _f64(T, F.shape)
    v = np.zeros_like(F)
    om = np.zeros_like(F)
    dens = np.zeros((rbs_total_nodes(ctx), 3)) if want_density else None
    its = np.zeros(max(1, rbs_suspension_count(ctx)), np.int32)
    rc = load().rbs_mobility_solve(ctx, _ptr(F), _ptr(T), float(tol), _ptr(v), _ptr(om), _ptr(dens), _ptr(its))
    _check(ctx, rc, (RBS_ENOTCONV,) if allow_notconv else ())
    return v, om, dens, (its if per_suspension else int(its.max()))


def rbs_mobility_solve_device(ctx, F_dev, T_dev, tol, v_dev, omega_dev, density_dev=None, allow_notconv=False,
                              per_suspension=False):
    its = np.zeros(max(1, rbs_suspension_count(ctx)), np.int32)
    rc = load().rbs_mobility_solve_device(ctx, _ptr(F_dev), _ptr(T_dev), float(tol), _ptr(v_dev), _ptr(omega_dev),
                                          _ptr(density_dev), _ptr(its))
    _check(ctx, rc, (RBS_ENOTCONV,) if allow_notconv else ())
    return its if per_suspension else int(its.max())


def rbs_advance(ctx, F, T, dt, steps, scheme=RBS_RK4, tol=1e-10) -> int:
    F = _f64(F, (-1, 3))
    T = _f64(T, F.shape)
    its = ctypes.c_int(0)
    _check(ctx, load().rbs_advance(ctx, _ptr(F), _ptr(T), float(dt), int(steps), int(scheme), float(tol),
                                   ctypes.addressof(its)))
    return its.value


def rbs_warmstart_record(ctx, F, T) -> None:
    F = _f64(F, (-1, 3))
    T = _f64(T, F.shape)
    _check(ctx, load().rbs_warmstart_record(ctx, _ptr(F), _ptr(T)))


def rbs_warmstart_train(ctx, epochs, batch=256, lr=1e-3, seed=0) -> float:
    loss = ctypes.c_double(0.0)
    _check(ctx, load().rbs_warmstart_train(ctx, int(epochs), int(batch), float(lr), int(seed), ctypes.addressof(loss)))
    return loss.value


def rbs_warmstart_weights(ctx, params: np.ndarray | None = None, scale: float = 1.0):
    """Without params: returns (flattened float32 parameters, output scale).  With params: loads them."""
    count = ctypes.c_longlong(0)
    sc = ctypes.c_float(scale)
    lib = load()
    if params is None:
        _check(ctx, lib.rbs_warmstart_weights(ctx, None, None, ctypes.addressof(count), None))
        out = np.zeros(count.value, np.float32)
        _check(ctx, lib.rbs_warmstart_weights(ctx, _ptr(out), None, None, ctypes.addressof(sc)))
        return out, sc.value
    p = np.ascontiguousarray(params, np.float32)
    _check(ctx, lib.rbs_warmstart_weights(ctx, None, _ptr(p), ctypes.addressof(count), ctypes.addressof(sc)))
    return None


def rbs_warmstart_features(ctx, F, T, n) -> np.ndarray:
    F = _f64(F, (-1, 3))
    T = _f64(T, F.shape)
    X = np.zeros((n, 128), np.float32)
    _check(ctx, load().rbs_warmstart_features(ctx, _ptr(F), _ptr(T), _ptr(X)))
    return X


def rbs_warmstart_targets(ctx, mu, n, n_out) -> np.ndarray:
    mu = _f64(mu, (-1, 3))
    out = np.zeros((n, n_out), np.float32)
    _check(ctx, load().rbs_warmstart_targets(ctx, _ptr(mu), _ptr(out)))
    return out


def rbs_warmstart_mlp(ctx, X, n_out, Yt=None, n_params=None):
    X = np.ascontiguousarray(X, np.float32)
    rows = X.shape[0]
    Y = np.zeros((rows, n_out), np.float32)
    grads = None
    loss = ctypes.c_double(0.0)
    yt = None
    if Yt is not None:
        yt = np.ascontiguousarray(Yt, np.float32)
        grads = np.zeros(n_params, np.float32)
    _check(ctx, load().rbs_warmstart_mlp(ctx, rows, _ptr(X), _ptr(yt), _ptr(Y), _ptr(grads), ctypes.addressof(loss)))
    return Y, grads, loss.value


def rbs_get_state(ctx, n):
    c = np.zeros((n, 3))
    q = np.zeros((n, 4))
    _check(ctx, load().rbs_get_state(ctx, _ptr(c), _ptr(q)))
    return c, q


def rbs_incident_density(ctx, F, T) -> np.ndarray:
    F = _f64(F, (-1, 3))
    T = _f64(T, F.shape)
    rho = np.zeros((rbs_total_nodes(ctx), 3))
    _check(ctx, load().rbs_incident_density(ctx, _ptr(F), _ptr(T), _ptr(rho)))
    return rho


def rbs_rigid_velocities(ctx, u, n):
    u = _f64(u, (-1, 3))
    v = np.zeros((n, 3))
    om = np.zeros((n, 3))
    _check(ctx, load().rbs_rigid_velocities(ctx, _ptr(u), _ptr(v), _ptr(om)))
    return v, om


def rbs_rigid_velocities_noalloc(ctx, u_dev, v_dev, omega_dev) -> None:
    """Device-buffer rigid velocities that allocate nothing (fixed 65,536-particle scratch)."""
    _check(ctx, load().rbs_rigid_velocities_noalloc(ctx, _ptr(u_dev), _ptr(v_dev), _ptr(omega_dev)))


def rbs_apply_operator(ctx, op: int, precision: int, x) -> np.ndarray:
    x = _f64(x, (-1, 3))
    y = np.zeros_like(x)
    _check(ctx, load().rbs_apply_operator(ctx, op, precision, _ptr(x), _ptr(y)))
    return y


def rbs_apply_operator_device(ctx, op: int, precision: int, x_dev, y_dev) -> None:
    _check(ctx, load().rbs_apply_operator_device(ctx, op, precision, _ptr(x_dev), _ptr(y_dev)))


def rbs_get_stats(ctx) -> dict:
    s = rbs_stats()
    _check(ctx, load().rbs_get_stats(ctx, ctypes.byref(s)))
    out = {}
    for name, _ in s._fields_:
        val = getattr(s, name)
        out[name] = list(val) if name.startswith("kernel_") or name == "pair_variant" else val
    return out


def rbs_reset_stats(ctx) -> None:
    _check(ctx, load().rbs_reset_stats(ctx))


def rbs_last_error(ctx) -> str:
    return load().rbs_last_error(ctx).decode()


class Context:
    """Owning wrapper: a context with a geometry, closed on exit."""

    def __init__(self, **options):
        self.ctx = rbs_create(**options)
        self.n = 0

    def set_geometry(self, semi_axes, p, nphi, centres, quats, suspension_id=None):
        rbs_set_geometry(self.ctx, semi_axes, p, nphi, centres, quats, suspension_id)
        self.n = int(np.asarray(semi_axes).reshape(-1, 3).shape[0])
        return self

    def set_shapes(self, shapes, shape_of, p, nphi, centres, quats, suspension_id=None):
        rbs_set_geometry_sh(self.ctx, shapes, shape_of, p, nphi, centres, quats, suspension_id)
        self.n = int(np.asarray(shape_of).reshape(-1).shape[0])
        return self

    def set_suspension(self, s):
        return self.set_geometry(s.semi_axes, s.p, s.nphi, s.centres, s.quats, s.suspension_id)

    def close(self):
        if self.ctx:
            rbs_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
