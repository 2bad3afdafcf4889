"""The learned warm start on the GPU against the oracle's definitions (oracle/warmstart.py), and its
effect on GMRES.

Tolerances: features and target coefficients are float32 outputs of float64 arithmetic (rel. 1e-6);
the network runs on bfloat16 operands with float32 accumulation, so its outputs and gradients are
compared with the float64 oracle evaluated on the same bfloat16-rounded weights and inputs within
3e-2 and 6e-2 (relative L2; bfloat16 keeps 8 significant bits for the hidden activations)."""
import numpy as np
import pytest

import oracle
import oracle.warmstart as ows
import suspensions

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbs():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1606_07428_gb300 import rbs as m
    return m


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


def bf16(a):
    """Round float32 values to bfloat16 (nearest even) and back."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def flatten(params):
    return np.concatenate([params[k].astype(np.float32).ravel() for k in ("W1", "b1", "W2", "b2", "W3", "b3")])


def test_features_and_targets_match_oracle(rbs):
    s = suspensions.random_ellipsoids(40, 4, 10, 0.1, 0.2, seed=61)
    ref = oracle.System(s.semi_axes, s.p, s.nphi, s.centres, s.quats)
    with rbs.Context(device=0) as ctx:
        ctx.set_suspension(s)
        X = rbs.rbs_warmstart_features(ctx.ctx, s.F, s.T, s.n)
        mu = suspensions.random_density(8, s.total_nodes)
        nb = ows.basis_permutation(4, 10).size
        C = rbs.rbs_warmstart_targets(ctx.ctx, mu, s.n, 3 * nb)
    Xr = ows.features(s.semi_axes, s.centres, s.quats, s.F, s.T)
    assert np.abs(X - Xr).max() < 1e-6 * max(1.0, np.abs(Xr).max())
    assert rel(C, ows.target_coefficients(ref, mu)) < 1e-6


def test_network_forward_and_gradients_match_oracle(rbs):
    s = suspensions.random_ellipsoids(6, 4, 8, 0.1, 0.2, seed=62)
    nb = ows.basis_permutation(4, 8).size
    D = 3 * nb
    params = ows.init_params(D, seed=7)
    params = {k: bf16(v.astype(np.float32)).astype(np.float64) for k, v in params.items()}
    rng = np.random.default_rng(9)
    X = bf16(rng.normal(size=(37, 128)).astype(np.float32))
    Yt = rng.normal(size=(37, D)).astype(np.float32)
    with rbs.Context(device=0) as ctx:
        ctx.set_suspension(s)
        flat = flatten(params)
        rbs.rbs_warmstart_weights(ctx.ctx, flat, scale=1.0)
        Y, grads, loss = rbs.rbs_warmstart_mlp(ctx.ctx, X, D, Yt, flat.size)
    y_ref, _ = ows.forward(params, X.astype(np.float64))
    L_ref, g_ref = ows.loss_and_grads(params, X.astype(np.float64), Yt.astype(np.float64))
    assert rel(Y, y_ref) < 3e-2
    assert abs(loss - L_ref) < 3e-2 * L_ref
    off = 0
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        size = params[k].size
        assert rel(grads[off:off + size], g_ref[k]) < 6e-2, k
        off += size


def perturbed(base, seed, amp=0.05):
    s = suspensions.Suspension(**{f: getattr(base, f) for f in ("semi_axes", "p", "nphi", "centres", "quats", "F", "T",
                                                               "suspension_id", "name")})
    rng = np.random.default_rng(seed)
    s.centres = base.centres + amp * rng.normal(size=base.centres.shape)
    return s


def test_learned_warm_start_cuts_iterations_not_the_answer(rbs):
    base = suspensions.random_ellipsoids(64, 6, 12, 0.08, 0.4, seed=63)
    base.F = np.tile([0.0, 0.0, -1.0], (base.n, 1))
    base.T = np.zeros((base.n, 3))
    with rbs.Context(device=0, restart=60) as ctx:
        for k in range(24):
            s = perturbed(base, 100 + k)
            ctx.set_suspension(s)
            rbs.rbs_mobility_solve(ctx.ctx, s.F, s.T, 1e-12)
            rbs.rbs_warmstart_record(ctx.ctx, s.F, s.T)
        loss0 = rbs.rbs_warmstart_train(ctx.ctx, 1, batch=128, lr=1e-3, seed=3)
        loss = rbs.rbs_warmstart_train(ctx.ctx, 300, batch=128, lr=1e-3, seed=3)
        assert loss < 0.2 * loss0
        params, scale = rbs.rbs_warmstart_weights(ctx.ctx)
    test = perturbed(base, 999)
    out = {}
    for mode in ("ZERO", "LEARNED"):
        with rbs.Context(device=0, restart=60, warm_start=getattr(rbs, "RBS_WARM_" + mode)) as ctx:
            ctx.set_suspension(test)
            if mode == "LEARNED":
                rbs.rbs_warmstart_weights(ctx.ctx, params, scale=scale)
            v, om, _, its = rbs.rbs_mobility_solve(ctx.ctx, test.F, test.T, 1e-12)
            out[mode] = (np.concatenate([v, om]), its)
    assert rel(out["LEARNED"][0], out["ZERO"][0]) < 1e-10
    assert out["LEARNED"][1] < out["ZERO"][1]


def test_previous_solution_warm_start(rbs):
    base = suspensions.random_ellipsoids(30, 5, 10, 0.08, 0.4, seed=64)
    with rbs.Context(device=0, warm_start=rbs.RBS_WARM_PREVIOUS) as ctx:
        ctx.set_suspension(base)
        _, _, _, its0 = rbs.rbs_mobility_solve(ctx.ctx, base.F, base.T, 1e-12)
        s = perturbed(base, 5, amp=0.01)
        ctx.set_suspension(s)
        v1, o1, _, its1 = rbs.rbs_mobility_solve(ctx.ctx, s.F, s.T, 1e-12)
    with rbs.Context(device=0) as ctx:
        ctx.set_suspension(s)
        v2, o2, _, its2 = rbs.rbs_mobility_solve(ctx.ctx, s.F, s.T, 1e-12)
    assert rel(np.concatenate([v1, o1]), np.concatenate([v2, o2])) < 1e-10
    assert its1 < its2
