"""GPU parity of the learned-start network against the FP64 oracle (oracle/mlp_oracle.py).

Features are FP64 and must match the oracle's independent point evaluation to 1e-12.
The network runs with BF16 operands and FP32 accumulation, so it is compared with the
FP64 oracle evaluated on the same BF16-rounded weights and inputs: forward within 1e-2
relative, gradients within 2e-2 relative per tensor (2-norm), the loss within 1e-2.
"""
import numpy as np
import pytest

import mlp_oracle as MO
import oracle as O
from paper_2301_05985_gb300 import workloads as W

from gpu_common import lib, perm_to_oracle, torch_cuda

pytestmark = pytest.mark.gpu

SHAPES = [(0, 216, 128), (27776, 128, 128), (44928, 128, 128), (61824, 128, 3)]  # (offset, fan_in, fan_out)


def unpack(p):
    Ws, bs = [], []
    off = 0
    for fi, fo in [(216, 128), (128, 128), (128, 128), (128, 3)]:
        Ws.append(p[off:off + fi * fo].reshape(fi, fo).astype(np.float64)); off += fi * fo
        bs.append(p[off:off + fo].astype(np.float64)); off += fo
    assert off == p.size
    return Ws, bs


def pack(Ws, bs):
    return np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in zip(Ws, bs)]).astype(np.float32)


def _ctx(oc):
    pnp = lib()
    torch = torch_cuda()
    mesh = pnp.Mesh(oc)
    ctx = pnp.Context(mesh, pnp.default_params(eps=0.05, dt=0.01), torch.cuda.current_stream().cuda_stream)
    ctx.mlp_init(seed=1)
    return pnp, torch, mesh, ctx


def test_features_match_oracle_point_evaluation():
    oc = W.random_balanced_octants(3, 1, 4, 0.3, 12)
    pnp, torch, mesh, ctx = _ctx(oc)
    om = O.OracleMesh(oc)
    perm = perm_to_oracle(mesh.ijk, om.ijk, oc.max_level)
    L = oc.max_level
    Uk = W.random_state(mesh.ijk, L, 1)
    Ukm1 = W.random_state(mesh.ijk, L, 2)
    uzk = W.random_velocity(mesh.ijk, L, 3, 1.0)[:, 2].copy()
    uzkm1 = W.random_velocity(mesh.ijk, L, 4, 1.0)[:, 2].copy()
    bc = W.all_natural_bcs(3)
    op = O.Params(eps=0.1, steady=True, bc_type=bc.types, bc_val=bc.values)

    def to_ora(x):
        o = np.zeros_like(x); o[perm] = x; return o

    Uk_o = om.make_consistent(to_ora(Uk), op)
    Ukm1_o = om.make_consistent(to_ora(Ukm1), op)
    Uk_l, Ukm1_l = Uk_o[perm], Ukm1_o[perm]
    nf = int((~mesh.hanging).sum())
    X = torch.zeros((nf, 216), dtype=torch.float64, device="cuda")
    nodes = torch.zeros(nf, dtype=torch.int32, device="cuda")
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    ctx.mlp_features(d(Uk_l), d(Ukm1_l), d(uzk), d(uzkm1), X, nodes)
    X = X.cpu().numpy()
    nodes = nodes.cpu().numpy()
    anc, lev = mesh.elements()
    # oracle elements are in input order; its node sizes come from its own element list
    onodes, F = O.stencil_features(om, oc.levels, Uk_o, Ukm1_o, to_ora(uzk), to_ora(uzkm1))
    ref = np.zeros((mesh.n_nodes, 216))
    ref[np.argsort(perm)[onodes]] = F  # oracle node -> library node
    assert sorted(nodes.tolist()) == sorted(np.argsort(perm)[onodes].tolist())
    err = np.abs(X - ref[nodes]).max() / np.abs(ref).max()
    assert err < 1e-13, err


def test_forward_and_gradients_match_oracle():
    oc = W.uniform_octants(3, 2)
    pnp, torch, mesh, ctx = _ctx(oc)
    rng = np.random.default_rng(5)
    Ws, bs = MO.init_params(7)
    bs = [b + rng.normal(0, 0.05, b.shape) for b in bs]
    p = pack(Ws, bs)
    ctx.mlp_set_weights(p)
    B = 777
    X = rng.normal(size=(B, 216)).astype(np.float32)
    Y = rng.normal(size=(B, 3)).astype(np.float32)
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.from_numpy(Y).cuda()
    out = torch.zeros((B, 3), dtype=torch.float32, device="cuda")
    ctx.mlp_forward(Xd, out)
    out = out.cpu().numpy()
    Wr, br = unpack(p)
    Wr = [MO.bf16_round(w) for w in Wr]
    ref, _, _ = MO.forward(Wr, br, MO.bf16_round(X))
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < 1e-2
    g = torch.zeros(pnp.PNP_MLP_PARAMS, dtype=torch.float32, device="cuda")
    loss = ctx.mlp_loss_grad(Xd, Yd, g)
    g = g.cpu().numpy().astype(np.float64)
    gW, gb, lref = MO.backward(Wr, br, MO.bf16_round(X), Y.astype(np.float64))
    assert abs(loss - lref) / lref < 1e-2
    gWg, gbg = unpack(g)
    for l in range(4):
        assert np.linalg.norm(gWg[l] - gW[l]) / np.linalg.norm(gW[l]) < 2e-2, l
        assert np.linalg.norm(gbg[l] - gb[l]) / np.linalg.norm(gb[l]) < 2e-2, l


def test_inference_spans_many_tiles_per_cta():
    """The tensor-core inference is persistent over 128-row tiles: 38,989 rows are 305
    tiles, two or three per CTA on a 152-SM GPU, the last one ragged (77 rows).  Against
    the oracle with BF16-rounded weights, inputs and hidden activations (what the kernel
    feeds its next layer), and against the unrounded oracle as in the small case."""
    oc = W.uniform_octants(3, 2)
    pnp, torch, mesh, ctx = _ctx(oc)
    rng = np.random.default_rng(11)
    Ws, bs = MO.init_params(3)
    bs = [b + rng.normal(0, 0.05, b.shape) for b in bs]
    p = pack(Ws, bs)
    ctx.mlp_set_weights(p)
    B = 2 * 152 * 128 + 77
    X = rng.normal(size=(B, 216)).astype(np.float32)
    out = torch.zeros((B, 3), dtype=torch.float32, device="cuda")
    ctx.mlp_forward(torch.from_numpy(X).cuda(), out)
    out = out.cpu().numpy().astype(np.float64)
    Wr, br = unpack(p)
    Wr = [MO.bf16_round(w) for w in Wr]
    a = MO.bf16_round(X)
    for l in range(4):
        z = a @ Wr[l] + br[l]
        a = MO.bf16_round(MO.gelu(z)) if l < 3 else z
    assert np.all(np.isfinite(out))
    scale = np.abs(a).max()
    assert np.abs(out - a).max() <= 1e-2 * scale, np.abs(out - a).max() / scale
    assert np.linalg.norm(out - a) / np.linalg.norm(a) < 2e-3
    ref, _, _ = MO.forward(Wr, br, MO.bf16_round(X))
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < 1e-2


def test_weights_round_trip_and_normalization():
    oc = W.uniform_octants(3, 2)
    pnp, torch, mesh, ctx = _ctx(oc)
    p = np.random.default_rng(0).normal(size=pnp.PNP_MLP_PARAMS).astype(np.float32)
    ctx.mlp_set_weights(p)
    assert np.array_equal(ctx.mlp_get_weights(), p)
    ctx.mlp_set_normalization([1, 2, 3, 4], [0.5, 1, 2, 4], [0.1, 0.2, 0.3], [1, 2, 3])
    a, b, c, d = ctx.mlp_get_normalization()
    assert a.tolist() == [1, 2, 3, 4] and d.tolist() == [1, 2, 3]


def test_training_fits_a_solver_trajectory():
    """Record a short trajectory of the solver, train, check the loss falls and the judged
    learned start is never worse than extrapolation."""
    oc = W.uniform_octants(3, 3)
    pnp, torch, mesh, ctx = _ctx(oc)
    bcs = W.equilibrium_bcs(3, 3.0)
    ctx.set_bcs(bcs)
    ctx.set_params(pnp.default_params(eps=0.05, dt=0.01, newton_rtol=1e-10, gmres_rtol=1e-12, gmres_restart=60,
                                      start_mode=pnp.PNP_START_EXTRAPOLATE))
    U0 = W.noisy_state(mesh.ijk, oc.max_level, seed=1, amp=1e-2, phi_bottom=3.0, phi_top=0.0)
    ctx.set_field(pnp.PNP_FIELD_U, U0)
    ctx.make_consistent()
    ctx.reset_history()
    states = [ctx.get_field(pnp.PNP_FIELD_U)]
    for _ in range(24):
        ctx.time_step()
        states.append(ctx.get_field(pnp.PNP_FIELD_U))
    S = torch.from_numpy(np.stack(states)).cuda()
    ctx.mlp_add_trajectory(S)
    st = ctx.mlp_train(steps=300, batch=2048, lr=2e-3, seed=3)
    assert st.loss_last < 0.5 * st.loss_first, st.as_dict()
    p = ctx.get_params(); p.start_mode = pnp.PNP_START_LEARNED
    ctx.set_params(p)
    st2 = ctx.time_step()
    assert st2.status == 0
    assert st2.start_used in (pnp.PNP_START_LEARNED, pnp.PNP_START_EXTRAPOLATE)
    assert st2.res0 <= st2.res_start_extrapolated * (1 + 1e-12)


def _adam_oracle(p0, grads, lr, b1, b2, eps):
    """The oracle's Adam applied to the packed parameters (one tensor) for each gradient."""
    P = [p0.astype(np.float64).copy()]
    state = {}
    out = []
    for g in grads:
        MO.adam_step(P, [], [g.astype(np.float64)], [], state, lr=lr, beta1=b1, beta2=b2, eps=eps)
        out.append((P[0].copy(), state["m"][0].copy(), state["v"][0].copy(), state["t"]))
    return out


def test_adam_update_matches_oracle_over_several_steps():
    """The library's Adam update (the one pnp_mlp_train applies after every batch) against
    the oracle's Adam for four consecutive steps fed the same gradients: parameters, both
    moments and the step count.  The gradients mix magnitudes over six decades and change
    sign between steps, so the bias correction, the betas and the moments carried from one
    step to the next all show.  FP32 arithmetic against FP64: moments within 1e-6 of their
    norm, parameters within FP32 rounding of the parameter plus 1e-5 of the step size."""
    oc = W.uniform_octants(3, 2)
    pnp, torch, mesh, ctx = _ctx(oc)
    rng = np.random.default_rng(21)
    P = pnp.PNP_MLP_PARAMS
    p0 = rng.normal(0, 0.1, P).astype(np.float32)
    ctx.mlp_set_weights(p0)
    lr, b1, b2, eps = 3e-3, 0.85, 0.995, 1e-7
    mags = 10.0 ** rng.uniform(-6, 0, P)
    grads = [(rng.choice([-1.0, 1.0], P) * mags * rng.uniform(0.5, 2.0, P)).astype(np.float32) for _ in range(4)]
    grads[2] = (-grads[1] * 0.5).astype(np.float32)  # a sign reversal
    ref = _adam_oracle(p0, grads, lr, b1, b2, eps)
    m0, v0, t0 = ctx.mlp_adam_state()
    assert t0 == 0 and not m0.any() and not v0.any()
    for t, g in enumerate(grads, start=1):
        ctx.mlp_adam_step(torch.from_numpy(g).cuda(), lr=lr, beta1=b1, beta2=b2, adam_eps=eps)
        p = ctx.mlp_get_weights().astype(np.float64)
        m, v, tt = ctx.mlp_adam_state()
        pr, mr, vr, tr = ref[t - 1]
        assert tt == tr == t
        assert np.linalg.norm(m - mr) <= 1e-6 * np.linalg.norm(mr), t
        assert np.linalg.norm(v - vr) <= 1e-6 * np.linalg.norm(vr), t
        assert np.abs(m - mr).max() <= 1e-6 * np.abs(mr).max(), t
        tol = 2.0**-23 * np.abs(pr) * t + 1e-5 * lr * t
        assert np.all(np.abs(p - pr) <= tol), (t, np.abs(p - pr).max())
        # each step moved the parameters by about lr at most (a bias correction that
        # shrinks towards zero with t would break this on the first steps)
        step = np.abs(p - (ref[t - 2][0] if t > 1 else p0))
        assert step.max() <= lr * (1.0 + 1e-3) / (1 - b1) + 1e-9


def test_training_steps_match_oracle_gradients_and_moments():
    """Three training steps on a fixed batch through the library's own gradient and Adam
    calls, against the oracle's FP64 backward pass on the same BF16-rounded weights and
    inputs and its Adam: the gradient and both Adam moments within the gradient test's
    2e-2 per tensor (the second moment, quadratic in the gradient, within 4e-2), and the
    loss within 1e-2 at every step."""
    oc = W.uniform_octants(3, 2)
    pnp, torch, mesh, ctx = _ctx(oc)
    rng = np.random.default_rng(8)
    Ws, bs = MO.init_params(5)
    bs = [b + rng.normal(0, 0.05, b.shape) for b in bs]
    p = pack(Ws, bs)
    ctx.mlp_set_weights(p)
    B = 1024
    X = rng.normal(size=(B, 216)).astype(np.float32)
    Y = rng.normal(size=(B, 3)).astype(np.float32)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    g = torch.zeros(pnp.PNP_MLP_PARAMS, dtype=torch.float32, device="cuda")
    lr = 1e-3
    P = [p.astype(np.float64)]
    state = {}
    Xr = MO.bf16_round(X)
    for t in range(1, 4):
        loss = ctx.mlp_loss_grad(Xd, Yd, g)
        ctx.mlp_adam_step(g, lr=lr)
        # the oracle: gradient at the library's current FP32 master weights rounded to BF16
        Wr, br = unpack(P[0].astype(np.float32))
        gW, gb, lref = MO.backward([MO.bf16_round(w) for w in Wr], br, Xr, Y.astype(np.float64))
        gref = pack(gW, gb).astype(np.float64)
        MO.adam_step(P, [], [gref], [], state, lr=lr)
        gg = g.cpu().numpy().astype(np.float64)
        m, v, tt = ctx.mlp_adam_state()
        assert tt == t
        assert abs(loss - lref) <= 1e-2 * lref, t
        for (off, fi, fo) in SHAPES:
            for a, b_, tol in [(gg, gref, 2e-2), (m, state["m"][0], 2e-2), (v, state["v"][0], 4e-2)]:
                sl = slice(off, off + fi * fo)
                assert np.linalg.norm(a[sl] - b_[sl]) <= tol * np.linalg.norm(b_[sl]), (t, off)
        # keep the oracle's master weights on the library's (their difference is the
        # gradient's BF16 error; the next step compares the update it makes from there)
        P[0] = ctx.mlp_get_weights().astype(np.float64)
