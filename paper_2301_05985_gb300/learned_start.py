"""Training data, training and evaluation of the learned Newton start (C-ABI driven).

The experiment: the 3D transient double-layer problem (unit cube, uniform level 5,
32,768 elements, 35,937 nodes, Lambda = 0.01, dt = 1e-3; phi = V on z = 0 and 0 on
z = 1, c+- = 1 on z = 1, zero flux elsewhere; c+- = 1 + seeded noise 1e-3, phi
linear at t = 0, double layer developed by a BDF1 step-size ramp).  Trajectories are
recorded with the FP32-J V inexact Newton solver at V = 10, 20, 30 (a step whose Newton
solve fails is split into half steps), the network is trained on them, and the time
steps at V = 25 (not seen in training) are then solved with the previous-step,
extrapolated and learned (judged) starts.
"""
from __future__ import annotations

import time

import numpy as np


def setup(pnp, W, torch, V, level=5, eps=0.01, dt=1e-3, seed=0, mode="plain"):
    oc = W.uniform_octants(3, level)
    mesh = pnp.Mesh(oc)
    prec = pnp.PNP_F64 if mode == "plain" else pnp.PNP_F32
    prm = pnp.default_params(eps=eps, dt=dt, newton_rtol=1e-8, gmres_rtol=1e-8, gmres_restart=60,
                             gmres_max_it=4000, precision=prec, start_mode=pnp.PNP_START_EXTRAPOLATE,
                             dt_retries=3)
    ctx = pnp.Context(mesh, prm, torch.cuda.current_stream().cuda_stream)
    ctx.set_bcs(W.equilibrium_bcs(3, V))
    U0 = W.noisy_state(mesh.ijk, oc.max_level, seed=seed, amp=1e-3, phi_bottom=V, phi_top=0.0)
    ctx.set_field(pnp.PNP_FIELD_U, U0)
    ctx.make_consistent()
    ctx.reset_history()
    develop_double_layer(pnp, ctx, dt)
    return mesh, ctx


def develop_double_layer(pnp, ctx, dt, dt0=1e-6, factor=4.0):
    """Start from a developed double layer (as the paper does for its electroconvection
    runs): BDF1 steps with the step size growing geometrically from dt0 to dt, then the
    history is reset so the recorded trajectory starts there with the target dt."""
    p = ctx.get_params()
    ramp = pnp.default_params(**{k: getattr(p, k) for k, _ in p._fields_})
    ramp.bdf_order, ramp.newton_max_it, ramp.start_mode = 1, 100, pnp.PNP_START_PREVIOUS
    h = dt0
    while h < dt:
        ramp.dt = h
        ctx.set_params(ramp)
        ctx.time_step()
        ctx.reset_history()
        h *= factor
    ctx.set_params(p)
    ctx.reset_history()


def record(pnp, torch, ctx, n_steps, coupled=False):
    """Time-step the context and return (states, Newton iterations, u_z): the device tensor
    [k+1, N, 3] of states at the full steps, k <= n_steps (recording stops at a step that
    fails even after splitting), and with coupled NS-PNP steps the last velocity component
    [k+1, N] at the same steps (None for PNP steps: the fluid is at rest)."""
    N = ctx.n_nodes
    S = torch.zeros((n_steps + 1, N, 3), dtype=torch.float64, device="cuda")
    UZ = torch.zeros((n_steps + 1, N), dtype=torch.float64, device="cuda") if coupled else None
    vel = torch.zeros((N, 3), dtype=torch.float64, device="cuda") if coupled else None
    ctx.get_field(pnp.PNP_FIELD_U, S[0], pnp.PNP_DEVICE)
    if coupled:
        ctx.get_field(pnp.PNP_FIELD_VELOCITY, vel, pnp.PNP_DEVICE)
        UZ[0] = vel[:, 2]
    its = []
    for k in range(n_steps):
        if coupled:
            st, _ = ctx.coupled_step(raise_on_error=False)
        else:
            st = ctx.time_step(raise_on_error=False)
        if st.status != pnp.PNP_OK:
            return S[:k + 1], its, (UZ[:k + 1] if coupled else None)
        its.append(st.newton_its)
        ctx.get_field(pnp.PNP_FIELD_U, S[k + 1], pnp.PNP_DEVICE)
        if coupled:
            ctx.get_field(pnp.PNP_FIELD_VELOCITY, vel, pnp.PNP_DEVICE)
            UZ[k + 1] = vel[:, 2]
    return S, its, UZ


def run(pnp, W, torch, train_V=(10.0, 20.0, 30.0), steps_per_V=667, test_V=25.0, test_steps=50, seeds=(0, 1, 2),
        train_steps=3000, batch=4096, lr=1e-3, level=5, mode="mixed", log=print):
    """Returns a dict of the experiment's numbers (training loss, per-start statistics)."""
    out = {"train_V": list(train_V), "steps_per_V": steps_per_V, "test_V": test_V, "test_steps": test_steps}
    mesh, ctx = setup(pnp, W, torch, train_V[0], level=level, mode=mode)
    ctx.mlp_init(seed=0)
    t0 = time.perf_counter()
    for V in train_V:
        m2, c2 = setup(pnp, W, torch, V, level=level, mode=mode)
        S, its, _ = record(pnp, torch, c2, steps_per_V)
        ctx.mlp_add_trajectory(S)
        log(f"trajectory V={V}: {len(its)} of {steps_per_V} steps, mean Newton its {np.mean(its):.2f}")
        del S
        c2.close()
    out["record_s"] = time.perf_counter() - t0
    st = ctx.mlp_train(steps=train_steps, batch=batch, lr=lr, seed=1)
    out["train"] = st.as_dict()
    log(f"training: loss {st.loss_first:.4f} -> {st.loss_last:.4f} in {st.wall_ms / 1e3:.2f} s")
    weights = ctx.mlp_get_weights()
    norm = ctx.mlp_get_normalization()
    results = {}
    for name, start in (("previous", pnp.PNP_START_PREVIOUS), ("extrapolated", pnp.PNP_START_EXTRAPOLATE),
                       ("learned", pnp.PNP_START_LEARNED)):
        its, kry, wall, used_learned, r0, splits, ratio = [], [], [], 0, [], 0, []
        for seed in seeds:
            m3, c3 = setup(pnp, W, torch, test_V, level=level, seed=100 + seed, mode=mode)
            if start == pnp.PNP_START_LEARNED:
                c3.mlp_init(seed=0)
                c3.mlp_set_weights(weights)
                c3.mlp_set_normalization(*norm)
            p = c3.get_params(); p.start_mode = start
            c3.set_params(p)
            for k in range(test_steps):
                torch.cuda.synchronize()
                t = time.perf_counter()
                s = c3.time_step()
                torch.cuda.synchronize()
                wall.append(time.perf_counter() - t)
                if k == 0:
                    continue  # first step: no history, all starts coincide
                its.append(s.newton_its)
                kry.append(s.krylov_its)
                r0.append(s.res0)
                used_learned += int(s.start_used == pnp.PNP_START_LEARNED)
                splits += int(s.substeps > 1)
                if s.res_start_extrapolated > 0:
                    ratio.append(s.res_start_learned / s.res_start_extrapolated)
            c3.close()
        results[name] = {"newton_its_mean": float(np.mean(its)), "krylov_its_mean": float(np.mean(kry)),
                         "ms_per_step": 1e3 * float(np.mean(wall)), "res0_mean": float(np.mean(r0)),
                         "learned_used": used_learned, "split_steps": splits, "steps": len(its),
                         "network_over_extrapolated": float(np.mean(ratio)) if ratio else None}
        log(f"{name:12s}: Newton {np.mean(its):.3f}  Krylov {np.mean(kry):.1f}  {1e3 * np.mean(wall):.2f} ms/step "
            f" ||F0|| {np.mean(r0):.3e}  learned used {used_learned}/{len(its)}  split {splits}"
            + (f"  ||F(net)||/||F(extrap)|| {np.mean(ratio):.3f}" if ratio else ""))
    out["results"] = results
    ctx.close()
    return out, weights, norm
