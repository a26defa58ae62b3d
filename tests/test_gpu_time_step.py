"""GPU time stepping beyond constant-step BDF: a failed step split into half steps.

The case: 2D, uniform level 5, Lambda = 0.01, V = 10, dt = 1e-2, from a noisy neutral
state with linear phi.  The oracle's exact Newton needs 12 iterations for the full BDF1
step and 9 and 5 for the two half steps, so a Newton limit of 9 makes the full step
fail and both halves succeed.
"""
import numpy as np
import pytest

import oracle as O
from paper_2301_05985_gb300 import workloads as W

from gpu_common import Pair, rel_err

pytestmark = pytest.mark.gpu


def test_failed_step_is_split_into_half_steps_matching_oracle():
    oc = W.uniform_octants(2, 5)
    V, eps, dt = 10.0, 0.01, 1e-2
    bcs = W.equilibrium_bcs(2, V)
    kw = dict(eps=eps, dt=dt, newton_rtol=1e-11, gmres_rtol=1e-12, gmres_restart=60, gmres_max_it=20000,
              start_mode=1, newton_max_it=60, dt_retries=1)
    P = Pair(oc, kw, bcs)
    L = oc.max_level
    U0 = W.noisy_state(P.mesh.ijk, L, seed=3, amp=1e-3, phi_bottom=V, phi_top=0.0)
    P.ctx.set_field(P.pnp.PNP_FIELD_U, U0)
    P.ctx.make_consistent()
    P.ctx.reset_history()
    U0o = P.to_ora(P.ctx.get_field(P.pnp.PNP_FIELD_U))
    vel = np.zeros((P.mesh.n_nodes, 2))

    def oracle_step(Uk, Ukm1, h, beta):
        op = O.Params(eps=eps, dt=h, beta=beta, bc_type=bcs.types, bc_val=bcs.values)
        r = O.newton(P.om, op, Uk, Uk, Ukm1, vel, rtol=1e-12, max_it=60)
        assert r.converged
        return r

    full = oracle_step(U0o, U0o, dt, (1.0, -1.0, 0.0))
    h1 = oracle_step(U0o, U0o, dt / 2, (1.0, -1.0, 0.0))
    h2 = oracle_step(h1.U, h1.U, dt / 2, (1.0, -1.0, 0.0))
    limit = max(h1.iterations, h2.iterations)
    assert full.iterations >= limit + 2  # the case really needs the split

    p = P.ctx.get_params()
    p.newton_max_it = limit
    P.ctx.set_params(p)
    st = P.ctx.time_step()
    assert st.status == 0 and st.substeps == 2
    assert rel_err(P.to_ora(P.ctx.get_field(P.pnp.PNP_FIELD_U)), h2.U) <= 1e-9
    p.newton_max_it = 60
    P.ctx.set_params(p)
    # after a split U^{k-1} is half a step behind: the next step is BDF1
    st = P.ctx.time_step()
    assert st.status == 0 and st.substeps == 1 and st.start_used == P.pnp.PNP_START_PREVIOUS
    s2 = oracle_step(h2.U, h2.U, dt, (1.0, -1.0, 0.0))
    assert rel_err(P.to_ora(P.ctx.get_field(P.pnp.PNP_FIELD_U)), s2.U) <= 1e-9
    # ... and the one after it BDF2 with full-step history again: extrapolated start, or
    # the previous state when the extrapolation's residual is the larger (the safeguard)
    st = P.ctx.time_step()
    assert st.status == 0 and st.substeps == 1
    assert st.start_used in (P.pnp.PNP_START_EXTRAPOLATE, P.pnp.PNP_START_PREVIOUS)
    if st.start_used == P.pnp.PNP_START_PREVIOUS:
        assert st.res0 == st.res_ref
    s3 = oracle_step(s2.U, h2.U, dt, (1.5, -2.0, 0.5))
    assert rel_err(P.to_ora(P.ctx.get_field(P.pnp.PNP_FIELD_U)), s3.U) <= 1e-9
    assert P.ctx.step_count() == 3


def test_failed_step_without_retries_reports_newton_failure():
    oc = W.uniform_octants(2, 5)
    V, eps, dt = 10.0, 0.01, 1e-2
    bcs = W.equilibrium_bcs(2, V)
    kw = dict(eps=eps, dt=dt, newton_rtol=1e-11, gmres_rtol=1e-12, gmres_restart=60, gmres_max_it=20000,
              newton_max_it=3, dt_retries=0)
    P = Pair(oc, kw, bcs)
    U0 = W.noisy_state(P.mesh.ijk, oc.max_level, seed=3, amp=1e-3, phi_bottom=V, phi_top=0.0)
    P.ctx.set_field(P.pnp.PNP_FIELD_U, U0)
    P.ctx.make_consistent()
    P.ctx.reset_history()
    st = P.ctx.time_step(raise_on_error=False)
    assert st.status == P.pnp.PNP_ERR_NEWTON_DIVERGED and st.newton_its == 3
    assert P.ctx.step_count() == 0


def _small_pair(**extra):
    oc = W.uniform_octants(2, 4)
    bcs = W.equilibrium_bcs(2, 1.0)
    kw = dict(eps=0.05, dt=1e-2, newton_rtol=1e-10, gmres_rtol=1e-10, gmres_restart=30, gmres_max_it=2000)
    kw.update(extra)
    P = Pair(oc, kw, bcs)
    U0 = W.noisy_state(P.mesh.ijk, oc.max_level, seed=1, amp=1e-2, phi_bottom=1.0, phi_top=0.0)
    P.ctx.set_field(P.pnp.PNP_FIELD_U, U0)
    P.ctx.make_consistent()
    P.ctx.reset_history()
    return P, U0


def test_non_finite_state_is_reported_and_the_context_stays_usable():
    """Failure detection on the host side of a solve: a NaN in the state makes the
    Newton solve return PNP_ERR_NAN (no device fault, no abort); a valid state then
    solves normally on the same context."""
    P, U0 = _small_pair()
    bad = U0.copy()
    bad[5, 0] = np.nan
    P.ctx.set_field(P.pnp.PNP_FIELD_U, bad)
    st = P.ctx.newton_solve(raise_on_error=False)
    assert st.status == P.pnp.PNP_ERR_NAN
    P.ctx.set_field(P.pnp.PNP_FIELD_U, U0)
    P.ctx.make_consistent()
    P.ctx.reset_history()
    st = P.ctx.time_step(raise_on_error=False)
    assert st.status == 0 and st.res_final <= 1e-10 * st.res_ref


def test_krylov_iteration_limit_is_reported():
    """A GMRES limit of 3 iterations at rtol 1e-12 returns PNP_ERR_KRYLOV_MAXIT with the
    iterations taken; the context stays usable."""
    P, U0 = _small_pair(gmres_max_it=3)
    torch = P.torch
    n = P.mesh.n_nodes
    U = torch.from_numpy(P.ctx.get_field(P.pnp.PNP_FIELD_U)).cuda()
    F = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    P.ctx.residual(U, F)
    x = torch.zeros_like(F)
    st = P.ctx.gmres(U, -F, x, 1e-12, raise_on_error=False)
    assert st.status == P.pnp.PNP_ERR_KRYLOV_MAXIT and st.krylov_its == 3
    p = P.ctx.get_params(); p.gmres_max_it = 2000; P.ctx.set_params(p)
    x.zero_()
    st = P.ctx.gmres(U, -F, x, 1e-10)
    assert st.status == 0


def test_staged_jv_wait_that_gives_up_is_reported_and_recovers():
    """The stored-linearisation J V streams its state through shared memory and waits for
    the bulk copies with a bounded poll loop.  A poll limit of 0 makes every wait give up
    at once while the copies still land (the block drains them before it exits): the call
    reports PNP_ERR_DEVICE_FLAG, the flag stays until the next linearisation, and after it
    the context computes the same J V as before."""
    oc = W.random_balanced_octants(3, 1, 4, 0.3, 12)
    P = Pair(oc, dict(eps=0.05, dt=1e-2, beta0=1.5, beta1=-2.0, beta2=0.5), W.membrane_bcs(3, 5.0, 2.0))
    ijk, L = P.mesh.ijk, oc.max_level
    P.set_state(Uk=W.random_state(ijk, L, 1), Ukm1=W.random_state(ijk, L, 2))
    U = P.dev(W.random_state(ijk, L, 3))
    V = P.dev(W.random_direction(ijk, L, 4).astype(np.float32))
    ref = P.torch.zeros_like(V)
    P.ctx.linearize(U)
    P.ctx.jv_linearized(V, ref)
    JV = P.torch.zeros_like(V)
    P.ctx.set_wait_limit(0)
    with pytest.raises(P.pnp.PnpError) as e:
        P.ctx.jv_linearized(V, JV)
    assert e.value.code == P.pnp.PNP_ERR_DEVICE_FLAG
    P.ctx.set_wait_limit(-1)
    with pytest.raises(P.pnp.PnpError) as e:  # latched until the next linearisation
        P.ctx.jv_linearized(V, JV)
    assert e.value.code == P.pnp.PNP_ERR_DEVICE_FLAG
    P.ctx.linearize(U)
    P.ctx.jv_linearized(V, JV)
    a, b = JV.cpu().numpy(), ref.cpu().numpy()
    assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max()
