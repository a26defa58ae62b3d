"""GPU parity on meshes with periodic side walls (the electroconvection setup of Sec. 5.2):
residual, J V (FP64, FP32 and through the stored linearisation) and the block diagonal
against the FP64 oracle, whose mesh build identifies the faces independently, and a
time step against the oracle's Newton step.  Tolerances as in the non-periodic tests."""
import numpy as np
import pytest

import oracle as O
from paper_2301_05985_gb300 import workloads as W

from gpu_common import Pair, field_max_err, rel_err

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5


def _cases():
    return [
        ("3d_octree_periodic_x", W.random_balanced_octants(3, 2, 4, 0.3, 12, periodic=1),
         dict(eps=0.02, dt=0.01, beta0=1.5, beta1=-2.0, beta2=0.5), W.membrane_bcs(3, 5.0, 2.0), False),
        ("3d_band_periodic_xy", W.with_periodic(W.membrane_band_octants(3, 5, 0.1), 3),
         dict(eps=0.01, dt=1e-3, beta0=1.5, beta1=-2.0, beta2=0.5), W.membrane_bcs(3, 20.0, 2.0), True),
        ("2d_octree_periodic_x", W.random_balanced_octants(2, 2, 5, 0.3, 12, periodic=1),
         dict(eps=0.02, dt=0.01, beta0=1.0, beta1=-1.0, beta2=0.0), W.membrane_bcs(2, 5.0, 2.0), False),
    ]


CASES = _cases()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_periodic_operators_match_oracle(case):
    _, oc, kw, bcs, fourier = case
    P = Pair(oc, kw, bcs)
    ijk, L = P.mesh.ijk, oc.max_level
    vel = W.fourier_velocity(ijk, L, 3, rms=0.2) if fourier else W.random_velocity(ijk, L, 3, 0.5)
    P.set_state(Uk=W.random_state(ijk, L, 1), Ukm1=W.random_state(ijk, L, 2), vel=vel[:, :oc.dim])
    U = W.random_state(ijk, L, 4)
    V = W.random_direction(ijk, L, 5)
    F, Fo = P.gpu_residual(U), P.oracle_residual(U)
    assert rel_err(F, Fo) <= TOL64 and np.all(field_max_err(F, Fo) <= TOL64)
    ref = P.oracle_jv(U, V)
    JV = P.gpu_jv(U, V, 0)
    assert rel_err(JV, ref) <= TOL64 and np.all(field_max_err(JV, ref) <= TOL64)
    assert np.all(field_max_err(P.gpu_jv(U, V, 1), ref) <= TOL32)
    P.ctx.linearize(P.dev(U))
    Vd = P.dev(V.astype(np.float32))
    JVl = P.torch.zeros_like(Vd)
    P.ctx.jv_linearized(Vd, JVl)
    assert np.all(field_max_err(JVl.cpu().numpy().astype(np.float64), ref) <= TOL32)
    # block diagonal (FP64 and FP32) against the oracle Jacobian's diagonal blocks
    J = P.oracle_jacobian(U).tocsr()
    n = P.mesh.n_nodes
    blk = np.zeros((n, 3, 3))
    for f in range(3):
        for g in range(3):
            blk[:, f, g] = np.asarray(J[3 * np.arange(n) + f, 3 * np.arange(n) + g]).reshape(-1)
    D = P.torch.zeros((n, 9), dtype=P.torch.float64, device="cuda")
    P.ctx.block_diag(P.dev(U), D)
    assert np.abs(D.cpu().numpy().reshape(n, 3, 3) - blk).max() <= TOL64 * np.abs(blk).max()
    D32 = P.torch.zeros((n, 9), dtype=P.torch.float32, device="cuda")
    P.ctx.block_diag(P.dev(U), D32)
    ent = np.abs(blk).max(axis=0)
    ent[ent == 0] = 1.0
    assert np.all(np.abs(D32.cpu().numpy().astype(np.float64).reshape(n, 3, 3) - blk).max(axis=0) <= TOL32 * ent)


@pytest.mark.parametrize("precision", [0, 1])
def test_periodic_time_step_matches_oracle_newton(precision):
    """One BDF1 step on a 2D octree periodic in x (membrane at y = 0, reservoir at y = 1),
    plain FP64 and mixed FP32-J V mode, against the oracle's Newton step."""
    oc = W.random_balanced_octants(2, 2, 5, 0.3, 12, periodic=1)
    V, eps, dt = 5.0, 0.02, 5e-3
    bcs = W.membrane_bcs(2, V, 2.0)
    kw = dict(eps=eps, dt=dt, newton_rtol=1e-11, gmres_rtol=1e-12, gmres_restart=60, gmres_max_it=20000,
              start_mode=0, precision=precision, newton_max_it=40)
    if precision:
        kw.update(gmres_inner=8, newton_rtol=1e-11)
    P = Pair(oc, kw, bcs)
    U0 = W.noisy_state(P.mesh.ijk, oc.max_level, seed=3, amp=1e-2, phi_bottom=0.0, phi_top=V)
    P.ctx.set_field(P.pnp.PNP_FIELD_U, U0)
    P.ctx.make_consistent()
    P.ctx.reset_history()
    U0o = P.to_ora(P.ctx.get_field(P.pnp.PNP_FIELD_U))
    op = O.Params(eps=eps, dt=dt, beta=(1.0, -1.0, 0.0), bc_type=bcs.types, bc_val=bcs.values)
    r = O.newton(P.om, op, U0o, U0o, U0o, np.zeros((P.mesh.n_nodes, 2)), rtol=1e-12, max_it=40)
    assert r.converged
    st = P.ctx.time_step()
    assert st.status == 0
    # mixed mode: inexact Newton with FP32 J V to the same residual tolerance
    assert rel_err(P.to_ora(P.ctx.get_field(P.pnp.PNP_FIELD_U)), r.U) <= (1e-9 if precision == 0 else 1e-7)
