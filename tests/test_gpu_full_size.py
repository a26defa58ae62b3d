"""GPU parity at the full sizes of the benchmark workloads, through the same launches the
bench times: every row of the FP64 residual, the FP64 J V, the FP32 J V and the FP32 J V
through the stored linearisation (the kernels of the inner Krylov solve) is compared with
the FP64 oracle.

Workloads:
- the 3D membrane-band octree: base level 5, level 8 for z_min < 0.05 (971,776 elements,
  1,047,407 nodes, 64,960 hanging); Lambda = 1e-3, dt = 1e-3, V = 20; membrane boundary
  table; zero velocity, as in the bench;
- the uniform level-7 cube (2,097,152 elements, 2,146,689 nodes); Lambda = 1e-3,
  dt = 1e-3, V = 30; divergence-free Fourier velocity of RMS 0.1.

The oracle needs about 15 s (membrane band) and 30 s (level 7) of host time per case.
Tolerances are the small cases': 1e-12 relative for FP64 (whole vector and per field),
2e-5 of each field's maximum for FP32.
"""
import numpy as np
import pytest

from paper_2301_05985_gb300 import workloads as W

from gpu_common import Pair, field_max_err, rel_err

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5


def _case(name):
    if name == "membrane_band_L5_8":
        oc = W.membrane_band_octants(5, 8, 0.05)
        bcs = W.membrane_bcs(3, 20.0, 2.0)
        vel = None
    else:
        oc = W.uniform_octants(3, 7)
        bcs = W.membrane_bcs(3, 30.0, 2.0)
        vel = "fourier"
    kw = dict(eps=1e-3, dt=1e-3, beta0=1.5, beta1=-2.0, beta2=0.5)
    P = Pair(oc, kw, bcs)
    ijk, L = P.mesh.ijk, oc.max_level
    v = W.fourier_velocity(ijk, L, 7, rms=0.1) if vel else None
    P.set_state(Uk=W.random_state(ijk, L, 31), Ukm1=W.random_state(ijk, L, 32), vel=v)
    U = W.random_state(ijk, L, 33)
    V = W.random_direction(ijk, L, 34)
    return P, U, V


@pytest.mark.parametrize("name", ["membrane_band_L5_8", "uniform_L7_fourier"])
def test_full_size_operators_match_oracle(name):
    P, U, V = _case(name)
    torch = P.torch
    # FP64 residual
    F = P.gpu_residual(U)
    Fo = P.oracle_residual(U)
    assert rel_err(F, Fo) <= TOL64
    assert np.all(field_max_err(F, Fo) <= TOL64)
    # FP64 and FP32 J V
    ref = P.oracle_jv(U, V)
    JV64 = P.gpu_jv(U, V, 0)
    assert rel_err(JV64, ref) <= TOL64
    assert np.all(field_max_err(JV64, ref) <= TOL64)
    JV32 = P.gpu_jv(U, V, 1)
    assert np.all(field_max_err(JV32, ref) <= TOL32), field_max_err(JV32, ref)
    # FP32 J V through the stored linearisation, two directions at one state
    P.ctx.linearize(P.dev(U))
    for d in (V, W.random_direction(P.mesh.ijk, P.oc.max_level, 35)):
        Vd = P.dev(d.astype(np.float32))
        JVl = torch.zeros_like(Vd)
        P.ctx.jv_linearized(Vd, JVl)
        JVl = JVl.cpu().numpy().astype(np.float64)
        ref_d = ref if d is V else P.oracle_jv(U, d)
        assert np.all(field_max_err(JVl, ref_d) <= TOL32), field_max_err(JVl, ref_d)


def test_linearized_jv_needs_a_current_linearisation():
    """A solver call replaces the stored linearisation: pnp_jv_linearized then refuses
    (PNP_ERR_STATE) until pnp_linearize is called again."""
    oc = W.uniform_octants(3, 3)
    bcs = W.membrane_bcs(3, 5.0, 2.0)
    P = Pair(oc, dict(eps=0.05, dt=1e-2, gmres_inner=4, precision=1, gmres_restart=20, gmres_max_it=200), bcs)
    ijk, L = P.mesh.ijk, oc.max_level
    P.set_state(Uk=W.random_state(ijk, L, 1), Ukm1=W.random_state(ijk, L, 1))
    U = P.dev(W.random_state(ijk, L, 2))
    V = P.dev(W.random_direction(ijk, L, 3).astype(np.float32))
    JV = P.torch.zeros_like(V)
    with pytest.raises(P.pnp.PnpError):
        P.ctx.jv_linearized(V, JV)
    P.ctx.linearize(U)
    P.ctx.jv_linearized(V, JV)
    b = P.torch.zeros_like(U)
    P.ctx.residual(U, b)
    x = P.torch.zeros_like(U)
    P.ctx.gmres(U, -b, x, 1e-3, P.pnp.PNP_F32, raise_on_error=False)
    with pytest.raises(P.pnp.PnpError):
        P.ctx.jv_linearized(V, JV)
