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


def test_full_size_ns_rows_match_oracle():
    """The Navier-Stokes rows at the membrane-band octree's full size (no-slip walls, the
    bench's Sc = 1 and kappa = 0.5, a random (v, p), velocity history and PNP state): the
    double-float residual and matrix action at 1e-12, the FP32 matrix action at 5e-5 per
    slot, every row against the oracle."""
    import oracle as O
    oc = W.membrane_band_octants(5, 8, 0.05)
    kw = dict(eps=1e-3, dt=1e-3, beta0=1.5, beta1=-2.0, beta2=0.5, ns_Sc=1.0, ns_kappa=0.5)
    P = Pair(oc, kw, W.membrane_bcs(3, 20.0, 2.0))
    ijk, L, n = P.mesh.ijk, oc.max_level, P.mesh.n_nodes
    bt, bv = O.no_slip_bcs(3)
    P.ctx.ns_set_bcs(bt, bv)
    vk, vkm1 = W.fourier_velocity(ijk, L, 41, rms=0.5), W.fourier_velocity(ijk, L, 42, rms=0.5)
    U = W.random_state(ijk, L, 43)
    P.ctx.set_field(P.pnp.PNP_FIELD_VELOCITY, vk)
    P.ctx.set_field(P.pnp.PNP_FIELD_VELOCITY_PREV, vkm1)
    P.ctx.set_field(P.pnp.PNP_FIELD_U, U)
    X = np.random.default_rng(44).standard_normal((n, 4))
    nsp = O.NsParams(Sc=1.0, kappa=0.5, eps=1e-3, dt=1e-3, beta=(1.5, -2.0, 0.5), bc_type=bt, bc_val=bv)
    o = P.to_ora
    args = (o(X), o(2.0 * vk - vkm1), o(vk), o(vkm1), o(U))
    torch = P.torch
    Xd = torch.from_numpy(X).cuda()
    F = torch.zeros_like(Xd)
    P.ctx.ns_residual(Xd, F)
    Fo = P.to_lib(P.om.ns_apply(nsp, *args, with_data=True))
    assert np.linalg.norm(F.cpu().numpy() - Fo) / np.linalg.norm(Fo) <= TOL64
    Y = torch.zeros_like(Xd)
    P.ctx.ns_matvec(Xd, Y, P.pnp.PNP_F64)
    Ao = P.to_lib(P.om.ns_apply(nsp, *args, with_data=False))
    Yh = Y.cpu().numpy()
    assert np.linalg.norm(Yh - Ao) / np.linalg.norm(Ao) <= TOL64
    for f in range(4):
        assert np.abs(Yh[:, f] - Ao[:, f]).max() <= 10 * TOL64 * np.abs(Ao[:, f]).max()
    X32 = Xd.float()
    Y32 = torch.zeros_like(X32)
    P.ctx.ns_matvec(X32, Y32, P.pnp.PNP_F32)
    Y32h = Y32.cpu().numpy().astype(np.float64)
    for f in range(4):
        assert np.abs(Y32h[:, f] - Ao[:, f]).max() <= 5e-5 * np.abs(Ao[:, f]).max()
