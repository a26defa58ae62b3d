"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances: FP64 residual / Jv / block diagonal within 1e-12 relative (2-norm of the
whole vector, and per field in max norm relative to the field's max), the bar of the
FP64 path.  FP32 Jv per field within 2e-5 relative to the field's max norm: the FP32
element arithmetic (unit roundoff 6e-8) over sums with cancellation of up to a few
hundred terms per row.
"""
import numpy as np
import pytest

import oracle as O
from paper_2301_05985_gb300 import workloads as W

from gpu_common import Pair, field_max_err, problem_cases, rel_err

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5
CASES = problem_cases()


def _setup(case, seed=0):
    name, oc, kw, bcs = case
    P = Pair(oc, kw, bcs)
    ijk = P.mesh.ijk
    L = oc.max_level
    P.set_state(Uk=W.random_state(ijk, L, seed + 1), Ukm1=W.random_state(ijk, L, seed + 2),
                vel=W.random_velocity(ijk, L, seed + 3, amp=2.0))
    U = W.random_state(ijk, L, seed + 4)
    V = W.random_direction(ijk, L, seed + 5)
    return P, U, V


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_residual_f64_matches_oracle(case):
    P, U, _ = _setup(case)
    F = P.gpu_residual(U)
    Fo = P.oracle_residual(U)
    assert rel_err(F, Fo) <= TOL64
    assert np.all(field_max_err(F, Fo) <= TOL64)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_jv_f64_matches_oracle(case):
    P, U, V = _setup(case)
    JV = P.gpu_jv(U, V, 0)
    ref = P.oracle_jv(U, V)
    J = P.oracle_jacobian(U)
    ref2 = (J @ V.reshape(-1)).reshape(-1, 3)
    assert rel_err(ref, ref2) <= 1e-13
    assert rel_err(JV, ref) <= TOL64
    assert np.all(field_max_err(JV, ref) <= TOL64)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_jv_f32_matches_oracle_per_field(case):
    P, U, V = _setup(case)
    JV = P.gpu_jv(U, V, 1)
    ref = P.oracle_jv(U, V)
    err = field_max_err(JV, ref)
    assert np.all(err <= TOL32), err


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_block_diagonal_matches_oracle_jacobian(case):
    P, U, _ = _setup(case)
    J = P.oracle_jacobian(U).tocsr()
    n = P.mesh.n_nodes
    ref = np.zeros((n, 3, 3))
    for f in range(3):
        for g in range(3):
            rows = 3 * np.arange(n) + f
            cols = 3 * np.arange(n) + g
            ref[:, f, g] = np.asarray(J[rows, cols]).reshape(-1)
    D = P.torch.zeros((n, 9), dtype=P.torch.float64, device="cuda")
    P.ctx.block_diag(P.dev(U), D)
    D = D.cpu().numpy().reshape(n, 3, 3)
    scale = np.abs(ref).max()
    assert np.abs(D - ref).max() <= TOL64 * scale
    # FP32 arithmetic (the mixed-precision preconditioner's blocks), entry by entry
    # against each entry's own scale over the mesh
    D32 = P.torch.zeros((n, 9), dtype=P.torch.float32, device="cuda")
    P.ctx.block_diag(P.dev(U), D32)
    D32 = D32.cpu().numpy().astype(np.float64).reshape(n, 3, 3)
    ent = np.abs(ref).max(axis=0)
    ent[ent == 0] = 1.0
    assert np.all(np.abs(D32 - ref).max(axis=0) <= TOL32 * ent), np.abs(D32 - ref).max(axis=0) / ent


def test_jv_is_exact_derivative_of_gpu_residual():
    """Richardson-combined central differences of the GPU residual (exact for a cubic)."""
    P, U, V = _setup(CASES[3], seed=7)
    JV = P.gpu_jv(U, V, 0)
    e = 1e-2
    D = lambda h: (P.gpu_residual(U + h * V) - P.gpu_residual(U - h * V)) / (2 * h)  # noqa: E731
    fd = (4 * D(e) - D(2 * e)) / 3
    assert rel_err(JV, fd) <= 1e-10


def test_residual_ignores_stored_hanging_values():
    """Hanging entries of U only enter their own constraint rows."""
    P, U, _ = _setup(CASES[3], seed=3)
    F1 = P.gpu_residual(U)
    U2 = U.copy()
    U2[P.mesh.hanging] += 5.0
    F2 = P.gpu_residual(U2)
    free = ~P.mesh.hanging
    # equal up to the summation order of the scatter
    assert np.abs(F1[free] - F2[free]).max() <= 1e-14 * np.abs(F1[free]).max()
    assert np.allclose(F2[P.mesh.hanging] - F1[P.mesh.hanging], 5.0, atol=1e-12)


@pytest.mark.parametrize("case", [CASES[1], CASES[3]], ids=[CASES[1][0], CASES[3][0]])
def test_patch_kernels_are_deterministic_and_match_atomic_path(case, monkeypatch):
    """The shared-memory patch kernels sum in a fixed order: two evaluations are bitwise
    equal; they agree with the default global-atomics kernels to rounding and with the
    oracle at the FP64 bar."""
    monkeypatch.setenv("PNP_ELEMENT_PATH", "patch")
    P, U, V = _setup(case)
    outs = [(P.gpu_residual(U), P.gpu_jv(U, V, 0), P.gpu_jv(U, V, 1)) for _ in range(2)]
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)
    assert rel_err(outs[0][0], P.oracle_residual(U)) <= TOL64
    assert rel_err(outs[0][1], P.oracle_jv(U, V)) <= TOL64
    monkeypatch.delenv("PNP_ELEMENT_PATH")
    name, oc, kw, bcs = case
    Q = Pair(oc, kw, bcs)
    Q.set_state(P.Uk, P.Ukm1, P.vel)
    F, JV, JV32 = outs[0]
    assert rel_err(Q.gpu_residual(U), F) <= 1e-14
    assert rel_err(Q.gpu_jv(U, V, 0), JV) <= 1e-14
    assert np.all(field_max_err(Q.gpu_jv(U, V, 1), JV32) <= 1e-5)


def test_norm2_is_reproducible_and_accurate():
    P, U, _ = _setup(CASES[2])
    torch = P.torch
    for n in (0, 1, 7, 1000, 3 * P.mesh.n_nodes, 2_000_003):
        x = torch.from_numpy(np.random.default_rng(n).normal(size=n)).cuda()
        a, b = P.ctx.norm2(x), P.ctx.norm2(x)
        assert a == b
        ref = float(np.linalg.norm(x.cpu().numpy()))
        assert abs(a - ref) <= 1e-14 * max(ref, 1e-300) + (0 if n else 0.0)


def test_gmres_solves_oracle_system():
    import scipy.sparse.linalg as spla
    P, U, V = _setup(CASES[1], seed=9)
    P.ctx.set_params(P.pnp.default_params(**P.params_kw, gmres_restart=40, gmres_max_it=4000))
    J = P.oracle_jacobian(U)
    b = W.random_direction(P.mesh.ijk, P.oc.max_level, 77)
    x_ref = spla.spsolve(J.tocsc(), b.reshape(-1)).reshape(-1, 3)
    x = P.torch.zeros((P.mesh.n_nodes, 3), dtype=P.torch.float64, device="cuda")
    st = P.ctx.gmres(P.dev(U), P.dev(b), x, 1e-11, 0)
    assert st.status == 0 and st.krylov_its > 0
    x = x.cpu().numpy()
    assert np.linalg.norm(J @ x.reshape(-1) - b.reshape(-1)) <= 1e-10 * np.linalg.norm(b)
    assert rel_err(x, x_ref) <= 1e-6


@pytest.mark.parametrize("inner", [0, 6])
def test_fp32_gmres_solves_oracle_system(inner):
    """FP32 J V inside GMRES: plain right preconditioning (inner = 0) and flexible GMRES
    with an inner FP32 GMRES(6) preconditioner both solve the oracle's system to the
    accuracy FP32 J V allows (the residual is measured with the oracle's FP64 Jacobian)."""
    import scipy.sparse.linalg as spla
    P, U, V = _setup(CASES[1], seed=9)
    P.ctx.set_params(P.pnp.default_params(**P.params_kw, gmres_restart=40, gmres_max_it=4000, gmres_inner=inner))
    J = P.oracle_jacobian(U)
    b = W.random_direction(P.mesh.ijk, P.oc.max_level, 77)
    x_ref = spla.spsolve(J.tocsc(), b.reshape(-1)).reshape(-1, 3)
    x = P.torch.zeros((P.mesh.n_nodes, 3), dtype=P.torch.float64, device="cuda")
    st = P.ctx.gmres(P.dev(U), P.dev(b), x, 1e-4, P.pnp.PNP_F32)
    assert st.status == 0 and st.krylov_its > 0
    x = x.cpu().numpy()
    # against the oracle's assembled FP64 Jacobian: the FP32 operator's error floor
    # (about 3e-5 relative on this case) plus the requested 1e-4
    assert np.linalg.norm(J @ x.reshape(-1) - b.reshape(-1)) <= 3e-4 * np.linalg.norm(b)
    assert rel_err(x, x_ref) <= 0.05
    if inner:
        assert st.jv_evals >= inner * st.krylov_its  # the inner steps ran


def test_fp64_flexible_gmres_solves_oracle_system():
    """Flexible GMRES with an inner FP64 GMRES(6) preconditioner (PNP_F64 with gmres_inner):
    the FP64 counterpart of the mixed-precision nested solver reaches the oracle's direct
    solution to FP64 accuracy."""
    import scipy.sparse.linalg as spla
    P, U, V = _setup(CASES[1], seed=9)
    P.ctx.set_params(P.pnp.default_params(**P.params_kw, gmres_restart=40, gmres_max_it=4000, gmres_inner=6))
    J = P.oracle_jacobian(U)
    b = W.random_direction(P.mesh.ijk, P.oc.max_level, 77)
    x_ref = spla.spsolve(J.tocsc(), b.reshape(-1)).reshape(-1, 3)
    x = P.torch.zeros((P.mesh.n_nodes, 3), dtype=P.torch.float64, device="cuda")
    st = P.ctx.gmres(P.dev(U), P.dev(b), x, 1e-11, P.pnp.PNP_F64)
    assert st.status == 0 and st.krylov_its > 0
    assert st.jv_evals >= 6 * st.krylov_its  # the inner steps ran
    x = x.cpu().numpy()
    assert np.linalg.norm(J @ x.reshape(-1) - b.reshape(-1)) <= 1e-10 * np.linalg.norm(b)
    assert rel_err(x, x_ref) <= 1e-8


def test_fp64_nested_inexact_newton_time_steps_match_oracle():
    """Three BDF steps with FP64 J V, the nested FP64 solver and Eisenstat-Walker forcing
    (the FP64 arm of the mixed-precision comparison) reach the oracle's steps."""
    oc = W.random_balanced_octants(3, 1, 4, 0.3, 21)
    bcs = W.membrane_bcs(3, 4.0, 2.0)
    kw = dict(eps=0.05, dt=0.01, newton_rtol=1e-11, gmres_restart=30, gmres_max_it=20000, start_mode=1,
              gmres_inner=8, newton_ew_f64=1, ew_eta_min=1e-6)
    P = Pair(oc, kw, bcs)
    L = oc.max_level
    U0 = W.noisy_state(P.mesh.ijk, L, seed=3, amp=1e-2, phi_bottom=0.0, phi_top=4.0)
    P.ctx.set_field(P.pnp.PNP_FIELD_U, U0)
    P.ctx.make_consistent()
    U0c = P.ctx.get_field(P.pnp.PNP_FIELD_U)
    P.ctx.reset_history()
    Uk, Ukm1 = P.to_ora(U0c), P.to_ora(U0c)
    for k in range(3):
        st = P.ctx.time_step()
        assert st.status == 0
        beta = O.bdf_coefficients(k)
        op = O.Params(eps=0.05, dt=0.01, beta=beta, bc_type=bcs.types, bc_val=bcs.values)
        start = Uk if k == 0 else 2 * Uk - Ukm1
        res = O.newton(P.om, op, start, Uk, Ukm1, None, rtol=1e-13)
        Ukm1, Uk = Uk, res.U
        Ug = P.ctx.get_field(P.pnp.PNP_FIELD_U)
        assert rel_err(P.to_ora(Ug), Uk) <= 1e-9, k


@pytest.mark.parametrize("ci", [1, 3])
def test_multigrid_preconditioned_gmres_solves_oracle_system(ci):
    """Flexible GMRES preconditioned by the geometric-multigrid V-cycle (FP32, coarse
    octrees by capping levels, injected state, block-Jacobi smoothing) solves the oracle's
    system to the accuracy FP32 J V allows, on a 2D and a 3D octree with hanging nodes."""
    import scipy.sparse.linalg as spla
    P, U, V = _setup(CASES[ci], seed=9)
    P.ctx.set_params(P.pnp.default_params(**P.params_kw, gmres_restart=40, gmres_max_it=4000, mg_levels=2))
    J = P.oracle_jacobian(U)
    b = W.random_direction(P.mesh.ijk, P.oc.max_level, 77)
    x_ref = spla.spsolve(J.tocsc(), b.reshape(-1)).reshape(-1, 3)
    x = P.torch.zeros((P.mesh.n_nodes, 3), dtype=P.torch.float64, device="cuda")
    st = P.ctx.gmres(P.dev(U), P.dev(b), x, 1e-4, P.pnp.PNP_F32)
    assert st.status == 0 and st.krylov_its > 0
    x = x.cpu().numpy()
    assert np.linalg.norm(J @ x.reshape(-1) - b.reshape(-1)) <= 3e-4 * np.linalg.norm(b)
    assert rel_err(x, x_ref) <= 0.05


def test_multigrid_time_steps_match_oracle():
    """Three BDF steps with the multigrid-preconditioned mixed solver reach the oracle's
    steps (the preconditioner changes the path, not the converged state)."""
    oc = W.random_balanced_octants(3, 1, 4, 0.3, 21)
    bcs = W.membrane_bcs(3, 4.0, 2.0)
    kw = dict(eps=0.05, dt=0.01, newton_rtol=1e-11, gmres_restart=40, gmres_max_it=20000, start_mode=1,
              precision=1, mg_levels=3, ew_eta_min=1e-6)
    P = Pair(oc, kw, bcs)
    L = oc.max_level
    U0 = W.noisy_state(P.mesh.ijk, L, seed=3, amp=1e-2, phi_bottom=0.0, phi_top=4.0)
    P.ctx.set_field(P.pnp.PNP_FIELD_U, U0)
    P.ctx.make_consistent()
    U0c = P.ctx.get_field(P.pnp.PNP_FIELD_U)
    P.ctx.reset_history()
    Uk, Ukm1 = P.to_ora(U0c), P.to_ora(U0c)
    for k in range(3):
        st = P.ctx.time_step()
        assert st.status == 0
        beta = O.bdf_coefficients(k)
        op = O.Params(eps=0.05, dt=0.01, beta=beta, bc_type=bcs.types, bc_val=bcs.values)
        start = Uk if k == 0 else 2 * Uk - Ukm1
        res = O.newton(P.om, op, start, Uk, Ukm1, None, rtol=1e-13)
        Ukm1, Uk = Uk, res.U
        Ug = P.ctx.get_field(P.pnp.PNP_FIELD_U)
        assert rel_err(P.to_ora(Ug), Uk) <= 1e-9, k


def test_newton_equilibrium_matches_oracle():
    """2D steady double layer, level 5, Lambda = 0.01, V = 1 (the equilibrium case):
    GPU Newton (FP64, exact-Jacobian GMRES) and the oracle's direct-solve Newton converge
    to the same discrete state."""
    oc = W.uniform_octants(2, 5)
    bcs = W.equilibrium_bcs(2, 1.0)
    kw = dict(eps=0.01, steady=1, newton_rtol=1e-10, line_search=0, gmres_rtol=1e-12, gmres_restart=60,
              gmres_max_it=20000)
    P = Pair(oc, kw, bcs)
    P.set_state()
    U0 = np.zeros((P.mesh.n_nodes, 3)); U0[:, :2] = 1.0
    U0[:, 2] = 1.0 - P.mesh.ijk[:, 1] / (1 << oc.max_level)
    P.ctx.set_field(P.pnp.PNP_FIELD_U, U0)
    st = P.ctx.newton_solve()
    assert st.status == 0 and st.newton_its <= 8
    Ug = P.ctx.get_field(P.pnp.PNP_FIELD_U)
    ref = O.newton(P.om, P.op, P.to_ora(U0), rtol=1e-12, line_search=False)
    Uo = P.to_lib(ref.U)
    assert rel_err(Ug, Uo) <= 1e-9
    # the converged residual is small in the oracle's own measure too
    assert np.linalg.norm(P.oracle_residual(Ug)) <= 1e-9 * st.res0


def test_bdf_time_steps_match_oracle():
    """Three BDF steps (BDF1 then BDF2) on a 3D octree with a prescribed velocity."""
    oc = W.random_balanced_octants(3, 1, 4, 0.3, 21)
    bcs = W.membrane_bcs(3, 4.0, 2.0)
    kw = dict(eps=0.05, dt=0.01, newton_rtol=1e-11, gmres_rtol=1e-12, gmres_restart=60, gmres_max_it=20000,
              start_mode=1)
    P = Pair(oc, kw, bcs)
    L = oc.max_level
    U0 = W.noisy_state(P.mesh.ijk, L, seed=3, amp=1e-2, phi_bottom=0.0, phi_top=4.0)
    vel = W.random_velocity(P.mesh.ijk, L, 5, amp=1.0)
    P.ctx.set_field(P.pnp.PNP_FIELD_U, U0)
    P.ctx.make_consistent()
    U0c = P.ctx.get_field(P.pnp.PNP_FIELD_U)
    P.ctx.reset_history()
    P.ctx.set_field(P.pnp.PNP_FIELD_VELOCITY, vel)
    P.ctx.set_field(P.pnp.PNP_FIELD_VELOCITY_PREV, vel)
    Uk, Ukm1 = P.to_ora(U0c), P.to_ora(U0c)
    v3 = P.to_ora(vel)
    for k in range(3):
        st = P.ctx.time_step()
        assert st.status == 0
        beta = O.bdf_coefficients(k)
        op = O.Params(eps=0.05, dt=0.01, beta=beta, bc_type=bcs.types, bc_val=bcs.values)
        start = Uk if k == 0 else 2 * Uk - Ukm1
        res = O.newton(P.om, op, start, Uk, Ukm1, v3, rtol=1e-13)
        Ukm1, Uk = Uk, res.U
        Ug = P.ctx.get_field(P.pnp.PNP_FIELD_U)
        assert rel_err(P.to_ora(Ug), Uk) <= 1e-9, k
    assert P.ctx.step_count() == 3


def test_inner_solve_graph_replay_matches_eager_launches():
    """The flexible solve's inner FP32 GMRES runs eagerly the first time and while
    profiling is on, and as a captured CUDA graph otherwise: both solve the same system
    to the requested tolerance, a replay counts its kernels and J V applications, and a
    change of the physical parameters triggers a new capture."""
    P, U, V = _setup(CASES[1], seed=9)
    P.ctx.set_params(P.pnp.default_params(**P.params_kw, gmres_restart=40, gmres_max_it=4000, gmres_inner=6))
    b = P.dev(W.random_direction(P.mesh.ijk, P.oc.max_level, 77))
    Ud = P.dev(U)

    def solve():
        x = P.torch.zeros_like(Ud)
        st = P.ctx.gmres(Ud, b, x, 1e-4, P.pnp.PNP_F32)
        assert st.status == 0
        return x.cpu().numpy(), st

    P.ctx.profile_enable(True)
    x_eager, st_e = solve()  # eager: profiling on
    P.ctx.profile_enable(False)
    c0 = P.pnp.graph_captures()
    x1, st1 = solve()  # first unprofiled solve: capture, then replays
    c1 = P.pnp.graph_captures()
    l0 = P.pnp.kernel_launches()
    x2, st2 = solve()  # replays only
    assert P.pnp.graph_captures() == c1 and c1 == c0 + 1
    assert P.pnp.kernel_launches() - l0 > 6 * st2.krylov_its  # replays counted
    assert st2.jv_evals >= 6 * st2.krylov_its
    for x in (x1, x2):
        assert rel_err(x, x_eager) <= 1e-3
    # new parameters (time step size) change the captured kernels' arguments: re-capture
    p = P.ctx.get_params()
    p.dt *= 0.5
    P.ctx.set_params(p)
    solve()
    assert P.pnp.graph_captures() == c1 + 1
