"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test ties one part of the oracle to something other than its own code:
exact polynomial integration (sympy), Kronecker-product Q1 operators, the full
strong form, finite differences of the residual, conservation, manufactured-solution
convergence rates (Sec. 5.1), the Gouy-Chapman double layer, and Newton's
quadratic convergence.  None of them needs a GPU.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from paper_2301_05985_gb300 import workloads as W


def _lex_index(mesh, n1):
    """Lexicographic (x fastest) index of every oracle node of a uniform grid with n1 nodes per axis."""
    idx = np.zeros(mesh.n_nodes, np.int64)
    scale = 1 << 0
    for a in range(mesh.dim):
        idx += mesh.ijk[:, a] * (n1 ** a) * scale
    return idx


def _kron_ops(dim, n):
    h = 1.0 / n
    m_e = h / 6.0 * np.array([[2.0, 1.0], [1.0, 2.0]])
    k_e = 1.0 / h * np.array([[1.0, -1.0], [-1.0, 1.0]])
    M1 = np.zeros((n + 1, n + 1)); K1 = np.zeros((n + 1, n + 1))
    for e in range(n):
        M1[e:e + 2, e:e + 2] += m_e
        K1[e:e + 2, e:e + 2] += k_e
    M1, K1 = sp.csr_matrix(M1), sp.csr_matrix(K1)
    if dim == 2:
        K = sp.kron(M1, K1) + sp.kron(K1, M1)
        M = sp.kron(M1, M1)
    else:
        K = sp.kron(M1, sp.kron(M1, K1)) + sp.kron(M1, sp.kron(K1, M1)) + sp.kron(K1, sp.kron(M1, M1))
        M = sp.kron(M1, sp.kron(M1, M1))
    return M.tocsr(), K.tocsr()


# ------------------------------------------------------------------------ mesh
def test_mesh_counts_uniform():
    for dim, lev in [(2, 3), (3, 2)]:
        m = O.OracleMesh(W.uniform_octants(dim, lev))
        assert m.n_elem == (1 << lev) ** dim
        assert m.n_nodes == ((1 << lev) + 1) ** dim
        assert m.n_hanging == 0


def test_mesh_rejects_unbalanced_and_overlaps():
    # one level-1 quadrant next to level-3 quadrants: a 2-level jump across a face
    L = 3
    anchors, levels = [], []
    for (ax, ay, l) in [(0, 4, 1), (4, 4, 1), (4, 0, 1)]:
        anchors.append((ax, ay)); levels.append(l)
    for i in range(4):
        for j in range(4):
            anchors.append((i, j)); levels.append(3)
    oc = W.Octants(2, L, np.array(anchors, np.int32), np.array(levels, np.uint8))
    with pytest.raises(ValueError, match="code 3"):
        O.OracleMesh(oc)
    # overlapping octants
    oc = W.Octants(2, 1, np.array([(0, 0), (0, 0), (1, 0), (0, 1), (1, 1)], np.int32),
                   np.array([0, 1, 1, 1, 1], np.uint8))
    with pytest.raises(ValueError):
        O.OracleMesh(oc)


def test_hanging_constraints_reproduce_linear_fields():
    """Parents/weights of every hanging node reproduce a globally linear field exactly."""
    for dim, seed in [(2, 1), (3, 2)]:
        oc = W.random_balanced_octants(dim, 1, 3 if dim == 3 else 4, 0.35, seed)
        m = O.OracleMesh(oc)
        assert m.n_hanging > 0
        a = np.array([0.3, -1.7, 2.1])[:dim]
        lin = 0.25 + m.x @ a
        U = np.zeros((m.n_nodes, 3)); U[:, 2] = lin
        U[m.hanging == 1, 2] = 123.0  # garbage, must be overwritten by interpolation
        p = O.Params(eps=0.3, steady=True, bc_type=np.zeros((2 * dim, 3), np.int32), bc_val=np.zeros((2 * dim, 3)))
        Uc = m.make_consistent(U, p)
        np.testing.assert_allclose(Uc[:, 2], lin, rtol=0, atol=1e-14)


def test_linear_field_interior_rows_vanish_on_hanging_mesh():
    """For linear phi and c = 0 the Poisson rows are 2 Lambda^2 (grad N_i, a): zero at every
    interior free node, and zero in sum, only if the constrained basis is conforming."""
    for dim, seed in [(2, 3), (3, 4)]:
        oc = W.random_balanced_octants(dim, 1, 3 if dim == 3 else 4, 0.35, seed)
        m = O.OracleMesh(oc)
        a = np.array([0.7, -0.4, 1.3])[:dim]
        U = np.zeros((m.n_nodes, 3)); U[:, 2] = m.x @ a
        bc = W.all_natural_bcs(dim)
        p = O.Params(eps=0.5, steady=True, bc_type=bc.types, bc_val=bc.values)
        F = m.residual(p, m.make_consistent(U, p))
        size = 1 << m.max_level
        interior = np.all((m.ijk > 0) & (m.ijk < size), axis=1) & (m.hanging == 0)
        assert np.abs(F[interior, 2]).max() < 1e-13
        assert abs(F[m.hanging == 0, 2].sum()) < 1e-13
        # c rows: steady, v = 0, c = 0 -> identically zero
        assert np.abs(F[m.hanging == 0, :2]).max() < 1e-14


# ------------------------------------------------------------------------ Q1 operators
@pytest.mark.parametrize("dim,lev", [(2, 3), (3, 2)])
def test_poisson_rows_equal_kronecker_stiffness(dim, lev):
    m = O.OracleMesh(W.uniform_octants(dim, lev))
    n = 1 << lev
    M, K = _kron_ops(dim, n)
    lex = _lex_index(m, n + 1)
    rng = np.random.default_rng(0)
    phi = rng.uniform(-1, 1, m.n_nodes)
    U = np.zeros((m.n_nodes, 3)); U[:, 2] = phi
    eps = 0.37
    bc = W.all_natural_bcs(dim)
    p = O.Params(eps=eps, steady=True, bc_type=bc.types, bc_val=bc.values)
    F = m.residual(p, U)
    phi_lex = np.zeros(m.n_nodes); phi_lex[lex] = phi
    ref = 2 * eps**2 * (K @ phi_lex)
    np.testing.assert_allclose(F[:, 2], ref[lex], rtol=0, atol=1e-13 * np.abs(ref).max())
    assert np.abs(F[:, :2]).max() < 1e-15


@pytest.mark.parametrize("dim,lev", [(2, 3), (3, 2)])
def test_transient_rows_equal_kronecker_mass_plus_stiffness(dim, lev):
    """v = 0, phi = 0, no history: F_s = (beta0/dt) M c_s + K c_s and
    F_phi = (tau beta0/dt - 1) M (c+ - c-) with the constant tau of a uniform grid."""
    m = O.OracleMesh(W.uniform_octants(dim, lev))
    n = 1 << lev
    M, K = _kron_ops(dim, n)
    lex = _lex_index(m, n + 1)
    rng = np.random.default_rng(1)
    U = np.zeros((m.n_nodes, 3)); U[:, :2] = rng.uniform(0.2, 2.0, (m.n_nodes, 2))
    dt, b0 = 0.01, 1.5
    bc = W.all_natural_bcs(dim)
    p = O.Params(eps=0.2, dt=dt, beta=(b0, 0.0, 0.0), bc_type=bc.types, bc_val=bc.values)
    F = m.residual(p, U)
    h = 1.0 / n
    tau = (4.0 / dt**2 + 6.0 * dim * (2.0 / h) ** 4) ** -0.5  # Sec. 3.1 with v = 0
    for s in range(2):
        c = np.zeros(m.n_nodes); c[lex] = U[:, s]
        ref = (b0 / dt) * (M @ c) + K @ c
        np.testing.assert_allclose(F[:, s], ref[lex], rtol=0, atol=1e-12 * np.abs(ref).max())
    q = np.zeros(m.n_nodes); q[lex] = U[:, 0] - U[:, 1]
    ref = (tau * b0 / dt - 1.0) * (M @ q)
    np.testing.assert_allclose(F[:, 2], ref[lex], rtol=0, atol=1e-12 * np.abs(ref).max())


# ------------------------------------------------------------------------ exact integration
def _poly_integral_unit_box(expr, syms):
    import sympy
    P = sympy.Poly(sympy.expand(expr), *syms)
    tot = 0.0
    for mon, coef in P.terms():
        t = float(coef)
        for e in mon:
            t /= (e + 1)
        tot += t
    return tot


@pytest.mark.parametrize("dim", [2, 3])
def test_galerkin_terms_match_exact_integration(dim):
    """With the fine-scale terms off, every term of Def. 3 is a polynomial that 2-point Gauss
    integrates exactly; compare with sympy's exact integration of the weak form on one element."""
    sympy = pytest.importorskip("sympy")
    xs = sympy.symbols("x0:%d" % dim)
    oc = W.Octants(dim, 0, np.zeros((1, dim), np.int32), np.zeros(1, np.uint8))
    m = O.OracleMesh(oc)
    rng = np.random.default_rng(7 + dim)
    U = rng.uniform(-1, 1, (m.n_nodes, 3)); Uk = rng.uniform(-1, 1, (m.n_nodes, 3))
    Ukm1 = rng.uniform(-1, 1, (m.n_nodes, 3)); vel = rng.uniform(-2, 2, (m.n_nodes, dim))
    eps, dt, beta = 0.3, 0.25, (1.5, -2.0, 0.5)
    bc = W.all_natural_bcs(dim)
    p = O.Params(eps=eps, dt=dt, beta=beta, vms=False, bc_type=bc.types, bc_val=bc.values)
    F = m.residual(p, U, Uk, Ukm1, vel)

    def shape(node):
        e = 1
        for k in range(dim):
            e *= xs[k] if m.ijk[node, k] else (1 - xs[k])
        return e

    N = [shape(i) for i in range(m.n_nodes)]
    fld = lambda arr: sum(arr[i] * N[i] for i in range(m.n_nodes))  # noqa: E731
    grad = lambda f: [sympy.diff(f, x) for x in xs]  # noqa: E731
    c = [fld(U[:, 0]), fld(U[:, 1])]
    phi = fld(U[:, 2])
    hist = [(beta[1] * fld(Uk[:, s]) + beta[2] * fld(Ukm1[:, s])) / dt for s in range(2)]
    v = [fld(vel[:, k]) for k in range(dim)]
    gphi = grad(phi)
    z = [1.0, -1.0]
    for i in range(m.n_nodes):
        gN = grad(N[i])
        for s in range(2):
            gc = grad(c[s])
            integrand = N[i] * (beta[0] / dt * c[s] + hist[s] + sum(v[k] * gc[k] for k in range(dim)))
            integrand += sum(gN[k] * (gc[k] + z[s] * c[s] * gphi[k]) for k in range(dim))
            ref = _poly_integral_unit_box(integrand, xs)
            assert abs(F[i, s] - ref) < 1e-12 * max(1.0, abs(ref)), (i, s, F[i, s], ref)
        integrand = 2 * eps**2 * sum(gN[k] * gphi[k] for k in range(dim)) - N[i] * (c[0] - c[1])
        ref = _poly_integral_unit_box(integrand, xs)
        assert abs(F[i, 2] - ref) < 1e-12 * max(1.0, abs(ref))


@pytest.mark.parametrize("dim", [2, 3])
def test_strong_residual_at_gauss_points(dim):
    """R_s of the oracle equals the full strong Nernst-Planck residual
    (b0 c + b1 c^k + b2 c^{k-1})/dt + v.grad c - div(grad c + z c grad phi), evaluated
    symbolically on the Q1 interpolant (so dropping the Laplacians must be exact)."""
    sympy = pytest.importorskip("sympy")
    xs = sympy.symbols("x0:%d" % dim)
    oc = W.Octants(dim, 0, np.zeros((1, dim), np.int32), np.zeros(1, np.uint8))
    m = O.OracleMesh(oc)
    rng = np.random.default_rng(11 + dim)
    U = rng.uniform(-1, 1, (m.n_nodes, 3)); Uk = rng.uniform(-1, 1, (m.n_nodes, 3))
    Ukm1 = rng.uniform(-1, 1, (m.n_nodes, 3)); vel = rng.uniform(-2, 2, (m.n_nodes, dim))
    dt, beta, CI = 0.2, (1.5, -2.0, 0.5), 6.0
    bc = W.all_natural_bcs(dim)
    p = O.Params(eps=0.1, dt=dt, beta=beta, C_I=CI, bc_type=bc.types, bc_val=bc.values)

    def shape(node):
        e = 1
        for k in range(dim):
            e *= xs[k] if m.ijk[node, k] else (1 - xs[k])
        return e

    N = [shape(i) for i in range(m.n_nodes)]
    fld = lambda arr: sum(arr[i] * N[i] for i in range(m.n_nodes))  # noqa: E731
    c = [fld(U[:, 0]), fld(U[:, 1])]
    phi = fld(U[:, 2])
    v = [fld(vel[:, k]) for k in range(dim)]
    z = [1, -1]
    g = 1 / math.sqrt(3)
    for q in range(1 << dim):
        pt = {xs[k]: 0.5 * (1 + (g if (q >> k) & 1 else -g)) for k in range(dim)}
        out = m.qp_eval(p, 0, q, U, Uk, Ukm1, vel)
        for s in range(2):
            hist = (beta[1] * fld(Uk[:, s]) + beta[2] * fld(Ukm1[:, s])) / dt
            flux = [sympy.diff(c[s], x) + z[s] * c[s] * sympy.diff(phi, x) for x in xs]
            strong = beta[0] / dt * c[s] + hist + sum(v[k] * sympy.diff(c[s], xs[k]) for k in range(dim)) \
                - sum(sympy.diff(flux[k], xs[k]) for k in range(dim))
            ref = float(strong.subs(pt))
            assert abs(out[s] - ref) < 1e-12 * max(1.0, abs(ref))
        # tau_c of Sec. 3.1 with G = (2/h)^2 I, h = 1
        vv = sum(float(v[k].subs(pt)) ** 2 for k in range(dim))
        tau = (4 / dt**2 + 4 * vv + CI * dim * 16) ** -0.5
        assert abs(out[2] - tau) < 1e-14


# ------------------------------------------------------------------------ Jacobian
def _random_problem(dim, seed, transient=True):
    oc = W.random_balanced_octants(dim, 1, 3 if dim == 3 else 4, 0.35, seed)
    m = O.OracleMesh(oc)
    bc = W.membrane_bcs(dim, V=3.0, membrane_c_plus=2.0)
    p = O.Params(eps=0.05, dt=0.05, beta=(1.5, -2.0, 0.5) if transient else (1, -1, 0), steady=not transient,
                 bc_type=bc.types, bc_val=bc.values)
    U = m.make_consistent(W.random_state(m.ijk, m.max_level, seed), p)
    Uk = W.random_state(m.ijk, m.max_level, seed + 100)
    Ukm1 = W.random_state(m.ijk, m.max_level, seed + 200)
    vel = W.random_velocity(m.ijk, m.max_level, seed, amp=2.0)
    V = W.random_direction(m.ijk, m.max_level, seed + 300)
    return m, p, U, Uk, Ukm1, vel, V


@pytest.mark.parametrize("dim,transient", [(2, True), (3, True), (2, False)])
def test_jacobian_matches_richardson_central_differences(dim, transient):
    """The residual is a cubic polynomial in U (tau_c does not depend on U), so the
    Richardson combination of central differences at steps e and 2e is exact."""
    m, p, U, Uk, Ukm1, vel, V = _random_problem(dim, 5 + dim, transient)
    J = m.jacobian(p, U, Uk, Ukm1, vel)
    JV = (J @ V.reshape(-1)).reshape(-1, 3)
    eps = 1e-2

    def D(e):
        return (m.residual(p, U + e * V, Uk, Ukm1, vel) - m.residual(p, U - e * V, Uk, Ukm1, vel)) / (2 * e)

    fd = (4 * D(eps) - D(2 * eps)) / 3
    assert np.linalg.norm(JV - fd) <= 1e-9 * np.linalg.norm(JV)
    # one-sided difference converges at first order (slope check)
    e1 = np.linalg.norm((m.residual(p, U + 1e-4 * V, Uk, Ukm1, vel) - m.residual(p, U, Uk, Ukm1, vel)) / 1e-4 - JV)
    e2 = np.linalg.norm((m.residual(p, U + 5e-5 * V, Uk, Ukm1, vel) - m.residual(p, U, Uk, Ukm1, vel)) / 5e-5 - JV)
    assert 1.8 < e1 / e2 < 2.2
    # the matrix-free linearisation is an independent derivation of the same operator
    JVmf = m.jv(p, U, V, Uk, Ukm1, vel)
    assert np.linalg.norm(JVmf - JV) <= 1e-13 * np.linalg.norm(JV)


def test_jv_is_linear_in_direction():
    m, p, U, Uk, Ukm1, vel, V = _random_problem(3, 21)
    Wd = W.random_direction(m.ijk, m.max_level, 99)
    a, b = 0.7, -2.3
    lhs = m.jv(p, U, a * V + b * Wd, Uk, Ukm1, vel)
    rhs = a * m.jv(p, U, V, Uk, Ukm1, vel) + b * m.jv(p, U, Wd, Uk, Ukm1, vel)
    assert np.linalg.norm(lhs - rhs) <= 1e-14 * np.linalg.norm(rhs)


@pytest.mark.parametrize("dim", [2, 3])
def test_fine_scale_terms_energy_identity(dim):
    """Steady, no forcing: R_s = (v - z_s grad phi).grad c_s = P_s.grad c_s, so the fine-scale
    part of the Nernst-Planck rows, (grad q, tau R_s P_s), tested with q = c_s gives
    sum_qp w tau R_s^2 >= 0, and the fine-scale part of the Poisson rows, (q, sum z tau R),
    tested with q = 1 gives sum_qp w sum_s z_s tau R_s.  Both right-hand sides come from the
    Gauss-point values of R and tau alone, which pins the sign and placement of the terms."""
    oc = W.random_balanced_octants(dim, 1, 3 if dim == 3 else 4, 0.35, 41 + dim)
    m = O.OracleMesh(oc)
    bc = W.all_natural_bcs(dim)
    pon = O.Params(eps=0.1, steady=True, vms=True, bc_type=bc.types, bc_val=bc.values)
    poff = O.Params(eps=0.1, steady=True, vms=False, bc_type=bc.types, bc_val=bc.values)
    U = m.make_consistent(W.random_state(m.ijk, m.max_level, 8), pon)
    vel = W.random_velocity(m.ijk, m.max_level, 9, amp=3.0)
    dF = m.residual(pon, U, adv=vel) - m.residual(poff, U, adv=vel)
    free = m.hanging == 0
    w = 0.5 ** (dim * (np.array(oc.levels, np.float64) + 1))  # (h/2)^dim per Gauss point
    e_sq = np.zeros(2); e_ch = 0.0
    for e in range(m.n_elem):
        for q in range(1 << dim):
            Rp, Rm, tau = m.qp_eval(pon, e, q, U, adv=vel)
            e_sq += w[e] * tau * np.array([Rp**2, Rm**2])
            e_ch += w[e] * tau * (Rp - Rm)
    for s in range(2):
        lhs = np.dot(U[free, s], dF[free, s])
        assert e_sq[s] > 0 and abs(lhs - e_sq[s]) < 1e-12 * e_sq[s]
    assert abs(dF[free, 2].sum() - e_ch) < 1e-12 * max(1.0, abs(e_ch))


# ------------------------------------------------------------------------ conservation
@pytest.mark.parametrize("dim", [2, 3])
def test_discrete_conservation_with_zero_flux(dim):
    """Zero flux everywhere and v = 0: every grad(q) term sums to grad(1) = 0, so
    sum_i F_{s,i} = integral of (beta0 c_s + beta1 c^k_s + beta2 c^{k-1}_s)/dt, and with a
    constant phi sum_i F_{phi,i} = -(1 - tau beta0/dt) int (c+ - c-) + tau int (h+ - h-)
    on a uniform-size region (tau constant).  The integral of a Q1 field over a cube is
    its corner mean times the volume."""
    oc = W.random_balanced_octants(dim, 1, 3 if dim == 3 else 4, 0.35, 31 + dim)
    m = O.OracleMesh(oc)
    bc = W.all_natural_bcs(dim)
    dt, beta = 0.1, (1.5, -2.0, 0.5)
    p = O.Params(eps=0.1, dt=dt, beta=beta, bc_type=bc.types, bc_val=bc.values)
    U = m.make_consistent(W.random_state(m.ijk, m.max_level, 3), p)
    Uk = m.make_consistent(W.random_state(m.ijk, m.max_level, 4), p)
    Ukm1 = m.make_consistent(W.random_state(m.ijk, m.max_level, 5), p)
    F = m.residual(p, U, Uk, Ukm1, None)
    free = m.hanging == 0
    lev = np.array(oc.levels)
    # oracle element order == input octant order
    vol = 0.5 ** (dim * lev.astype(np.float64))
    for s in range(2):
        field = (beta[0] * U[:, s] + beta[1] * Uk[:, s] + beta[2] * Ukm1[:, s]) / dt
        integral = np.sum(vol * field[m.el_nodes].mean(axis=1))
        assert abs(F[free, s].sum() - integral) < 1e-12 * abs(integral)


# ------------------------------------------------------------------------ MMS (Sec. 5.1)
@pytest.mark.slow
@pytest.mark.parametrize("eps", [math.sqrt(0.5), 0.1])
def test_mms_spatial_rate_is_two(eps):
    errs = []
    levels = [3, 4, 5, 6]
    for lev in levels:
        mesh, U, Uex, _ = O.mms_run(W.uniform_octants(2, lev), eps, dt=1.0, n_steps=0, steady=True)
        errs.append(O.l2_error(mesh, U, Uex))
    errs = np.array(errs)
    slopes = np.log2(errs[:-1] / errs[1:])
    assert np.all(np.abs(slopes[-1] - 2.0) < 0.15), slopes


@pytest.mark.slow
def test_mms_spatial_rate_is_two_3d():
    errs = []
    for lev in [2, 3, 4]:
        mesh, U, Uex, _ = O.mms_run(W.uniform_octants(3, lev), math.sqrt(0.5), dt=1.0, n_steps=0, steady=True)
        errs.append(O.l2_error(mesh, U, Uex))
    errs = np.array(errs)
    slopes = np.log2(errs[:-1] / errs[1:])
    assert np.all(np.abs(slopes[-1] - 2.0) < 0.3), slopes


@pytest.mark.slow
def test_mms_temporal_rate_is_two():
    """BDF2 (BDF1 first step) with the extrapolated velocity: successive differences of
    the solution at t = 0.4 under dt halving shrink by 4 on a fixed mesh."""
    sols = []
    for nst in [4, 8, 16, 32]:
        mesh, U, _, t = O.mms_run(W.uniform_octants(2, 4), math.sqrt(0.5), dt=0.4 / nst, n_steps=nst)
        assert abs(t - 0.4) < 1e-12
        sols.append(U)
    d = [np.linalg.norm(sols[i] - sols[i + 1]) for i in range(3)]
    ratios = [d[i] / d[i + 1] for i in range(2)]
    assert abs(math.log2(ratios[-1]) - 2.0) < 0.2, ratios


# ------------------------------------------------------------------------ equilibrium
def _gouy_chapman(y, V, lam):
    return 4.0 * np.arctanh(np.tanh(V / 4.0) * np.exp(-y / lam))


@pytest.mark.slow
def test_gouy_chapman_convergence():
    """Steady PNP with v = 0, zero flux at the bottom and sides: c+- = exp(-+phi) and
    Lambda^2 phi'' = sinh(phi), phi(0) = V  ->  tanh(phi/4) = tanh(V/4) exp(-y/Lambda)
    (domain = 20 Lambda, far-field correction ~ e^-20).  Error must fall at rate ~2."""
    lam, V = 0.05, 1.0
    errs = []
    for lev in [5, 6, 7]:
        oc = W.uniform_octants(2, lev)
        m = O.OracleMesh(oc)
        bc = W.equilibrium_bcs(2, V)
        p = O.Params(eps=lam, steady=True, bc_type=bc.types, bc_val=bc.values)
        U0 = np.zeros((m.n_nodes, 3)); U0[:, :2] = 1.0; U0[:, 2] = V * (1 - m.x[:, 1])
        res = O.newton(m, p, U0, rtol=1e-12, max_it=40)
        assert res.converged
        phi = res.U[:, 2]
        # x-invariance of the 1D solution
        for yv in np.unique(m.ijk[:, 1]):
            row = phi[m.ijk[:, 1] == yv]
            assert row.max() - row.min() < 1e-10
        ex = _gouy_chapman(m.x[:, 1], V, lam)
        errs.append(np.sqrt(np.mean((phi - ex) ** 2)))
        # Boltzmann relation c+ = exp(-phi) holds to discretisation accuracy
        assert np.max(np.abs(res.U[:, 0] * np.exp(phi) - 1.0)) < 0.05
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert abs(slopes[-1] - 2.0) < 0.25, (errs, slopes)


def test_newton_quadratic_on_equilibrium_config():
    """2D steady double layer, uniform level 5, Lambda = 0.01, V = 1 (the small
    equilibrium configuration): Newton reaches 1e-10 quickly, quadratically at the end."""
    m = O.OracleMesh(W.uniform_octants(2, 5))
    bc = W.equilibrium_bcs(2, 1.0)
    p = O.Params(eps=0.01, steady=True, bc_type=bc.types, bc_val=bc.values)
    U0 = np.zeros((m.n_nodes, 3)); U0[:, :2] = 1.0; U0[:, 2] = 1.0 - m.x[:, 1]
    res = O.newton(m, p, U0, rtol=1e-10, max_it=20, line_search=False)
    assert res.converged and res.iterations <= 6
    n = np.array(res.norms)
    # the last two reductions are (at least) quadratic
    for k in (-2, -1):
        assert n[k] <= 10.0 * n[k - 1] ** 2 / n[0]
    # the damped (backtracking) variant reaches the same state
    res2 = O.newton(m, p, U0, rtol=1e-10, max_it=40, line_search=True)
    assert res2.converged
    assert np.abs(res2.U - res.U).max() < 1e-8


def test_golden_boundary_table():
    """Boundary conditions of the electroconvection benchmark (Table tab:BC-AliMani)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "bc_electroconvection.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    bc = W.membrane_bcs(3, V=20.0, membrane_c_plus=2.0)
    face = {"top": 5, "bottom": 4}
    field = {"phi": 2, "c+": 0, "c-": 1}
    for wall, var, kind, val in rows:
        f, k = face[wall], field[var]
        if kind == "dirichlet":
            assert bc.types[f, k] == W.DIRICHLET and bc.values[f, k] == float(val.replace("V", "20"))
        else:
            assert bc.types[f, k] == W.NATURAL


def test_element_range_sums_reproduce_the_serial_oracle():
    """The element-range entry points (used to time the oracle across host threads on a
    sample of elements) add up, over a partition of the elements and run concurrently from
    several threads, to the serial residual and J V on every PDE row."""
    import threading
    oc = W.random_balanced_octants(3, 1, 4, 0.3, 17)
    m = O.OracleMesh(oc)
    bcs = W.membrane_bcs(3, 5.0, 2.0)
    p = O.Params(eps=0.05, dt=0.01, beta=(1.5, -2.0, 0.5), bc_type=bcs.types, bc_val=bcs.values)
    L = oc.max_level
    U, Uk, Ukm1 = (W.random_state(m.ijk, L, s) for s in (1, 2, 3))
    V = W.random_direction(m.ijk, L, 4)
    vel = W.random_velocity(m.ijk, L, 5, 0.5)
    F = m.residual(p, U, Uk, Ukm1, vel)
    JV = m.jv(p, U, V, Uk, Ukm1, vel)
    cuts = np.linspace(0, m.n_elem, 5).astype(int)
    parts = [(np.zeros((m.n_nodes, 3)), np.zeros((m.n_nodes, 3))) for _ in range(4)]

    def run(i):
        m.residual_elements(p, U, Uk, Ukm1, vel, cuts[i], cuts[i + 1], parts[i][0])
        m.jv_elements(p, U, V, Uk, Ukm1, vel, cuts[i], cuts[i + 1], parts[i][1])

    th = [threading.Thread(target=run, args=(i,)) for i in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    kind, _ = m.bc_rows(p)
    pde = (kind == 0) & (m.hanging[:, None] == 0)
    Fs = sum(a for a, _ in parts)
    Js = sum(b for _, b in parts)
    assert np.abs(Fs[pde] - F[pde]).max() <= 1e-13 * np.abs(F[pde]).max()
    assert np.abs(Js[pde] - JV[pde]).max() <= 1e-13 * np.abs(JV[pde]).max()
