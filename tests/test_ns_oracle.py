"""Pins of the oracle's Navier-Stokes block (Def. 3, Sec. 3.1) against what the
mathematics fixes, independently of the oracle's own element loop:

* the element matrix of one cell against Kronecker products of the exact 1D Q1 mass,
  stiffness and convection matrices (the 2-point Gauss rule is exact for every term);
* hydrostatic balance: a constant charge in a linear potential gives a gradient body
  force, balanced exactly by a linear pressure with v = 0 (octrees with hanging nodes);
* uniform translation: a constant velocity on an all-periodic mesh is steady under
  BDF2 (the coefficients sum to zero) and the advection of a constant vanishes;
* second-order convergence of the steady manufactured solution of Eq. manufac_sol;
* the affine structure: F(X) - F(0) equals the assembled matrix times X.
"""
import numpy as np
import pytest

import oracle as O
from paper_2301_05985_gb300 import workloads as W

G = 1.0 / np.sqrt(3.0)


def _one_cell_ops(h):
    """Exact 1D matrices on [0, h]: mass, stiffness, C[a][b] = int N_a N_b'."""
    M1 = h / 6.0 * np.array([[2.0, 1.0], [1.0, 2.0]])
    K1 = 1.0 / h * np.array([[1.0, -1.0], [-1.0, 1.0]])
    C1 = np.array([[-0.5, 0.5], [-0.5, 0.5]])
    return M1, K1, C1


def _kron_element_matrix_2d(h, va, Sc, kap, tau_m, tau_s):
    """Element matrix of the NS rows, unknowns per node (v_x, v_y, v_z, p), node index
    c = x + 2 y, from Kronecker products (y-major) of the exact 1D matrices."""
    M1, K1, C1 = _one_cell_ops(h)
    kr = np.kron
    M = kr(M1, M1)
    D = [kr(M1, C1), kr(C1, M1)]                      # int N_a d_i N_b
    # E[i][j] = int d_i N_a d_j N_b; the y factor is the left one
    E = [[kr(M1, K1), kr(C1, C1.T)], [kr(C1.T, C1), kr(K1, M1)]]
    K = E[0][0] + E[1][1]
    A = va[0] * D[0] + va[1] * D[1]                   # int N_a v.grad N_b
    B = sum(va[j] * va[k] * E[j][k] for j in range(2) for k in range(2))  # int (v.grad N_a)(v.grad N_b)
    isc = 1.0 / Sc
    Kmat = np.zeros((16, 16))

    def put(fi, fj, blk):
        Kmat[fi::4, fj::4] += blk

    for i in range(2):
        # Galerkin N_a R_m,i + viscous + SUPG (1/Sc) tau_m (v.grad N_a) R_m,i
        put(i, i, isc * kap * M + isc * A + K + isc * tau_m * (isc * kap * A.T + isc * B))
        put(i, 3, D[i] + isc * tau_m * sum(va[j] * E[j][i] for j in range(2)))
        # grad-div: tau_sol (d_i N_a)(div v)
        for k in range(2):
            put(i, k, tau_s * E[i][k])
        # solenoidality: N_a div v + tau_m grad N_a . R_m
        put(3, i, D[i] + tau_m * isc * (kap * D[i].T + sum(va[j] * E[i][j] for j in range(2))))
    put(3, 3, tau_m * K)
    return Kmat


def test_one_cell_matrix_matches_kronecker_products():
    h = 1.0
    oc = W.uniform_octants(2, 0)
    mesh = O.OracleMesh(oc)
    assert mesh.n_elem == 1 and mesh.n_nodes == 4
    Sc, dt, C_I = 2.5, 0.1, 6.0
    beta = (1.5, -2.0, 0.5)
    va = np.array([0.7, -0.4])
    p = O.NsParams(Sc=Sc, kappa=0.3, eps=0.2, dt=dt, beta=beta, C_I=C_I, pin=False)
    adv = np.tile(np.array([va[0], va[1], 0.0]), (4, 1))
    A = mesh.ns_matrix(p, adv).toarray()
    # oracle node order -> c = x + 2 y
    perm = np.argsort(mesh.ijk[:, 0] + 2 * mesh.ijk[:, 1])
    idx = (4 * perm[:, None] + np.arange(4)[None, :]).reshape(-1)
    A = A[np.ix_(idx, idx)]
    G2 = (2.0 / h) ** 2
    tau_m = (4.0 / dt**2 + G2 * va @ va + C_I * Sc**2 * 2 * G2 * G2) ** -0.5
    tau_s = 1.0 / (2 * G2 * tau_m)
    ref = _kron_element_matrix_2d(h, va, Sc, beta[0] / dt, tau_m, tau_s)
    rows = [r for r in range(16) if r % 4 != 2]      # slot 2 is inactive in 2D (identity rows)
    np.testing.assert_allclose(A[np.ix_(rows, rows)], ref[np.ix_(rows, rows)], rtol=1e-13, atol=1e-13)
    # without the fine scales the matrix is the plain Galerkin one
    p0 = O.NsParams(Sc=Sc, kappa=0.3, eps=0.2, dt=dt, beta=beta, C_I=C_I, pin=False, vms=False)
    A0 = mesh.ns_matrix(p0, adv).toarray()[np.ix_(idx, idx)]
    ref0 = _kron_element_matrix_2d(h, va, Sc, beta[0] / dt, 0.0, 0.0)
    np.testing.assert_allclose(A0[np.ix_(rows, rows)], ref0[np.ix_(rows, rows)], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("dim,seed", [(2, 1), (3, 2)])
def test_hydrostatic_balance_is_exact_on_octrees(dim, seed):
    oc = W.random_balanced_octants(dim, 2, 5 if dim == 2 else 4, 0.35, seed)
    mesh = O.OracleMesh(oc)
    assert mesh.n_hanging > 0
    rho0, gvec = 0.8, np.array([0.3, -1.1, 0.6])[:dim]
    kappa, eps = 0.5, 0.25
    U = np.zeros((mesh.n_nodes, 3))
    U[:, 0] = 1.0 + 0.5 * rho0
    U[:, 1] = 1.0 - 0.5 * rho0
    U[:, 2] = mesh.x @ gvec                        # phi linear: grad phi = g
    bt, bv = O.no_slip_bcs(dim)
    p = O.NsParams(Sc=1.0, kappa=kappa, eps=eps, dt=1e-2, beta=(1.5, -2.0, 0.5), bc_type=bt, bc_val=bv)
    rng = np.random.default_rng(seed)
    adv = 0.3 * rng.standard_normal((mesh.n_nodes, 3))   # any advection: v = 0 is not moved
    X = mesh.ns_solve(p, adv, None, None, U)
    fb = kappa / (2.0 * eps**2)
    p_exact = -fb * rho0 * (mesh.x @ gvec)          # grad p = -body force, p(origin) = 0
    np.testing.assert_allclose(X[:, :3], 0.0, atol=1e-10 * fb)
    np.testing.assert_allclose(X[:, 3], p_exact, atol=1e-10 * fb)


def test_uniform_translation_is_steady_under_bdf2():
    oc = W.with_periodic(W.uniform_octants(3, 3), 7)
    mesh = O.OracleMesh(oc)
    U0 = np.array([0.4, -0.2, 0.9])
    V = np.tile(U0, (mesh.n_nodes, 1))
    p = O.NsParams(Sc=0.7, kappa=0.5, eps=0.3, dt=5e-3, beta=(1.5, -2.0, 0.5), bc_type=np.zeros((6, 4), np.int32),
                   bc_val=np.zeros((6, 4)))
    U = np.ones((mesh.n_nodes, 3))   # neutral: no body force
    X = mesh.ns_solve(p, 2 * V - V, V, V, U)
    # rounding: the BDF mass coefficient 1.5 / (Sc dt) ~ 430 multiplies entries of size 1
    np.testing.assert_allclose(X[:, :3], V, atol=1e-12)
    np.testing.assert_allclose(X[:, 3], 0.0, atol=1e-9)
    # a BDF2 step from a history with a jump is not steady (the history terms enter)
    X2 = mesh.ns_solve(p, V, V, 0.5 * V, U)
    assert np.abs(X2[:, :3] - V).max() > 1e-3


def _mms_error(level, Sc=1.0, kappa=0.5, eps=0.5):
    oc = W.uniform_octants(2, level)
    mesh = O.OracleMesh(oc)
    bt = np.ones((4, 4), np.int32)
    bt[:, 3] = 0
    p = O.NsParams(Sc=Sc, kappa=kappa, eps=eps, steady=True, mms=True, pin=True, bc_type=bt,
                   bc_val=np.zeros((4, 4)))
    vals, _ = O.ns_mms_eval(p, 2, 0.0, mesh.x)
    pnp_vals, _ = O.mms_eval(2, eps, 0.0, True, mesh.x)
    p.pin_val = float(vals[np.argmin(mesh.ijk.sum(axis=1)), 3])
    adv = np.zeros((mesh.n_nodes, 3)); adv[:, :2] = vals[:, :2]
    X = mesh.ns_solve(p, adv, None, None, pnp_vals[:, :3])
    h = 1.0 / (1 << level)
    ev = np.sqrt(h**2 * np.sum((X[:, :2] - vals[:, :2]) ** 2))
    ep = np.sqrt(h**2 * np.sum((X[:, 3] - vals[:, 3]) ** 2))
    return ev, ep


def test_manufactured_solution_converges_at_second_order():
    errs = [_mms_error(l) for l in (3, 4, 5)]
    ev = np.array([e[0] for e in errs]); ep = np.array([e[1] for e in errs])
    rv = np.log2(ev[:-1] / ev[1:])
    assert np.all(rv > 1.8), (ev, rv)
    # the pressure converges too (equal-order pairs with residual-based stabilisation)
    assert ep[-1] < 0.5 * ep[0], ep


def test_residual_is_affine_with_the_assembled_matrix():
    oc = W.random_balanced_octants(3, 2, 4, 0.35, 5)
    mesh = O.OracleMesh(oc)
    rng = np.random.default_rng(0)
    n = mesh.n_nodes
    bt, bv = O.no_slip_bcs(3, walls=(4, 5))
    bv[5, 0] = 0.3
    p = O.NsParams(Sc=2.0, kappa=0.5, eps=0.3, dt=1e-2, beta=(1.5, -2.0, 0.5), bc_type=bt, bc_val=bv)
    adv, Vk, Vkm1 = (0.2 * rng.standard_normal((n, 3)) for _ in range(3))
    U = 1.0 + 0.1 * rng.standard_normal((n, 3))
    X = rng.standard_normal((n, 4))
    F = mesh.ns_apply(p, X, adv, Vk, Vkm1, U, with_data=True)
    F0 = mesh.ns_apply(p, None, adv, Vk, Vkm1, U, with_data=True)
    AX = mesh.ns_apply(p, X, adv, Vk, Vkm1, U, with_data=False)
    A = mesh.ns_matrix(p, adv)
    np.testing.assert_allclose(AX.reshape(-1), A @ X.reshape(-1), rtol=1e-12, atol=1e-12 * np.abs(AX).max())
    np.testing.assert_allclose(F - F0, AX, rtol=1e-11, atol=1e-11 * np.abs(AX).max())


def test_element_range_sums_reproduce_the_serial_ns_rows():
    """The element-range entry point the CPU baseline times across threads adds up, over a
    partition of the elements, to the serial rows (PDE rows; the others are set apart)."""
    oc = W.random_balanced_octants(3, 2, 4, 0.3, 5)
    mesh = O.OracleMesh(oc)
    rng = np.random.default_rng(1)
    n = mesh.n_nodes
    bt, bv = O.no_slip_bcs(3)
    p = O.NsParams(Sc=1.3, kappa=0.5, eps=0.2, dt=1e-2, beta=(1.5, -2.0, 0.5), bc_type=bt, bc_val=bv)
    X, a, vk, vkm1 = (rng.standard_normal((n, k)) for k in (4, 3, 3, 3))
    U = 1.0 + 0.1 * rng.standard_normal((n, 3))
    kind, _ = mesh.ns_bc_rows(p)
    for data in (True, False):
        F = np.zeros((n, 4))
        cuts = [0, 37, 300, mesh.n_elem]
        for i in range(3):
            mesh.ns_apply_elements(p, X, a, vk, vkm1, U, data, cuts[i], cuts[i + 1], F)
        G = mesh.ns_apply(p, X, a, vk, vkm1, U, with_data=data)
        np.testing.assert_allclose(F[kind == 0], G[kind == 0], rtol=0, atol=1e-12 * np.abs(G).max())
