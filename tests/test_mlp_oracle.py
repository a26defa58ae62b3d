"""Pins of the FP64 network oracle: central differences, special cases, closed forms."""
import math

import numpy as np
import pytest

import mlp_oracle as M


def test_gelu_closed_forms():
    z = np.array([-3.0, -1.0, 0.0, 0.5, 2.0])
    # Phi(z) from the complementary error function of the standard library
    Phi = np.array([0.5 * math.erfc(-v / math.sqrt(2)) for v in z])
    np.testing.assert_allclose(M.gelu(z), z * Phi, rtol=1e-14, atol=1e-15)
    assert M.gelu(np.array([0.0]))[0] == 0.0
    # derivative against a central difference of the closed form
    h = 1e-6
    fd = (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(M.gelu_prime(z), fd, rtol=1e-8, atol=1e-10)
    # limits: GELU ~ identity for large z, ~ 0 for very negative z
    assert abs(M.gelu(np.array([10.0]))[0] - 10.0) < 1e-12
    assert abs(M.gelu(np.array([-10.0]))[0]) < 1e-20


def test_backward_matches_central_differences():
    rng = np.random.default_rng(3)
    layers = (12, 9, 7, 5, 3)
    Ws, bs = M.init_params(1, layers)
    for b in bs:
        b += rng.normal(0, 0.1, b.shape)
    X = rng.normal(size=(11, 12))
    Y = rng.normal(size=(11, 3))
    gW, gb, _ = M.backward(Ws, bs, X, Y)
    h = 1e-6
    for l in range(len(Ws)):
        for (i, j) in [(0, 0), (layers[l] - 1, layers[l + 1] - 1), (layers[l] // 2, 1)]:
            Wp = [w.copy() for w in Ws]; Wp[l][i, j] += h
            Wm = [w.copy() for w in Ws]; Wm[l][i, j] -= h
            fd = (M.loss(Wp, bs, X, Y) - M.loss(Wm, bs, X, Y)) / (2 * h)
            assert abs(fd - gW[l][i, j]) < 1e-7 * max(1.0, abs(fd))
        for j in [0, layers[l + 1] - 1]:
            bp = [b.copy() for b in bs]; bp[l][j] += h
            bm = [b.copy() for b in bs]; bm[l][j] -= h
            fd = (M.loss(Ws, bp, X, Y) - M.loss(Ws, bm, X, Y)) / (2 * h)
            assert abs(fd - gb[l][j]) < 1e-7 * max(1.0, abs(fd))


def test_linear_special_case():
    """With every hidden layer driven far into GELU's linear regime the network is an affine
    map whose least-squares gradient is known in closed form."""
    rng = np.random.default_rng(5)
    layers = (4, 3, 3, 3, 2)
    Ws = [np.eye(4)[:, :3] * 1.0, np.eye(3), np.eye(3), rng.normal(size=(3, 2))]
    bs = [np.full(3, 50.0), np.zeros(3), np.zeros(3), np.zeros(2)]
    # with the +50 shift, GELU(z) = z to double precision, so out = (X[:, :3] + 50) W4
    X = rng.normal(size=(6, 4)) * 0.1
    Y = rng.normal(size=(6, 2))
    out, _, _ = M.forward(Ws, bs, X)
    Aff = X[:, :3] + 50.0
    np.testing.assert_allclose(out, Aff @ Ws[3], rtol=1e-13)
    gW, gb, _ = M.backward(Ws, bs, X, Y)
    np.testing.assert_allclose(gW[3], Aff.T @ (2 * (out - Y) / out.size), rtol=1e-10)


def test_adam_first_step_is_sign_times_lr():
    """Adam's bias-corrected first step moves every parameter by lr * g / (|g| + eps)."""
    Ws, bs = M.init_params(2, (5, 4, 4, 4, 3))
    rng = np.random.default_rng(9)
    X = rng.normal(size=(8, 5)); Y = rng.normal(size=(8, 3))
    gW, gb, _ = M.backward(Ws, bs, X, Y)
    W0 = [w.copy() for w in Ws]
    M.adam_step(Ws, bs, gW, gb, {}, lr=1e-3)
    for w0, w1, g in zip(W0, Ws, gW):
        np.testing.assert_allclose(w0 - w1, 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-6, atol=1e-12)


def test_adam_later_steps_closed_forms():
    """Adam's moments and bias correction beyond the first step.  With the same gradient g
    at every step, m_t = (1 - b1^t) g and v_t = (1 - b2^t) g^2 exactly, so the corrected
    moments are g and g^2 and every step moves a parameter by lr g / (|g| + eps).  With
    the gradients g, -g, 3g the moments follow the recurrences written out by hand.  A
    bias correction frozen at t = 1, moments not carried between steps, or swapped
    betas fail one of these."""
    b1, b2, lr, eps = 0.9, 0.999, 1e-2, 1e-8
    g = np.array([[0.5, -2.0], [1e-3, 4.0]])
    gb = np.array([-0.25])
    W = [np.zeros((2, 2))]
    b = [np.ones(1)]
    state = {}
    for t in range(1, 6):
        M.adam_step(W, b, [g], [gb], state, lr=lr, beta1=b1, beta2=b2, eps=eps)
        np.testing.assert_allclose(state["m"][0], (1 - b1**t) * g, rtol=1e-14)
        np.testing.assert_allclose(state["v"][0], (1 - b2**t) * g * g, rtol=1e-13)
        np.testing.assert_allclose(W[0], -t * lr * g / (np.abs(g) + eps), rtol=1e-12)
        np.testing.assert_allclose(b[0], 1.0 - t * lr * gb / (np.abs(gb) + eps), rtol=1e-12)
        assert state["t"] == t
    # a changing gradient: g1 = g, g2 = -g, g3 = 3 g
    W = [np.zeros((2, 2))]
    b = [np.zeros(1)]
    state = {}
    seq = [1.0, -1.0, 3.0]
    m = np.zeros((2, 2)); v = np.zeros((2, 2)); p = np.zeros((2, 2))
    for t, s in enumerate(seq, start=1):
        M.adam_step(W, b, [s * g], [s * gb], state, lr=lr, beta1=b1, beta2=b2, eps=eps)
        # by hand: t = 2 gives m = (1 - b1)(b1 - 1) g, v = (1 - b2)(b2 + 1) g^2
        m = b1 * m + (1 - b1) * s * g
        v = b2 * v + (1 - b2) * (s * g) ** 2
        p = p - lr * (m / (1 - b1**t)) / (np.sqrt(v / (1 - b2**t)) + eps)
        if t == 2:
            np.testing.assert_allclose(m, -(1 - b1) ** 2 * g, rtol=1e-14)
            np.testing.assert_allclose(v, (1 - b2 * b2) * g * g, rtol=1e-13)
        np.testing.assert_allclose(state["m"][0], m, rtol=1e-14)
        np.testing.assert_allclose(state["v"][0], v, rtol=1e-13)
        np.testing.assert_allclose(W[0], p, rtol=1e-12, atol=1e-15)
    # after g, -g the corrected first moment is -(1 - b1)^2 g / (1 - b1^2) = -(1 - b1)/(1 + b1) g
    st2 = {}
    W2, b2_ = [np.zeros((2, 2))], [np.zeros(1)]
    M.adam_step(W2, b2_, [g], [gb], st2, lr=lr, beta1=b1, beta2=b2, eps=eps)
    M.adam_step(W2, b2_, [-g], [-gb], st2, lr=lr, beta1=b1, beta2=b2, eps=eps)
    mh = st2["m"][0] / (1 - b1**2)
    np.testing.assert_allclose(mh, -(1 - b1) / (1 + b1) * g, rtol=1e-13)


@pytest.mark.parametrize("dim,seed", [(3, 2), (3, 7), (2, 4)])
def test_stencil_features_reproduce_linear_fields(dim, seed):
    """Point evaluation of the Q1 fields is exact for globally linear fields (on meshes with
    hanging nodes), the stencil spacing is the finest incident element, and points outside
    the domain are clamped to it."""
    import oracle as O
    from paper_2301_05985_gb300 import workloads as W
    oc = W.random_balanced_octants(dim, 1, 3 if dim == 3 else 4, 0.35, seed)
    m = O.OracleMesh(oc)
    a = np.array([[0.3, -1.2, 0.7], [1.1, 0.4, -0.9], [-0.5, 2.0, 0.25]])[:, :dim]
    U = 0.1 + m.x @ a.T
    uz = 0.2 - m.x[:, dim - 1]
    bc = W.all_natural_bcs(dim)
    p = O.Params(eps=0.1, steady=True, bc_type=bc.types, bc_val=bc.values)
    U = m.make_consistent(U, p)
    nodes, F = O.stencil_features(m, oc.levels, U, 2 * U, uz, -uz)
    npt = 3**dim
    hmin = m.node_sizes(oc.levels)
    size = 1 << m.max_level
    pts = np.clip(m.ijk[nodes][:, None, :] + hmin[nodes][:, None, None] * O.stencil_offsets(dim)[None], 0, size) / size
    for f in range(3):
        ref = 0.1 + pts @ a[f]
        np.testing.assert_allclose(F[:, f * npt:(f + 1) * npt], ref, atol=1e-14)
        np.testing.assert_allclose(F[:, (4 + f) * npt:(5 + f) * npt], 2 * ref, atol=1e-14)
    np.testing.assert_allclose(F[:, 3 * npt:4 * npt], 0.2 - pts[:, :, dim - 1], atol=1e-14)
    np.testing.assert_allclose(F[:, 7 * npt:8 * npt], -(0.2 - pts[:, :, dim - 1]), atol=1e-14)
    # the centre point is the node itself
    np.testing.assert_allclose(F[:, npt // 2], U[nodes, 0], atol=1e-15)
    # stencil spacing is the finest incident element: a node shared by a finest-level element
    finest = (1 << m.max_level) >> int(oc.levels.max())
    assert hmin.min() == finest


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2**-8, 1.0 + 3 * 2**-9, -2.5, 3.0e-5])
    r = M.bf16_round(x)
    assert r[0] == 1.0
    assert r[1] == 1.0          # tie rounds to even (1 + 2^-8 is halfway between 1 and 1 + 2^-7)
    assert r[2] == 1.0 + 2**-7  # above the halfway point
    assert r[3] == -2.5
    assert abs(r[4] - 3.0e-5) <= 3.0e-5 * 2**-8
