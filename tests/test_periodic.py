"""Periodic side walls (the electroconvection setup of Sec. 5.2: the x sides of the cell
are periodic).  The oracle and the library identify the faces x_k = 0 and x_k = 1
independently; these CPU tests pin the oracle's periodic residual to what the
identification must satisfy, and check the library's host mesh build against it.

Pins:
- translation: on a periodic axis the domain has no origin, so shifting the octree and
  the state by a whole number of coarse cells along it shifts the residual with them;
- support: with a state and a refinement that depend on z only, every node of a z level
  has the same row (a face left unidentified would give its nodes half the support);
- conservation: zero flux on the non-periodic faces and v = 0 leave only the time
  derivative in the sum of the species rows, as in the non-periodic pin.
"""
import numpy as np
import pytest

import oracle as O
from paper_2301_05985_gb300 import workloads as W


@pytest.fixture(scope="module")
def pnp():
    from paper_2301_05985_gb300 import build as B
    B.build()
    from paper_2301_05985_gb300 import pnp as P
    return P


def _node_map(om):
    return {tuple(x): i for i, x in enumerate(om.ijk.tolist())}


@pytest.mark.parametrize("dim,base,top,frac,seed,mask", [(2, 2, 5, 0.3, 12, 1), (2, 2, 5, 0.3, 14, 3),
                                                          (3, 1, 3, 0.35, 2, 1), (3, 2, 4, 0.3, 12, 3)])
def test_periodic_mesh_builder_matches_oracle(pnp, dim, base, top, frac, seed, mask):
    oc = W.random_balanced_octants(dim, base, top, frac, seed, periodic=mask)
    m = pnp.Mesh(oc)
    om = O.OracleMesh(oc)
    assert (m.n_elem, m.n_nodes, m.n_hanging) == (om.n_elem, om.n_nodes, om.n_hanging)
    size = 1 << oc.max_level
    for k in range(dim):
        if (mask >> k) & 1:
            assert m.ijk[:, k].max() < size and om.ijk[:, k].max() < size  # x = 1 is x = 0
    a = {tuple(x): h for x, h in zip(m.ijk.tolist(), m.hanging)}
    b = {tuple(x): bool(h) for x, h in zip(om.ijk.tolist(), om.hanging)}
    assert a == b
    assert m.n_hanging > 0


def test_periodic_rejections_agree(pnp):
    """Octrees balanced only without the wrap: both builds reject exactly the same ones."""
    n_rej = 0
    for seed in range(10, 30):
        oc = W.with_periodic(W.random_balanced_octants(2, 2, 5, 0.3, seed), 1)
        try:
            O.OracleMesh(oc)
            ora_ok = True
        except ValueError:
            ora_ok = False
        try:
            pnp.Mesh(oc)
            lib_ok = True
        except pnp.PnpError as e:
            assert e.code == pnp.PNP_ERR_MESH_UNBALANCED
            lib_ok = False
        assert ora_ok == lib_ok, seed
        n_rej += not ora_ok
    assert 0 < n_rej < 20


def test_periodic_rejects_a_level_zero_axis(pnp):
    oc = W.with_periodic(W.uniform_octants(2, 0), 1)
    with pytest.raises(ValueError):
        O.OracleMesh(oc)
    with pytest.raises(pnp.PnpError):
        pnp.Mesh(oc)


def _params(bcs, dt=0.02):
    return O.Params(eps=0.05, dt=dt, beta=(1.5, -2.0, 0.5), bc_type=bcs.types, bc_val=bcs.values)


@pytest.mark.parametrize("dim,mask", [(2, 1), (3, 1), (3, 3)])
def test_periodic_residual_is_translation_invariant(dim, mask):
    base, top = (2, 5) if dim == 2 else (2, 4)
    oc = W.random_balanced_octants(dim, base, top, 0.3, 12, periodic=mask)
    L = oc.max_level
    size = 1 << L
    shift = np.zeros(dim, np.int64)
    shift[0] = 3 * (size >> base)  # three coarse cells along x
    oc2 = W.Octants(dim, L, ((oc.anchors + shift) % size).astype(np.int32), oc.levels.copy(), mask)
    m1, m2 = O.OracleMesh(oc), O.OracleMesh(oc2)
    bcs = W.membrane_bcs(dim, 4.0, 2.0)
    p = _params(bcs)
    U = m1.make_consistent(W.random_state(m1.ijk, L, 5), p)
    Uk = m1.make_consistent(W.random_state(m1.ijk, L, 6), p)
    Ukm1 = m1.make_consistent(W.random_state(m1.ijk, L, 7), p)
    vel = W.random_velocity(m1.ijk, L, 8, 0.5)
    # node i of mesh 1 sits at (x + shift) mod size in mesh 2
    at2 = _node_map(m2)

    def target(x):
        y = list(x)
        y[0] = (y[0] + int(shift[0])) % size
        return tuple(y)

    perm = np.array([at2[target(x)] for x in m1.ijk.tolist()])

    def moved(X):
        Y = np.zeros_like(X)
        Y[perm] = X
        return Y

    F1 = m1.residual(p, U, Uk, Ukm1, vel)
    F2 = m2.residual(p, moved(U), moved(Uk), moved(Ukm1), moved(vel))
    assert np.abs(F2[perm] - F1).max() <= 1e-12 * np.abs(F1).max()
    # the shift is not a symmetry of the non-periodic problem
    oc_np = W.with_periodic(oc, 0)
    oc2_np = W.with_periodic(oc2, 0)
    try:
        n1, n2 = O.OracleMesh(oc_np), O.OracleMesh(oc2_np)
    except ValueError:
        return  # not balanced without the wrap: nothing to contrast with
    G1 = n1.residual(p, n1.make_consistent(W.random_state(n1.ijk, L, 5), p))
    G2 = n2.residual(p, n2.make_consistent(W.random_state(n2.ijk, L, 5), p))
    assert G1.shape[0] != F1.shape[0]  # the sides are separate nodes there


@pytest.mark.parametrize("mask", [1, 3])
def test_periodic_support_with_z_only_state(mask):
    oc = W.with_periodic(W.membrane_band_octants(2, 4, 0.2), mask)
    om = O.OracleMesh(oc)
    L = oc.max_level
    bcs = W.membrane_bcs(3, 4.0, 2.0)
    p = _params(bcs)
    z = om.ijk[:, 2].astype(np.float64) / (1 << L)

    def zstate(a, b):
        U = np.stack([1.0 + a * np.sin(np.pi * z), 1.0 - b * np.cos(np.pi * z), 4.0 * (1 - z) + a * z * z], axis=1)
        return om.make_consistent(U, p)

    F = om.residual(p, zstate(0.3, 0.2), zstate(0.25, 0.1), zstate(0.2, 0.05))
    free = om.hanging == 0
    scale = np.abs(F).max()
    # rows may depend only on the coordinates of the non-periodic axes
    keep = [k for k in range(3) if not (mask >> k) & 1]
    groups = {}
    for i in np.nonzero(free)[0]:
        groups.setdefault(tuple(om.ijk[i, keep].tolist()), []).append(i)
    n_multi = 0
    for key, idx in groups.items():
        rows = F[idx]
        n_multi += len(idx) > 1
        assert np.abs(rows - rows[0]).max() <= 1e-12 * scale, key
    assert n_multi > 0


@pytest.mark.parametrize("dim,mask", [(2, 1), (3, 3)])
def test_periodic_discrete_conservation(dim, mask):
    oc = W.random_balanced_octants(dim, 1 if dim == 3 else 2, 3 if dim == 3 else 5, 0.35, 12, periodic=mask)
    m = O.OracleMesh(oc)
    bc = W.all_natural_bcs(dim)
    dt, beta = 0.1, (1.5, -2.0, 0.5)
    p = O.Params(eps=0.1, dt=dt, beta=beta, bc_type=bc.types, bc_val=bc.values)
    U = m.make_consistent(W.random_state(m.ijk, m.max_level, 3), p)
    Uk = m.make_consistent(W.random_state(m.ijk, m.max_level, 4), p)
    Ukm1 = m.make_consistent(W.random_state(m.ijk, m.max_level, 5), p)
    F = m.residual(p, U, Uk, Ukm1, None)
    free = m.hanging == 0
    vol = 0.5 ** (dim * np.array(oc.levels).astype(np.float64))
    for s in range(2):
        field = (beta[0] * U[:, s] + beta[1] * Uk[:, s] + beta[2] * Ukm1[:, s]) / dt
        integral = np.sum(vol * field[m.el_nodes].mean(axis=1))
        assert abs(F[free, s].sum() - integral) < 1e-12 * abs(integral)


def test_periodic_mask_is_validated(pnp):
    oc = W.uniform_octants(2, 2)
    for mask in (-1, 4, 8):
        with pytest.raises(pnp.PnpError) as e:
            pnp.Mesh(W.with_periodic(oc, mask))
        assert e.value.code == pnp.PNP_ERR_ARG
    # a periodic axis carries no boundary-face bits: no node of the mesh lies on x = 1
    m = pnp.Mesh(W.with_periodic(oc, 1))
    assert m.ijk[:, 0].max() == (1 << 2) - 1 and m.ijk[:, 1].max() == 1 << 2
