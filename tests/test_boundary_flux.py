"""Pins of the oracle's boundary flux, the terms of the boundary current of Sec. 5.2
(the net species flux through the top boundary): for fields linear in the face's normal
coordinate the Q1 interpolation is exact and the flux has a closed form on any 2:1 mesh,
hanging nodes included; an identified (periodic) face carries none."""
import numpy as np
import pytest

import oracle as O
from paper_2301_05985_gb300 import workloads as W


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("ax", [0, 1, 2])
def test_flux_of_linear_fields_is_exact(dim, ax):
    if ax >= dim:
        pytest.skip("axis beyond dim")
    oc = W.random_balanced_octants(dim, 2, 5 if dim == 2 else 4, 0.3, 12)
    om = O.OracleMesh(oc)
    assert om.n_hanging > 0
    x = om.ijk[:, ax].astype(np.float64) / (1 << oc.max_level)
    a, b, c0, c1, g0, g1 = 1.3, 0.7, 2.0, -0.5, 0.4, -2.5
    bcs = W.all_natural_bcs(dim)
    p = O.Params(eps=0.1, dt=0.1, bc_type=bcs.types, bc_val=bcs.values)
    U = om.make_consistent(np.stack([a + b * x, c0 + c1 * x, g0 + g1 * x], axis=1), p)
    # high face x_ax = 1, outward normal +e_ax; low face x_ax = 0, normal -e_ax
    hi = om.boundary_flux(U, 2 * ax + 1)
    lo = om.boundary_flux(U, 2 * ax)
    assert np.allclose(hi, [b + (a + b) * g1, c1 - (c0 + c1) * g1], rtol=1e-13, atol=0)
    assert np.allclose(lo, [-(b + a * g1), -(c1 - c0 * g1)], rtol=1e-13, atol=0)


def test_flux_scales_with_face_area_on_a_uniform_mesh():
    """A field linear in z on a uniform 3D grid: every top element contributes its area."""
    for lev in (2, 3):
        om = O.OracleMesh(W.uniform_octants(3, lev))
        z = om.ijk[:, 2].astype(np.float64) / (1 << lev)
        U = np.stack([1.0 + z, np.ones_like(z), np.zeros_like(z)], axis=1)
        assert np.allclose(om.boundary_flux(U, 5), [1.0, 0.0], atol=1e-14)


def test_flux_through_an_identified_face_is_zero():
    oc = W.random_balanced_octants(2, 2, 5, 0.3, 12, periodic=1)
    om = O.OracleMesh(oc)
    U = W.random_state(om.ijk, oc.max_level, 3)
    assert np.array_equal(om.boundary_flux(U, 0), [0.0, 0.0])
    assert np.array_equal(om.boundary_flux(U, 1), [0.0, 0.0])
    assert np.any(om.boundary_flux(U, 3) != 0.0)


# ------------------------------------------------------------------ plane averages
@pytest.mark.parametrize("dim", [2, 3])
def test_plane_average_of_linear_fields_is_exact(dim):
    """On every node level of a 2:1 octree (planes through element sides and through the
    middle of coarse elements), the plane average of a field linear in the normal
    coordinate is its value there, and of a field linear in a tangential coordinate the
    value at the middle."""
    oc = W.random_balanced_octants(dim, 2, 5 if dim == 2 else 4, 0.3, 12)
    om = O.OracleMesh(oc)
    L = oc.max_level
    size = 1 << L
    z = om.ijk[:, dim - 1].astype(np.float64) / size
    x = om.ijk[:, 0].astype(np.float64) / size
    bcs = W.all_natural_bcs(dim)
    p = O.Params(eps=0.1, dt=0.1, bc_type=bcs.types, bc_val=bcs.values)
    U = om.make_consistent(np.stack([1.3 + 0.7 * z, 2.0 - 0.5 * x, -1.0 + 3.0 * z], axis=1), p)
    levels = np.unique(om.ijk[:, dim - 1])
    assert len(levels) > (1 << 2) + 1  # finer levels than the base grid
    for zl in levels:
        zz = zl / size
        got = om.plane_integral(U, dim - 1, int(zl))
        assert np.allclose(got, [1.3 + 0.7 * zz, 2.0 - 0.25, -1.0 + 3.0 * zz], rtol=1e-13, atol=1e-13), zl


def test_plane_average_over_a_period():
    """sin(2 pi x) sampled on a uniform periodic grid: its Q1 interpolant averages to 0."""
    oc = W.with_periodic(W.uniform_octants(2, 4), 1)
    om = O.OracleMesh(oc)
    x = om.ijk[:, 0].astype(np.float64) / (1 << 4)
    U = np.stack([np.sin(2 * np.pi * x), 1.0 + np.cos(2 * np.pi * x), x * 0], axis=1)
    for yl in range(0, 17, 5):
        assert np.allclose(om.plane_integral(U, 1, yl), [0.0, 1.0, 0.0], atol=1e-14)
