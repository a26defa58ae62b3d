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
