"""GPU parity of the boundary flux (the terms of the boundary current of Sec. 5.2)
against the FP64 oracle: every face of octrees with hanging nodes, periodic sides
included, at seeded states.  Tolerance: 1e-12 of the largest flux magnitude."""
import numpy as np
import pytest

from paper_2301_05985_gb300 import workloads as W

from gpu_common import Pair

pytestmark = pytest.mark.gpu

CASES = [
    ("2d_octree", W.random_balanced_octants(2, 2, 5, 0.3, 12), W.membrane_bcs(2, 5.0, 2.0)),
    ("3d_octree", W.random_balanced_octants(3, 1, 4, 0.3, 12), W.membrane_bcs(3, 5.0, 2.0)),
    ("3d_band_periodic_xy", W.with_periodic(W.membrane_band_octants(3, 5, 0.1), 3), W.membrane_bcs(3, 20.0, 2.0)),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_boundary_flux_matches_oracle(case):
    _, oc, bcs = case
    P = Pair(oc, dict(eps=0.02, dt=0.01), bcs)
    U = W.random_state(P.mesh.ijk, oc.max_level, 7)
    Ud = P.dev(U)
    Uo = P.to_ora(U)
    for face in range(2 * oc.dim):
        got = P.ctx.boundary_flux(Ud, face)
        ref = P.om.boundary_flux(Uo, face)
        scale = max(np.abs(ref).max(), 1e-300)
        assert np.abs(got - ref).max() <= 1e-12 * scale, (face, got, ref)
    top = 2 * oc.dim - 1
    f = P.om.boundary_flux(Uo, top)
    assert abs(P.ctx.boundary_current(Ud, top) + (f[0] - f[1])) <= 1e-12 * np.abs(f).max()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_plane_average_matches_oracle(case):
    _, oc, bcs = case
    P = Pair(oc, dict(eps=0.02, dt=0.01), bcs)
    U = W.random_state(P.mesh.ijk, oc.max_level, 9)
    Ud, Uo = P.dev(U), P.to_ora(U)
    size = 1 << oc.max_level
    for axis in range(oc.dim):
        coords = np.unique(P.mesh.ijk[:, axis])
        if not (oc.periodic >> axis) & 1:
            assert coords[-1] == size
        for zl in coords:
            got = P.ctx.plane_average(Ud, axis, int(zl))
            ref = P.om.plane_integral(Uo, axis, int(zl))
            assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), (axis, zl)
    prof = P.ctx.averaged_profile(Ud, oc.dim - 1, np.unique(P.mesh.ijk[:, oc.dim - 1]))
    assert prof.shape[1] == 3 and np.all(np.isfinite(prof))
