"""GPU checks of the refinement indicator (pnp_element_gradient) and of the
solution-adaptive octree built from it.

The indicator is |grad u| of each Q1 field at the element centre.  For a globally linear
field it equals |a| on every element, hanging corners included (the constraints
reproduce linear fields); for u = x_k^2 sampled at the nodes of a uniform grid the
centre derivative along k is exactly 2 x_k at the centre.  Tolerance: 1e-12 relative.
"""
import numpy as np
import pytest

from paper_2301_05985_gb300 import workloads as W

from gpu_common import lib, torch_cuda

pytestmark = pytest.mark.gpu


def _ctx(oc):
    pnp, torch = lib(), torch_cuda()
    mesh = pnp.Mesh(oc)
    ctx = pnp.Context(mesh, pnp.default_params(eps=0.05, dt=0.01), torch.cuda.current_stream().cuda_stream)
    return pnp, torch, mesh, ctx


@pytest.mark.parametrize("dim,seed", [(3, 3), (2, 5)])
def test_gradient_of_linear_fields_is_exact_with_hanging_nodes(dim, seed):
    oc = W.random_balanced_octants(dim, 1, 5 if dim == 3 else 6, 0.3, seed)
    pnp, torch, mesh, ctx = _ctx(oc)
    assert mesh.n_hanging > 0
    x = mesh.ijk / float(1 << oc.max_level)
    a = np.array([[0.3, -1.2, 0.7], [1.1, 0.4, -0.9], [-0.5, 2.0, 0.25]])[:, :dim]
    U = 0.1 + x @ a.T
    # hanging entries hold garbage: the kernel must take them from the constraints
    U[mesh.hanging] = 1e6
    G = torch.zeros((mesh.n_elem, 3), dtype=torch.float64, device="cuda")
    ctx.element_gradient(torch.from_numpy(U).cuda(), G)
    G = G.cpu().numpy()
    ref = np.linalg.norm(a, axis=1)
    assert np.abs(G - ref[None, :]).max() <= 1e-12 * ref.max()


def test_gradient_of_quadratic_field_on_a_uniform_grid():
    oc = W.uniform_octants(3, 4)
    pnp, torch, mesh, ctx = _ctx(oc)
    x = mesh.ijk / float(1 << oc.max_level)
    U = np.stack([x[:, 0] ** 2, 0.5 * x[:, 1] ** 2, x[:, 2] ** 2 - x[:, 0] ** 2], axis=1)
    G = torch.zeros((mesh.n_elem, 3), dtype=torch.float64, device="cuda")
    ctx.element_gradient(torch.from_numpy(U).cuda(), G)
    G = G.cpu().numpy()
    anc, lev = mesh.elements()
    xc = (anc + 0.5 * (1 << (oc.max_level - lev))[:, None]) / float(1 << oc.max_level)
    ref = np.stack([2 * xc[:, 0], xc[:, 1], 2 * np.hypot(xc[:, 2], xc[:, 0])], axis=1)
    assert np.abs(G - ref).max() <= 1e-12 * np.abs(ref).max()


def test_gradient_refined_octree_is_balanced_and_refines_the_debye_layer():
    """The electroconvection recipe on a miniature (levels 3-6): the pre-solve's gradients
    are largest in the Debye layer at the membrane, so the finest level appears there and
    only there, and the refined octree passes the mesh's 2:1 and cover checks."""
    from paper_2301_05985_gb300 import refine as R
    pnp, torch = lib(), torch_cuda()
    rec = R.RefineRecipe(base=3, band_level=5, fine=6, band=0.1, theta=5.0, presolve_steps=2)
    oc, target, info = R.gradient_refined_octants(pnp, torch, torch.cuda.current_stream().cuda_stream, rec,
                                                  eps=0.02, volt=10.0, dt=1e-3)
    assert info["refined_by_gradient"] > 0
    mesh = pnp.Mesh(oc, target_levels=target)
    anc, lev = mesh.elements()
    z0 = anc[:, 2] / float(1 << oc.max_level)
    assert lev.max() == 6 and z0[lev == 6].max() < 0.1
    assert np.all(lev[z0 < 0.1] >= 5)
    assert mesh.n_elem > oc.n
