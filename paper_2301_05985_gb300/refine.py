"""Solution-adaptive octree for the 3D electroconvection workload (the paper's Sec. 5.2
refines near the ion-selective surface and where the concentration varies fastest).

Orchestration only: every step runs in the library (a PNP pre-solve through
``pnp_time_step``, the element gradients through ``pnp_element_gradient``, refinement and
2:1 balance through ``pnp_mesh_create_refined``); this module chooses the target level of
each octant from those results.

Recipe (stated with the workload):
1. pre-solve mesh: base level ``base`` everywhere, level ``band_level - 1`` for octants with
   z_min < ``band``, 2:1 graded (``workloads.membrane_band_octants``);
2. ``presolve_steps`` BDF steps of the PNP block from the seeded initial state with the
   workload's physics (mixed-precision Newton);
3. targets: level ``band_level`` for every octant with z_min < ``band``; level ``fine`` for
   every octant whose max(|grad c+|, |grad c-|) at its centre exceeds ``theta``;
4. refine to the targets and 2:1 balance.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import workloads as W


@dataclasses.dataclass
class RefineRecipe:
    base: int = 6
    band_level: int = 9
    fine: int = 10
    band: float = 0.01
    theta: float = 60.0
    presolve_steps: int = 3


def gradient_refined_octants(pnp, torch, stream: int, recipe: RefineRecipe, eps: float, volt: float, dt: float,
                             membrane_c_plus: float = 2.0, seed: int = 0, amp: float = 1e-3):
    """Octants of the solution-adaptive octree (max level ``recipe.fine``) and a summary."""
    r = recipe
    oc0 = W.membrane_band_octants(r.base, r.band_level - 1, r.band)
    mesh0 = pnp.Mesh(oc0)
    p = pnp.default_params(eps=eps, dt=dt, precision=pnp.PNP_F32, start_mode=pnp.PNP_START_EXTRAPOLATE,
                           newton_rtol=1e-8, gmres_restart=60, gmres_max_it=3000, dt_retries=2, gmres_inner=24)
    ctx0 = pnp.Context(mesh0, p, stream)
    ctx0.set_bcs(W.membrane_bcs(3, volt, membrane_c_plus))
    ctx0.set_field(pnp.PNP_FIELD_U, W.noisy_state(mesh0.ijk, oc0.max_level, seed=seed, amp=amp, phi_bottom=0.0,
                                                  phi_top=volt))
    ctx0.make_consistent()
    ctx0.reset_history()
    its = []
    for _ in range(r.presolve_steps):
        its.append(ctx0.time_step().newton_its)
    U = torch.empty((mesh0.n_nodes, 3), dtype=torch.float64, device="cuda")
    ctx0.get_field(pnp.PNP_FIELD_U, U, pnp.PNP_DEVICE)
    G = torch.empty((mesh0.n_elem, 3), dtype=torch.float64, device="cuda")
    ctx0.element_gradient(U, G)
    g = torch.maximum(G[:, 0], G[:, 1]).cpu().numpy()
    anchors, levels = mesh0.elements()
    ctx0.close()
    mesh0.close()
    shift = r.fine - oc0.max_level
    anchors = anchors.astype(np.int64) << shift
    zmin = anchors[:, 2] / float(1 << r.fine)
    target = levels.astype(np.int64)
    target[zmin < r.band] = np.maximum(target[zmin < r.band], r.band_level)
    target[g > r.theta] = r.fine
    oc = W.Octants(3, r.fine, anchors.astype(np.int32), levels.astype(np.uint8))
    info = {"presolve_mesh": {"n_elem": int(levels.size), "levels": [int(levels.min()), int(levels.max())]},
            "presolve_newton_its": its, "refined_by_gradient": int((g > r.theta).sum()),
            "grad_max": float(g.max())}
    return oc, target.astype(np.uint8), info
