"""Octree refinement to target levels with 2:1 balancing (pnp_mesh_create_refined), against
an independent pure-Python construction (paper_2301_05985_gb300.workloads.refine_and_balance:
split to the targets, then repeatedly split any leaf that has a face, edge or corner
neighbour two or more levels finer, found by sampling points).  Both must give the same
leaves: the coarsest balanced octree that meets the targets is unique."""
import numpy as np
import pytest

from paper_2301_05985_gb300 import workloads as W

from gpu_common import lib


def _leaves(anchors, levels):
    return sorted((tuple(int(v) for v in a), int(l)) for a, l in zip(anchors, levels))


def _check(oc, target):
    pnp = lib()
    mesh = pnp.Mesh(oc, target_levels=target)
    a, lv = mesh.elements()
    ref = W.refine_and_balance(oc, target)
    assert _leaves(a, lv) == _leaves(ref.anchors, ref.levels)
    # every octant reached its target
    s = 1 << oc.max_level
    for anc, l, t in zip(oc.anchors, oc.levels, target):
        inside = np.all((a >= anc) & (a < anc + (s >> l)), axis=1)
        assert inside.any() and lv[inside].min() >= t
    return mesh


@pytest.mark.parametrize("dim,seed", [(3, 1), (3, 4), (2, 2), (2, 9)])
def test_random_targets_match_python_balance(dim, seed):
    oc = W.random_balanced_octants(dim, 1, 5 if dim == 3 else 6, 0.25, seed)
    rng = np.random.default_rng(seed)
    target = oc.levels.astype(np.int64) + (rng.random(oc.n) < 0.08) * rng.integers(1, 3, oc.n)
    target = np.minimum(target, oc.max_level).astype(np.uint8)
    _check(oc, target)


def test_single_deep_octant_ripples_to_the_coarse_grid():
    """One level-2 octant refined to level 6 inside a uniform level-2 cube: the balance
    ripples outward one level per layer (face, edge and corner neighbours)."""
    oc = W.uniform_octants(3, 2, 6)
    target = oc.levels.copy()
    i = int(np.flatnonzero(np.all(oc.anchors == [16, 16, 0], axis=1))[0])
    target[i] = 6
    mesh = _check(oc, target)
    assert mesh.n_hanging > 0


def test_periodic_axes_balance_across_the_wrap():
    oc = W.with_periodic(W.uniform_octants(2, 2, 6), 1)
    target = oc.levels.copy()
    i = int(np.flatnonzero(np.all(oc.anchors == [0, 16], axis=1))[0])
    target[i] = 6  # at x = 0: the balance must reach the elements at x = 1 across the wrap
    mesh = _check(oc, target)
    a, lv = mesh.elements()
    assert lv[a[:, 0] == 64 - 16].max() >= 3  # refined across the identified faces


def test_no_targets_keeps_a_balanced_octree_and_balances_an_unbalanced_one():
    oc = W.membrane_band_octants(2, 5, 0.1)
    mesh = _check(oc, oc.levels.copy())
    assert mesh.n_elem == oc.n
    # an unbalanced octree (level 5 next to level 2) is balanced
    bad = W.layered_octants(3, [(5, 0.25), (2, 1.0)])
    mesh2 = _check(bad, bad.levels.copy())
    assert mesh2.n_elem > bad.n


def test_bad_input_is_rejected():
    pnp = lib()
    oc = W.uniform_octants(3, 2, 4)
    with pytest.raises(pnp.PnpError) as e:
        pnp.Mesh(oc, target_levels=np.full(oc.n, 5, np.uint8))
    assert e.value.code == pnp.PNP_ERR_ARG
    dup = W.Octants(3, 4, np.concatenate([oc.anchors, oc.anchors[:1]]), np.concatenate([oc.levels, oc.levels[:1]]))
    with pytest.raises(pnp.PnpError) as e:
        pnp.Mesh(dup, target_levels=dup.levels.copy())
    assert e.value.code == pnp.PNP_ERR_MESH
    # a coarse octant covering fine ones
    over = W.Octants(3, 4, np.concatenate([oc.anchors, [[0, 0, 0]]]).astype(np.int32),
                     np.concatenate([oc.levels, [1]]).astype(np.uint8))
    with pytest.raises(pnp.PnpError) as e:
        pnp.Mesh(over, target_levels=over.levels.copy())
    assert e.value.code == pnp.PNP_ERR_MESH
