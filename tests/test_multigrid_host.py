"""Host-side multigrid pieces: the coarse octrees and the grid transfers.

The prolongation is checked against the oracle's own point evaluation of the coarse Q1
field (its std::map mesh and its constraint matrix, independent of the library's mesh
code) at every fine node: P x_c must equal the coarse field at the fine node points, on
octrees with hanging nodes on both levels.  Linear fields are reproduced exactly.  The
injection maps every coarse node to the fine node at the same point."""
import numpy as np
import pytest

import oracle as O
from paper_2301_05985_gb300 import workloads as W

from gpu_common import lib


def _csr_apply(ptr, col, w, x):
    out = np.zeros((ptr.size - 1,) + x.shape[1:])
    for i in range(ptr.size - 1):
        out[i] = (w[ptr[i]:ptr[i + 1], None] * x[col[ptr[i]:ptr[i + 1]]]).sum(axis=0)
    return out


@pytest.mark.parametrize("dim,seed", [(3, 5), (3, 8), (2, 3)])
def test_prolongation_is_the_coarse_field_at_fine_nodes(dim, seed):
    pnp = lib()
    oc = W.random_balanced_octants(dim, 1, 4 if dim == 3 else 6, 0.3, seed)
    fine = pnp.Mesh(oc)
    cap = int(oc.levels.max()) - 1
    coarse = fine.coarsen(cap)
    ca, cl = coarse.elements()
    assert cl.max() == cap and coarse.n_elem < fine.n_elem
    ptr, col, w, inj = fine.transfer(coarse)
    # columns are independent coarse nodes only
    assert not coarse.hanging[col].any()
    # the oracle's point evaluation of a coarse field at the fine node points
    om = O.OracleMesh(W.Octants(dim, coarse.max_level, ca, cl))
    rng = np.random.default_rng(seed)
    xc = rng.normal(size=(coarse.n_nodes, 3))
    bc = W.all_natural_bcs(dim)
    p = O.Params(eps=0.1, steady=True, bc_type=bc.types, bc_val=bc.values)
    # the coarse field in the oracle's node order, made conforming (hanging from parents)
    key = lambda a: sum(a[:, k].astype(np.int64) * (2 ** oc.max_level + 1) ** k for k in range(dim))  # noqa: E731
    ko, kl = key(om.ijk), key(coarse.ijk)
    order = np.argsort(kl)
    o2l = order[np.searchsorted(kl[order], ko)]
    xo = om.make_consistent(xc[o2l], p)
    xl = np.zeros_like(xc)
    xl[o2l] = xo
    ref = om.eval_points(xo, fine.ijk.astype(np.int64))
    got = _csr_apply(ptr, col, w.astype(np.float64), xl)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    # linear fields are reproduced exactly
    a = np.array([0.7, -1.3, 0.4])[:dim]
    lin_c = coarse.ijk @ a
    lin_f = fine.ijk @ a
    assert np.abs(_csr_apply(ptr, col, w.astype(np.float64), lin_c[:, None])[:, 0] - lin_f).max() <= 1e-9
    # injection: the same points
    assert np.array_equal(fine.ijk[inj], coarse.ijk)
    # weights sum to one on every row (partition of unity)
    sums = np.add.reduceat(w.astype(np.float64), ptr[:-1])
    assert np.allclose(sums, 1.0, atol=1e-7)


def test_coarsening_keeps_balance_down_to_a_uniform_grid():
    pnp = lib()
    oc = W.membrane_band_octants(3, 6, 0.1)
    m = pnp.Mesh(oc)
    for cap in (5, 4, 3, 2):
        c = m.coarsen(cap)  # pnp_mesh_create's 2:1 and cover checks run on it
        _, lv = c.elements()
        assert lv.max() == cap and lv.min() == min(cap, 3)
    assert m.coarsen(2).n_elem == 64
