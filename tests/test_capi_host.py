"""Host-side checks of the C-ABI library (no GPU needed).

* the shared library builds, loads, and exports every function ``include/pnp.h``
  declares;
* the library's host mesh builder (pure host code) agrees with the oracle's
  independent construction: same nodes, same hanging nodes with the same parents,
  same rejections of unbalanced or overlapping octants.
"""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_2301_05985_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pnp():
    from paper_2301_05985_gb300 import build as B
    B.build()
    from paper_2301_05985_gb300 import pnp as P
    return P


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", fn)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        txt = re.sub(r"//[^\n]*", "", txt)
        for m in re.finditer(r"\b(pnp_[a-z0-9_]+)\s*\(", txt):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol(pnp):
    names = _declared_functions()
    assert "pnp_jv" in names and "pnp_residual" in names
    L = C.CDLL(pnp.LIB_PATH)
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", pnp.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (pnp_[a-z0-9_]+)", out))
    assert names <= exported, names - exported
    # every declared symbol has a Python signature in the binding
    assert names <= set(pnp.SIGNATURES), names - set(pnp.SIGNATURES)


def test_struct_layouts_match_header(pnp, tmp_path):
    """Field offsets of the ctypes mirrors equal those the C compiler gives the header."""
    p = pnp.default_params()
    assert p.C_I == 6.0 and p.gmres_restart == 30 and p.newton_rtol == 1e-8
    structs = (("pnp_params", pnp.pnp_params), ("pnp_solve_stats", pnp.pnp_solve_stats),
               ("pnp_ns_stats", pnp.pnp_ns_stats), ("pnp_train_cfg", pnp.pnp_train_cfg),
               ("pnp_train_stats", pnp.pnp_train_stats))
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pnp.h"', 'int main(void){',
             'printf("PNP_MLP_PARAMS size %d\\n", PNP_MLP_PARAMS);']
    for cname, py in structs:
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    want = {}
    for ln in out:
        if ln:
            s, f, v = ln.split()
            want[(s, f)] = int(v)
    assert want[("PNP_MLP_PARAMS", "size")] == pnp.PNP_MLP_PARAMS
    for cname, py in structs:
        assert C.sizeof(py) == want[(cname, "size")]
        for f, _ in py._fields_:
            assert getattr(py, f).offset == want[(cname, f)], (cname, f)


def _mesh_pair(pnp, oc):
    m = pnp.Mesh(oc)
    om = O.OracleMesh(oc)
    return m, om


@pytest.mark.parametrize("dim,base,top,frac,seed", [(2, 1, 4, 0.35, 1), (2, 2, 5, 0.3, 7), (3, 1, 3, 0.35, 2),
                                                     (3, 1, 3, 0.5, 5)])
def test_mesh_builder_matches_oracle(pnp, dim, base, top, frac, seed):
    oc = W.random_balanced_octants(dim, base, top, frac, seed)
    m, om = _mesh_pair(pnp, oc)
    assert (m.n_elem, m.n_nodes, m.n_hanging) == (om.n_elem, om.n_nodes, om.n_hanging)
    a = {tuple(x): h for x, h in zip(m.ijk.tolist(), m.hanging)}
    b = {tuple(x): bool(h) for x, h in zip(om.ijk.tolist(), om.hanging)}
    assert a == b
    # element set equal, library order is Morton order (sorted interleaved bits)
    anc, lev = m.elements()
    assert sorted(zip(map(tuple, anc.tolist()), lev.tolist())) == sorted(
        zip(map(tuple, oc.anchors.tolist()), oc.levels.tolist()))


def test_mesh_builder_node_order_is_morton(pnp):
    m = pnp.Mesh(W.uniform_octants(3, 3))

    def key(p):
        k = 0
        for bit in range(8):
            for a in range(3):
                k |= ((p[a] >> bit) & 1) << (3 * bit + a)
        return k

    keys = [key(p) for p in m.ijk.tolist()]
    assert keys == sorted(keys)


def test_mesh_builder_rejections(pnp):
    L = 3
    anchors = [(0, 4), (4, 4), (4, 0)] + [(i, j) for i in range(4) for j in range(4)]
    levels = [1, 1, 1] + [3] * 16
    with pytest.raises(pnp.PnpError) as e:
        pnp.Mesh(W.Octants(2, L, np.array(anchors, np.int32), np.array(levels, np.uint8)))
    assert e.value.code == pnp.PNP_ERR_MESH_UNBALANCED
    with pytest.raises(O.__class__ if False else ValueError):
        O.OracleMesh(W.Octants(2, L, np.array(anchors, np.int32), np.array(levels, np.uint8)))
    # corner-only 2-level jump in 3D (edge/corner balance)
    L = 3
    oc = W.uniform_octants(3, 1, L)
    keep = [i for i in range(oc.n) if tuple(oc.anchors[i]) != (0, 0, 0)]
    a = [tuple(oc.anchors[i]) for i in keep]
    lv = [1] * len(a)
    # refine octant (0,0,0) of level 1 into level 2, then its far corner child into level 3
    for c in range(8):
        ch = tuple(2 * ((c >> k) & 1) for k in range(3))
        if ch == (2, 2, 2):
            for cc in range(8):
                a.append(tuple(2 + ((cc >> k) & 1) for k in range(3)))
                lv.append(3)
        else:
            a.append(ch)
            lv.append(2)
    with pytest.raises(pnp.PnpError) as e:
        pnp.Mesh(W.Octants(3, L, np.array(a, np.int32), np.array(lv, np.uint8)))
    assert e.value.code == pnp.PNP_ERR_MESH_UNBALANCED
    # gap / overlap / misalignment
    oc = W.uniform_octants(2, 2)
    with pytest.raises(pnp.PnpError) as e:
        pnp.Mesh(W.Octants(2, 2, oc.anchors[1:].copy(), oc.levels[1:].copy()))
    assert e.value.code == pnp.PNP_ERR_MESH
    bad = oc.anchors.copy(); bad[0] = (1, 0)
    with pytest.raises(pnp.PnpError) as e:
        pnp.Mesh(W.Octants(2, 2, bad, oc.levels.copy()))
    assert e.value.code == pnp.PNP_ERR_MESH
    with pytest.raises(pnp.PnpError) as e:
        pnp.Mesh(W.Octants(4, 2, oc.anchors, oc.levels))
    assert e.value.code == pnp.PNP_ERR_ARG


@pytest.mark.parametrize("dim,base,top,frac,seed", [(3, 1, 4, 0.3, 12), (3, 2, 4, 0.5, 5), (2, 2, 5, 0.3, 11),
                                                     (3, 3, 3, 0.0, 0)])
def test_patch_layout_invariants(pnp, dim, base, top, frac, seed):
    """Morton patches of the shared-memory kernels: every element slot maps to its target
    node, elements of one colour share no target, every non-hanging node is covered and
    hanging nodes are not, and the partial-row count matches the shared coverage."""
    oc = W.random_balanced_octants(dim, base, top, frac, seed)
    s = pnp.Mesh(oc).patch_stats()
    assert s["violations"] == 0, s
    assert s["max_nodes"] <= 640 and s["max_colors"] <= 64


def test_membrane_band_mesh_counts(pnp):
    """The 3D near-membrane band mesh (base level 5, level 8 for z_min < 0.05, graded)."""
    oc = W.membrane_band_octants(5, 8, 0.05)
    levels, counts = np.unique(oc.levels, return_counts=True)
    assert dict(zip(levels.tolist(), counts.tolist())) == {8: 256 * 256 * 14, 7: 128 * 128, 6: 64 * 64 * 2,
                                                            5: 32 * 32 * 29}
    m = pnp.Mesh(oc)
    assert m.n_elem == 971776
    assert m.n_nodes == 257 * 257 * 15 + 129 * 129 + 2 * 65 * 65 + 33 * 33 * 29
    # hanging: level-8 nodes on z = 14/256 not on the level-7 lattice, etc.
    assert m.n_hanging == (257**2 - 129**2) + (129**2 - 65**2) + (65**2 - 33**2)


@pytest.mark.parametrize("field,value", [
    ("eps", 0.0), ("dt", -1.0), ("gmres_restart", 0), ("gmres_restart", 201), ("precision", 7),
    ("bdf_order", 3), ("mg_omega", 2.5), ("ns_blocks", 0), ("ns_blocks", 17), ("ns_Sc", 0.0),
    ("ns_rtol", -1.0), ("ns_inner_rtol", 1.0), ("ns_max_it", 0), ("ns_pin", 2), ("ns_mg_levels", 17),
    ("ns_inner_max_it", 0), ("ns_fgmres", -1), ("ns_fgmres", 201)])
def test_context_rejects_out_of_range_params(pnp, field, value):
    """Parameter checks run before any device call: no GPU is needed to see them fail."""
    mesh = pnp.Mesh(W.uniform_octants(3, 2))
    p = pnp.default_params(eps=1e-2, dt=1e-3)
    setattr(p, field, value)
    with pytest.raises(pnp.PnpError) as e:
        pnp.Context(mesh, p)
    assert e.value.code == pnp.PNP_ERR_ARG
    mesh.close()
