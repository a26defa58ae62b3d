"""Seeded synthetic inputs: octree meshes, boundary conditions, initial states, velocity.

This module is the only code shared by the CUDA path's tests/benchmark and the CPU
oracle's tests.  It holds none of the method's arithmetic (no residual, no
quadrature, no Jacobian): only octant lists, boundary-condition tables, and
pseudo-random fields evaluated at integer node coordinates.

Conventions
-----------
* The domain is the unit square/cube.  Octants are given by integer anchors in
  units of ``2**-max_level`` and a refinement level ``l`` (edge ``2**-l``).
* Node coordinates are integers in the same units (0 .. 2**max_level).
* Face numbering: ``2*axis + side`` (x-=0, x+=1, y-=2, y+=3, z-=4, z+=5).
* Field numbering: c+ = 0, c- = 1, phi = 2.
* Random values come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
  pseudorandom number generators", OOPSLA 2014) keyed by the seed, the field and
  the node's coordinates at a fixed 2**-20 resolution, so that a node gets the same
  value whatever the mesh numbering or max_level.
"""
from __future__ import annotations

import dataclasses
import numpy as np

C_PLUS, C_MINUS, PHI = 0, 1, 2
NATURAL, DIRICHLET = 0, 1

_MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)


# ----------------------------------------------------------------------------- octants
@dataclasses.dataclass
class Octants:
    dim: int
    max_level: int
    anchors: np.ndarray  # int32 [n, dim]
    levels: np.ndarray   # uint8 [n]
    periodic: int = 0    # bit k: axis k periodic (faces x_k = 0 and 1 identified)

    @property
    def n(self) -> int:
        return int(self.levels.shape[0])


def uniform_octants(dim: int, level: int, max_level: int | None = None) -> Octants:
    """All octants of a uniform level-``level`` grid of the unit square/cube."""
    L = level if max_level is None else max_level
    n1 = 1 << level
    s = 1 << (L - level)
    axes = [np.arange(n1, dtype=np.int64) * s] * dim
    grid = np.meshgrid(*axes, indexing="ij")
    anchors = np.stack([g.reshape(-1) for g in grid], axis=1).astype(np.int32)
    levels = np.full(anchors.shape[0], level, dtype=np.uint8)
    return Octants(dim, L, anchors, levels)


def layered_octants(dim: int, layers: list[tuple[int, float]]) -> Octants:
    """Octree graded in the last coordinate: ``layers`` = [(level, top), ...] bottom-up.

    Layer ``i`` fills ``[top_{i-1}, top_i)`` of the last axis with uniform octants of
    its level; every layer boundary must be aligned to both adjacent levels.  This
    describes a near-membrane refined band with 2:1 grading above it.
    """
    L = max(l for l, _ in layers)
    size = 1 << L
    out_a, out_l = [], []
    z0 = 0
    for level, top in layers:
        s = 1 << (L - level)
        z1 = int(round(top * size))
        if z0 % s or z1 % s or z1 <= z0:
            raise ValueError(f"layer top {top} not aligned to level {level}")
        n1 = 1 << level
        lat = [np.arange(n1, dtype=np.int64) * s] * (dim - 1)
        zs = np.arange(z0, z1, s, dtype=np.int64)
        grid = np.meshgrid(*lat, zs, indexing="ij")
        out_a.append(np.stack([g.reshape(-1) for g in grid], axis=1))
        out_l.append(np.full(out_a[-1].shape[0], level, dtype=np.uint8))
        z0 = z1
    if z0 != size:
        raise ValueError("layers do not reach the top of the domain")
    return Octants(dim, L, np.concatenate(out_a).astype(np.int32), np.concatenate(out_l))


def membrane_band_octants(base_level: int = 5, fine_level: int = 8, band: float = 0.05) -> Octants:
    """3D unit cube, base level everywhere, ``fine_level`` for octants whose z_min < band.

    The fine band is extended upward to the next level-(fine-1) boundary and graded
    one level per layer (each intermediate layer thick enough to be aligned to the
    next coarser level), which is the smallest 2:1-balanced octree containing the
    requested refinement.
    """
    L = fine_level
    size = 1 << L
    s = 1
    # smallest multiple of the fine size strictly covering every fine octant with z_min < band
    top = 0
    while top / size < band:
        top += s
    layers = []
    level = fine_level
    while level > base_level:
        coarser = 1 << (L - level + 1)
        top = -(-top // coarser) * coarser  # align to the next coarser level
        layers.append((level, top / size))
        level -= 1
        top += 1 << (L - level)  # at least one octant of the next level
    layers.append((base_level, 1.0))
    # merge consecutive identical levels
    return layered_octants(3, layers)


def with_periodic(oc: Octants, periodic: int) -> Octants:
    """The same octants with periodic axes (bit k: axis k)."""
    return dataclasses.replace(oc, periodic=int(periodic))


def _children(a, l, dim, L):
    s = 1 << (L - l - 1)
    for c in range(1 << dim):
        yield tuple(a[k] + (s if (c >> k) & 1 else 0) for k in range(dim)), l + 1


def balance_leaves(leaves: dict, dim: int, L: int, periodic: int = 0) -> dict:
    """Split leaves ({anchor tuple: level}, modified in place) until no leaf has a face,
    edge or corner neighbour two or more levels finer.  Neighbours are found by sampling
    the points just outside each face, edge and corner at the finest spacing (small
    meshes only: pure Python)."""
    size = 1 << L
    dirs = [d for d in np.ndindex(*([3] * dim)) if any(v != 1 for v in d)]

    def find_leaf(pt):
        # leaf containing integer point pt (inside the domain); search coarse-to-fine
        for l in range(0, L + 1):
            s = 1 << (L - l)
            a = tuple((p // s) * s for p in pt)
            if leaves.get(a) == l:
                return a, l
        return None

    changed = True
    while changed:
        changed = False
        for a, l in list(leaves.items()):
            if leaves.get(a) != l:
                continue
            s = 1 << (L - l)
            for d in dirs:
                pts = []
                for k in range(dim):
                    dk = d[k] - 1
                    if dk < 0:
                        pts.append([a[k] - 1])
                    elif dk > 0:
                        pts.append([a[k] + s])
                    else:
                        pts.append(list(range(a[k], a[k] + s)))
                for pt in np.array(np.meshgrid(*pts, indexing="ij")).reshape(dim, -1).T:
                    pt = [int(p) % size if (periodic >> k) & 1 else int(p) for k, p in enumerate(pt)]
                    if any(p < 0 or p >= size for p in pt):
                        continue
                    nb = find_leaf(tuple(int(p) for p in pt))
                    if nb is not None and nb[1] < l - 1:
                        na, nl = nb
                        del leaves[na]
                        for ca, cl in _children(na, nl, dim, L):
                            leaves[ca] = cl
                        changed = True
    return leaves


def refine_and_balance(oc: Octants, target) -> Octants:
    """Each octant split down to ``target`` (its level at least), then 2:1 balanced with
    ``balance_leaves`` (small meshes only: pure Python)."""
    L, dim = oc.max_level, oc.dim
    leaves: dict[tuple, int] = {}

    def put(a, l, t):
        if l >= t:
            leaves[a] = l
            return
        for ca, cl in _children(a, l, dim, L):
            put(ca, cl, t)

    for a, l, t in zip(oc.anchors, oc.levels, target):
        put(tuple(int(v) for v in a), int(l), int(t))
    balance_leaves(leaves, dim, L, oc.periodic)
    anchors = np.array(sorted(leaves.keys()), dtype=np.int32)
    levels = np.array([leaves[tuple(int(v) for v in a)] for a in anchors], dtype=np.uint8)
    return Octants(dim, L, anchors, levels, int(oc.periodic))


def random_balanced_octants(dim: int, base_level: int, max_level: int, frac: float, seed: int,
                            periodic: int = 0) -> Octants:
    """A seeded random 2:1-balanced octree (face, edge and corner balance).

    Start from a uniform base grid, refine a random fraction of leaves level by level,
    then refine any leaf that has a neighbour two or more levels finer until none does.
    With periodic axes (bit k), neighbours are also looked up across the identified faces.
    Intended for small meshes (tests): pure Python dictionaries.
    """
    rng = np.random.default_rng(seed)
    L = max_level
    leaves: dict[tuple, int] = {}
    base = uniform_octants(dim, base_level, L)
    for a in base.anchors:
        leaves[tuple(int(v) for v in a)] = base_level

    def children(a, l):
        s = 1 << (L - l - 1)
        for c in range(1 << dim):
            yield tuple(a[k] + (s if (c >> k) & 1 else 0) for k in range(dim)), l + 1

    for lev in range(base_level, max_level):
        cand = [a for a, l in leaves.items() if l == lev]
        pick = rng.random(len(cand)) < frac
        for a, p in zip(cand, pick):
            if p:
                del leaves[a]
                for ca, cl in children(a, lev):
                    leaves[ca] = cl

    balance_leaves(leaves, dim, L, periodic)
    anchors = np.array(sorted(leaves.keys()), dtype=np.int32)
    levels = np.array([leaves[tuple(int(v) for v in a)] for a in anchors], dtype=np.uint8)
    return Octants(dim, L, anchors, levels, int(periodic))


# ----------------------------------------------------------------------------- BCs
@dataclasses.dataclass
class BoundaryConditions:
    """``types[face][field]`` in {NATURAL, DIRICHLET}; ``values[face][field]`` constants."""
    types: np.ndarray   # int32 [2*dim, 3]
    values: np.ndarray  # float64 [2*dim, 3]


def membrane_bcs(dim: int, V: float, membrane_c_plus: float | None) -> BoundaryConditions:
    """Ion-selective membrane at the bottom face, reservoir at the top face.

    Top (last axis = 1): phi = V, c+ = c- = 1 (Dirichlet).
    Bottom (last axis = 0): phi = 0; c+ = ``membrane_c_plus`` (Dirichlet) or zero flux
    when None; c- zero flux.  Side faces: zero flux for every field.
    """
    nf = 2 * dim
    t = np.zeros((nf, 3), np.int32)
    v = np.zeros((nf, 3), np.float64)
    bot, top = 2 * (dim - 1), 2 * (dim - 1) + 1
    t[top, :] = DIRICHLET
    v[top] = (1.0, 1.0, V)
    t[bot, PHI] = DIRICHLET
    v[bot, PHI] = 0.0
    if membrane_c_plus is not None:
        t[bot, C_PLUS] = DIRICHLET
        v[bot, C_PLUS] = membrane_c_plus
    return BoundaryConditions(t, v)


def equilibrium_bcs(dim: int, V: float) -> BoundaryConditions:
    """Steady double layer: phi = V at the bottom face and 0 at the top face, c+- = 1 at
    the top face, zero flux elsewhere (phi zero-Neumann on the sides)."""
    nf = 2 * dim
    t = np.zeros((nf, 3), np.int32)
    v = np.zeros((nf, 3), np.float64)
    bot, top = 2 * (dim - 1), 2 * (dim - 1) + 1
    t[top, :] = DIRICHLET
    v[top] = (1.0, 1.0, 0.0)
    t[bot, PHI] = DIRICHLET
    v[bot, PHI] = V
    return BoundaryConditions(t, v)


def all_natural_bcs(dim: int) -> BoundaryConditions:
    return BoundaryConditions(np.zeros((2 * dim, 3), np.int32), np.zeros((2 * dim, 3)))


# ----------------------------------------------------------------------------- random
def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser applied elementwise to uint64 ``x`` (wrapping arithmetic)."""
    x = (x + np.uint64(0x9E3779B97F4A7C15)) & _MASK64
    z = x
    z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _MASK64
    z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _MASK64
    return z ^ (z >> np.uint64(31))


def uniform01(seed: int, stream: int, ijk: np.ndarray, max_level: int) -> np.ndarray:
    """Uniform [0,1) numbers keyed by (seed, stream, node coordinates); float64 [n]."""
    with np.errstate(over="ignore"):
        shift = 20 - max_level
        c = ijk.astype(np.uint64) << np.uint64(shift)
        key = np.full(c.shape[0], np.uint64(seed) * np.uint64(0x9E3779B97F4A7C15) & _MASK64, np.uint64)
        key ^= np.uint64(stream) << np.uint64(56)
        for k in range(c.shape[1]):
            key ^= c[:, k] << np.uint64(21 * k)
            key = splitmix64(key)
        r = splitmix64(key)
    return (r >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def noisy_state(ijk: np.ndarray, max_level: int, seed: int, amp: float = 1e-3,
                phi_bottom: float = 0.0, phi_top: float = 1.0) -> np.ndarray:
    """Initial state [n, 3]: c+- = 1 + amp*(2u-1), phi linear in the last coordinate."""
    n, dim = ijk.shape
    U = np.empty((n, 3))
    U[:, 0] = 1.0 + amp * (2.0 * uniform01(seed, 0, ijk, max_level) - 1.0)
    U[:, 1] = 1.0 + amp * (2.0 * uniform01(seed, 1, ijk, max_level) - 1.0)
    zeta = ijk[:, dim - 1].astype(np.float64) / (1 << max_level)
    U[:, 2] = phi_bottom + (phi_top - phi_bottom) * zeta
    return U


def random_state(ijk: np.ndarray, max_level: int, seed: int, lo=(0.5, 0.5, -1.0), hi=(1.5, 1.5, 1.0)) -> np.ndarray:
    """Generic non-equilibrium state [n, 3] with per-field uniform ranges."""
    U = np.empty((ijk.shape[0], 3))
    for f in range(3):
        U[:, f] = lo[f] + (hi[f] - lo[f]) * uniform01(seed, 8 + f, ijk, max_level)
    return U


def random_direction(ijk: np.ndarray, max_level: int, seed: int) -> np.ndarray:
    """Random Krylov-like direction [n, 3], entries in [-1, 1], unit 2-norm."""
    V = np.empty((ijk.shape[0], 3))
    for f in range(3):
        V[:, f] = 2.0 * uniform01(seed, 16 + f, ijk, max_level) - 1.0
    return V / np.linalg.norm(V)


def random_velocity(ijk: np.ndarray, max_level: int, seed: int, amp: float) -> np.ndarray:
    """Nodal velocity [n, dim] with entries uniform in [-amp, amp] (not divergence-free)."""
    dim = ijk.shape[1]
    v = np.empty((ijk.shape[0], dim))
    for k in range(dim):
        v[:, k] = amp * (2.0 * uniform01(seed, 24 + k, ijk, max_level) - 1.0)
    return v


def fourier_velocity(ijk: np.ndarray, max_level: int, seed: int, rms: float = 0.1, n_modes: int = 8) -> np.ndarray:
    """Divergence-free 3D velocity u = curl(b * psi) at the nodes, RMS |u| = ``rms``.

    b = prod_i x_i^2 (1 - x_i)^2 vanishes with its gradient on every wall, so u = 0
    there.  psi is a vector of seeded Fourier sums
    psi_c = sum_m A_{c,m} sin(2 pi k_{c,m}.x + theta_{c,m}) with integer wave
    vectors, |k|_inf <= 4.
    """
    assert ijk.shape[1] == 3
    rng = np.random.default_rng(seed)
    x = ijk.astype(np.float64) / (1 << max_level)
    b = np.prod(x**2 * (1 - x) ** 2, axis=1)
    db = np.empty_like(x)
    for i in range(3):
        others = np.prod(np.delete(x**2 * (1 - x) ** 2, i, axis=1), axis=1)
        xi = x[:, i]
        db[:, i] = others * (2 * xi * (1 - xi) ** 2 - 2 * xi**2 * (1 - xi))
    psi = np.zeros((x.shape[0], 3))
    dpsi = np.zeros((x.shape[0], 3, 3))  # dpsi[:, c, j] = d psi_c / d x_j
    for c in range(3):
        for _ in range(n_modes):
            k = rng.integers(-4, 5, size=3)
            if not k.any():
                k[0] = 1
            A = rng.normal()
            th = rng.uniform(0, 2 * np.pi)
            arg = 2 * np.pi * (x @ k) + th
            psi[:, c] += A * np.sin(arg)
            for j in range(3):
                dpsi[:, c, j] += A * np.cos(arg) * 2 * np.pi * k[j]
    # A_c = b psi_c ; dA_c/dx_j = db_j psi_c + b dpsi_cj
    dA = db[:, None, :] * psi[:, :, None] + b[:, None, None] * dpsi
    u = np.stack([dA[:, 2, 1] - dA[:, 1, 2], dA[:, 0, 2] - dA[:, 2, 0], dA[:, 1, 0] - dA[:, 0, 1]], axis=1)
    r = np.sqrt(np.mean(np.sum(u**2, axis=1)))
    return u * (rms / r) if r > 0 else u
