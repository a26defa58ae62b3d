"""Python side of the FP64 CPU oracle (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline and ``--impl reference``
legs of ``bench.py`` import this module.  The library's product path never does.

It wraps ``pnp_oracle.cpp`` (mesh, residual, analytic Jacobian, matrix-free Jv) and
adds the solution algorithms of the paper written out plainly:

* Newton's method on the PNP block (Sec. 4.1, Eq. newton_linear_system) with the
  analytic Jacobian, solved by a sparse direct factorisation (a library primitive),
  optional backtracking line search, stop on ||F(U^m)||_2 <= rtol ||F(U^0)||_2.
* BDF time stepping (Def. 1 of Sec. 3): BDF1 on the first step, constant-step BDF2
  (beta = 3/2, -2, 1/2) after it; the advection velocity is the extrapolation
  v~ = 2 v^k - v^{k-1} (Eq. averaging1) of a caller-supplied velocity history.
* The method-of-manufactured-solutions driver of Sec. 5.1.
* The semi-implicit VMS Navier-Stokes block (Def. 3, Sec. 3.1): a linear system in
  (v, p) solved by a sparse direct factorisation, and the block iteration of Sec. 4.1
  (NS from the latest PNP state, then PNP Newton with the new velocity as advection).
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import sys

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)
import build as _build  # noqa: E402

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        vp, i64p, dp, i32p = C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_double), C.POINTER(C.c_int32)
        L.ora_mesh_build.restype = vp
        L.ora_mesh_build.argtypes = [C.c_int, C.c_int, C.c_int64, i32p, C.POINTER(C.c_uint8), C.c_int, i32p]
        L.ora_mesh_free.argtypes = [vp]
        L.ora_mesh_sizes.argtypes = [vp, i64p, i64p, i64p]
        L.ora_mesh_nodes.argtypes = [vp, i64p, i32p, i64p]
        L.ora_mesh_constraints.restype = C.c_int64
        L.ora_mesh_constraints.argtypes = [vp, i64p, i64p, dp]
        L.ora_residual.argtypes = [vp, vp, dp, dp, dp, dp, dp]
        L.ora_jacobian.restype = C.c_int64
        L.ora_jacobian.argtypes = [vp, vp, dp, dp, dp, dp, i64p, i64p, dp]
        L.ora_jv.argtypes = [vp, vp, dp, dp, dp, dp, dp, dp]
        L.ora_residual_elements.argtypes = [vp, vp, dp, dp, dp, dp, C.c_int64, C.c_int64, dp]
        L.ora_jv_elements.argtypes = [vp, vp, dp, dp, dp, dp, dp, C.c_int64, C.c_int64, dp]
        L.ora_qp_eval.argtypes = [vp, vp, C.c_int64, C.c_int, dp, dp, dp, dp, dp]
        L.ora_bc_rows.argtypes = [vp, vp, i32p, dp]
        L.ora_mms.argtypes = [C.c_int, C.c_double, C.c_double, C.c_int, C.c_int64, dp, dp, dp]
        L.ora_eval_points.argtypes = [vp, dp, C.c_int64, i64p, dp]
        L.ora_boundary_flux.argtypes = [vp, C.c_int, dp, dp]
        L.ora_plane_integral.argtypes = [vp, C.c_int, C.c_int64, dp, dp]
        L.ora_ns_apply.argtypes = [vp, vp, dp, dp, dp, dp, dp, C.c_int, dp]
        L.ora_ns_apply_elements.argtypes = [vp, vp, dp, dp, dp, dp, dp, C.c_int, C.c_int64, C.c_int64, dp]
        L.ora_ns_matrix.restype = C.c_int64
        L.ora_ns_matrix.argtypes = [vp, vp, dp, i64p, i64p, dp]
        L.ora_ns_bc_rows.argtypes = [vp, vp, i32p, dp]
        L.ora_ns_mms.argtypes = [vp, C.c_int, C.c_double, C.c_int64, dp, dp, dp]
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


class _Params(C.Structure):
    _fields_ = [
        ("eps", C.c_double), ("dt", C.c_double), ("beta0", C.c_double), ("beta1", C.c_double),
        ("beta2", C.c_double), ("C_I", C.c_double), ("t", C.c_double),
        ("steady", C.c_int32), ("vms", C.c_int32), ("mms", C.c_int32), ("pad", C.c_int32),
        ("bc_type", (C.c_int32 * 3) * 6), ("bc_val", (C.c_double * 3) * 6),
    ]


@dataclasses.dataclass
class Params:
    """Parameters of the discrete PNP residual.

    eps   : Lambda (non-dimensional Debye length; Poisson coefficient 2 Lambda^2, Eq. nondim_poisson)
    dt    : time step;  beta = (beta0, beta1, beta2) BDF coefficients
    C_I   : constant of tau_c (6 in Sec. 3.1)
    steady: drop d/dt terms;  vms: include the fine-scale terms;  mms: manufactured forcing
    bc_type / bc_val : [2*dim, 3] per face, per field (0 natural, 1 Dirichlet)
    """
    eps: float
    dt: float = 1.0
    beta: tuple = (1.0, -1.0, 0.0)
    C_I: float = 6.0
    t: float = 0.0
    steady: bool = False
    vms: bool = True
    mms: bool = False
    bc_type: np.ndarray | None = None
    bc_val: np.ndarray | None = None

    def to_c(self) -> _Params:
        p = _Params()
        p.eps, p.dt = self.eps, self.dt
        p.beta0, p.beta1, p.beta2 = self.beta
        p.C_I, p.t = self.C_I, self.t
        p.steady, p.vms, p.mms = int(self.steady), int(self.vms), int(self.mms)
        if self.bc_type is not None:
            for f in range(self.bc_type.shape[0]):
                for k in range(3):
                    p.bc_type[f][k] = int(self.bc_type[f, k])
                    p.bc_val[f][k] = float(self.bc_val[f, k])
        return p


class _NsParams(C.Structure):
    _fields_ = [
        ("Sc", C.c_double), ("kappa", C.c_double), ("eps", C.c_double), ("dt", C.c_double),
        ("beta0", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double), ("C_I", C.c_double),
        ("t", C.c_double), ("pin_val", C.c_double),
        ("steady", C.c_int32), ("vms", C.c_int32), ("mms", C.c_int32), ("pin", C.c_int32),
        ("bc_type", (C.c_int32 * 4) * 6), ("bc_val", (C.c_double * 4) * 6),
    ]


@dataclasses.dataclass
class NsParams:
    """Parameters of the linear VMS Navier-Stokes block.

    Sc    : Schmidt number (inertia coefficient 1/Sc; 1/Re = Sc in tau_m)
    kappa : electrohydrodynamic coupling constant; eps: Lambda (body force kappa/(2 Lambda^2))
    dt, beta : time step and BDF coefficients;  C_I: constant of tau_m (6)
    steady: drop d/dt terms;  vms: include the fine-scale terms;  mms: manufactured forcing
    pin   : fix the pressure of the node at the origin to pin_val
    bc_type / bc_val : [2*dim, 4] per face, per slot (v_x, v_y, v_z, p): 0 natural, 1 Dirichlet
    """
    Sc: float = 1.0
    kappa: float = 0.5
    eps: float = 1.0
    dt: float = 1.0
    beta: tuple = (1.0, -1.0, 0.0)
    C_I: float = 6.0
    t: float = 0.0
    steady: bool = False
    vms: bool = True
    mms: bool = False
    pin: bool = True
    pin_val: float = 0.0
    bc_type: np.ndarray | None = None
    bc_val: np.ndarray | None = None

    def to_c(self) -> _NsParams:
        p = _NsParams()
        p.Sc, p.kappa, p.eps, p.dt = self.Sc, self.kappa, self.eps, self.dt
        p.beta0, p.beta1, p.beta2 = self.beta
        p.C_I, p.t, p.pin_val = self.C_I, self.t, self.pin_val
        p.steady, p.vms, p.mms, p.pin = int(self.steady), int(self.vms), int(self.mms), int(self.pin)
        if self.bc_type is not None:
            for f in range(self.bc_type.shape[0]):
                for k in range(4):
                    p.bc_type[f][k] = int(self.bc_type[f, k])
                    p.bc_val[f][k] = float(self.bc_val[f, k])
        return p


def no_slip_bcs(dim: int, walls=None):
    """Velocity Dirichlet 0 on the faces in `walls` (default: all 2*dim faces); pressure natural."""
    bt = np.zeros((2 * dim, 4), np.int32)
    for f in (range(2 * dim) if walls is None else walls):
        bt[f, :3] = 1
    return bt, np.zeros((2 * dim, 4))


class OracleMesh:
    """Mesh built by the oracle's own construction (std::map on coordinates)."""

    def __init__(self, octants):
        L = lib()
        err = C.c_int32(0)
        a = np.ascontiguousarray(octants.anchors, dtype=np.int32)
        lv = np.ascontiguousarray(octants.levels, dtype=np.uint8)
        self.periodic = int(getattr(octants, "periodic", 0))
        self.h = L.ora_mesh_build(octants.dim, octants.max_level, octants.n, _p(a, C.c_int32),
                                  _p(lv, C.c_uint8), self.periodic, C.byref(err))
        if not self.h:
            raise ValueError(f"oracle mesh build failed (code {err.value})")
        self.dim, self.max_level = octants.dim, octants.max_level
        ne, nn, nh = C.c_int64(), C.c_int64(), C.c_int64()
        L.ora_mesh_sizes(self.h, C.byref(ne), C.byref(nn), C.byref(nh))
        self.n_elem, self.n_nodes, self.n_hanging = ne.value, nn.value, nh.value
        self.ijk = np.zeros((self.n_nodes, self.dim), np.int64)
        self.hanging = np.zeros(self.n_nodes, np.int32)
        self.el_nodes = np.zeros((self.n_elem, 1 << self.dim), np.int64)
        L.ora_mesh_nodes(self.h, _p(self.ijk, C.c_int64), _p(self.hanging, C.c_int32), _p(self.el_nodes, C.c_int64))
        self.x = self.ijk.astype(np.float64) / (1 << self.max_level)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ora_mesh_free(self.h)
            self.h = None

    # ------------------------------------------------------------------ helpers
    def constraints(self):
        L = lib()
        k = L.ora_mesh_constraints(self.h, None, None, None)
        r = np.zeros(k, np.int64); c = np.zeros(k, np.int64); w = np.zeros(k)
        L.ora_mesh_constraints(self.h, _p(r, C.c_int64), _p(c, C.c_int64), _p(w, C.c_double))
        return r, c, w

    def _vel3(self, adv):
        v = np.zeros((self.n_nodes, 3))
        if adv is not None:
            adv = np.asarray(adv, dtype=np.float64).reshape(self.n_nodes, -1)
            v[:, : adv.shape[1]] = adv
        return v

    def _z(self, X):
        return np.zeros((self.n_nodes, 3)) if X is None else np.ascontiguousarray(X, dtype=np.float64).reshape(self.n_nodes, 3)

    def bc_rows(self, p: Params):
        kind = np.zeros((self.n_nodes, 3), np.int32)
        g = np.zeros((self.n_nodes, 3))
        pc = p.to_c()
        lib().ora_bc_rows(self.h, C.byref(pc), _p(kind, C.c_int32), _p(g, C.c_double))
        return kind, g

    def make_consistent(self, U, p: Params):
        """Impose Dirichlet values and interpolate hanging nodes from their parents."""
        U = np.array(U, dtype=np.float64).reshape(self.n_nodes, 3)
        kind, g = self.bc_rows(p)
        U[kind == 1] = g[kind == 1]
        r, c, w = self.constraints()
        if len(r):
            hv = np.zeros((self.n_nodes, 3))
            np.add.at(hv, r, w[:, None] * U[c])
            hn = np.unique(r)
            U[hn] = hv[hn]
        return U

    # ------------------------------------------------------------------ operators
    def residual(self, p: Params, U, Uk=None, Ukm1=None, adv=None):
        U = self._z(U); Uk = self._z(Uk); Ukm1 = self._z(Ukm1); v = self._vel3(adv)
        F = np.zeros((self.n_nodes, 3))
        pc = p.to_c()
        lib().ora_residual(self.h, C.byref(pc), _p(U, C.c_double), _p(Uk, C.c_double), _p(Ukm1, C.c_double),
                           _p(v, C.c_double), _p(F, C.c_double))
        return F

    def boundary_flux(self, U, face: int):
        """[int_face n.(grad c+ + c+ grad phi), int_face n.(grad c- - c- grad phi)] over
        boundary face `face` (outward normal): the species terms of the boundary current
        of Sec. 5.2."""
        U = self._z(U)
        out = np.zeros(2)
        lib().ora_boundary_flux(self.h, int(face), _p(U, C.c_double), _p(out, C.c_double))
        return out

    def plane_integral(self, U, axis: int, coord: int):
        """Integrals of (c+, c-, phi) over the plane x_axis = coord 2^-max_level (the
        x-averaged profiles of Sec. 5.2 on the unit domain)."""
        U = self._z(U)
        out = np.zeros(3)
        lib().ora_plane_integral(self.h, int(axis), int(coord), _p(U, C.c_double), _p(out, C.c_double))
        return out

    def jacobian(self, p: Params, U, Uk=None, Ukm1=None, adv=None) -> sp.csr_matrix:
        U = self._z(U); Uk = self._z(Uk); Ukm1 = self._z(Ukm1); v = self._vel3(adv)
        pc = p.to_c()
        L = lib()
        args = (self.h, C.byref(pc), _p(U, C.c_double), _p(Uk, C.c_double), _p(Ukm1, C.c_double), _p(v, C.c_double))
        k = L.ora_jacobian(*args, None, None, None)
        I = np.zeros(k, np.int64); J = np.zeros(k, np.int64); X = np.zeros(k)
        L.ora_jacobian(*args, _p(I, C.c_int64), _p(J, C.c_int64), _p(X, C.c_double))
        n = 3 * self.n_nodes
        return sp.coo_matrix((X, (I, J)), shape=(n, n)).tocsr()

    def jv(self, p: Params, U, V, Uk=None, Ukm1=None, adv=None):
        U = self._z(U); V = self._z(V); Uk = self._z(Uk); Ukm1 = self._z(Ukm1); v = self._vel3(adv)
        JV = np.zeros((self.n_nodes, 3))
        pc = p.to_c()
        lib().ora_jv(self.h, C.byref(pc), _p(U, C.c_double), _p(Uk, C.c_double), _p(Ukm1, C.c_double),
                     _p(v, C.c_double), _p(V, C.c_double), _p(JV, C.c_double))
        return JV

    def residual_elements(self, p: Params, U, Uk, Ukm1, adv, e0: int, e1: int, F):
        """Add the element contributions of elements e0 <= e < e1 into F [n_nodes, 3]
        (C-contiguous float64, modified in place; no Dirichlet or constraint rows)."""
        U = self._z(U); Uk = self._z(Uk); Ukm1 = self._z(Ukm1); v = self._vel3(adv)
        pc = p.to_c()
        lib().ora_residual_elements(self.h, C.byref(pc), _p(U, C.c_double), _p(Uk, C.c_double),
                                    _p(Ukm1, C.c_double), _p(v, C.c_double), int(e0), int(e1), _p(F, C.c_double))
        return F

    def jv_elements(self, p: Params, U, V, Uk, Ukm1, adv, e0: int, e1: int, JV):
        """Add the element contributions of elements e0 <= e < e1 into JV [n_nodes, 3]
        (C-contiguous float64, modified in place; no Dirichlet or constraint rows)."""
        U = self._z(U); V = self._z(V); Uk = self._z(Uk); Ukm1 = self._z(Ukm1); v = self._vel3(adv)
        pc = p.to_c()
        lib().ora_jv_elements(self.h, C.byref(pc), _p(U, C.c_double), _p(Uk, C.c_double), _p(Ukm1, C.c_double),
                              _p(v, C.c_double), _p(V, C.c_double), int(e0), int(e1), _p(JV, C.c_double))
        return JV

    def eval_points(self, U, pts):
        """Q1 field U [n_nodes, 3] at integer points pts [k, dim] -> [k, 3]."""
        U = self._z(U)
        pts = np.ascontiguousarray(pts, dtype=np.int64)
        out = np.zeros((pts.shape[0], 3))
        lib().ora_eval_points(self.h, _p(U, C.c_double), pts.shape[0], _p(pts, C.c_int64), _p(out, C.c_double))
        return out

    def node_sizes(self, levels):
        """Edge (integer units) of the finest element having each node as a corner."""
        s_el = (1 << self.max_level) >> np.asarray(levels, np.int64)
        hmin = np.full(self.n_nodes, 1 << self.max_level, np.int64)
        for c in range(self.el_nodes.shape[1]):
            np.minimum.at(hmin, self.el_nodes[:, c], s_el)
        return hmin

    # ------------------------------------------------------------------ Navier-Stokes block
    def _x4(self, X):
        return np.zeros((self.n_nodes, 4)) if X is None else np.ascontiguousarray(X, dtype=np.float64).reshape(self.n_nodes, 4)

    def ns_apply(self, p: NsParams, X, adv=None, Vk=None, Vkm1=None, U=None, with_data=True):
        """NS rows [n_nodes, 4] of X: the residual of the linear system (with_data) or the
        matrix times X."""
        X = self._x4(X); a = self._vel3(adv); vk = self._vel3(Vk); vkm1 = self._vel3(Vkm1); U = self._z(U)
        F = np.zeros((self.n_nodes, 4))
        pc = p.to_c()
        lib().ora_ns_apply(self.h, C.byref(pc), _p(X, C.c_double), _p(a, C.c_double), _p(vk, C.c_double),
                           _p(vkm1, C.c_double), _p(U, C.c_double), int(bool(with_data)), _p(F, C.c_double))
        return F

    def ns_apply_elements(self, p: NsParams, X, adv, Vk, Vkm1, U, with_data, e0: int, e1: int, F):
        """Add the element contributions of elements e0 <= e < e1 into F [n_nodes, 4]
        (C-contiguous float64, modified in place; no Dirichlet or constraint rows)."""
        X = self._x4(X); a = self._vel3(adv); vk = self._vel3(Vk); vkm1 = self._vel3(Vkm1); U = self._z(U)
        pc = p.to_c()
        lib().ora_ns_apply_elements(self.h, C.byref(pc), _p(X, C.c_double), _p(a, C.c_double), _p(vk, C.c_double),
                                    _p(vkm1, C.c_double), _p(U, C.c_double), int(bool(with_data)), int(e0), int(e1),
                                    _p(F, C.c_double))
        return F

    def ns_matrix(self, p: NsParams, adv=None) -> sp.csr_matrix:
        a = self._vel3(adv)
        pc = p.to_c()
        L = lib()
        k = L.ora_ns_matrix(self.h, C.byref(pc), _p(a, C.c_double), None, None, None)
        I = np.zeros(k, np.int64); J = np.zeros(k, np.int64); X = np.zeros(k)
        L.ora_ns_matrix(self.h, C.byref(pc), _p(a, C.c_double), _p(I, C.c_int64), _p(J, C.c_int64), _p(X, C.c_double))
        n = 4 * self.n_nodes
        return sp.coo_matrix((X, (I, J)), shape=(n, n)).tocsr()

    def ns_bc_rows(self, p: NsParams):
        kind = np.zeros((self.n_nodes, 4), np.int32)
        g = np.zeros((self.n_nodes, 4))
        pc = p.to_c()
        lib().ora_ns_bc_rows(self.h, C.byref(pc), _p(kind, C.c_int32), _p(g, C.c_double))
        return kind, g

    def ns_solve(self, p: NsParams, adv=None, Vk=None, Vkm1=None, U=None):
        """The (v, p) of the linear NS system: A X = -F(0) by a sparse direct solve."""
        b = -self.ns_apply(p, None, adv, Vk, Vkm1, U, with_data=True).reshape(-1)
        A = self.ns_matrix(p, adv)
        return spla.spsolve(A.tocsc(), b).reshape(-1, 4)

    def qp_eval(self, p: Params, e: int, q: int, U, Uk=None, Ukm1=None, adv=None):
        U = self._z(U); Uk = self._z(Uk); Ukm1 = self._z(Ukm1); v = self._vel3(adv)
        out = np.zeros(3)
        pc = p.to_c()
        lib().ora_qp_eval(self.h, C.byref(pc), e, q, _p(U, C.c_double), _p(Uk, C.c_double),
                          _p(Ukm1, C.c_double), _p(v, C.c_double), _p(out, C.c_double))
        return out


def mms_eval(dim: int, eps: float, t: float, steady: bool, x: np.ndarray):
    """Manufactured fields (c+, c-, phi, u, v, w) and forcing (f+, f-, f_phi) at points x."""
    n = x.shape[0]
    x3 = np.zeros((n, 3)); x3[:, : x.shape[1]] = x
    vals = np.zeros((n, 6)); forc = np.zeros((n, 3))
    lib().ora_mms(dim, eps, t, int(steady), n, _p(x3, C.c_double), _p(vals, C.c_double), _p(forc, C.c_double))
    return vals, forc


# ---------------------------------------------------------------------- solvers
@dataclasses.dataclass
class NewtonResult:
    U: np.ndarray
    norms: list
    converged: bool
    iterations: int


def newton(mesh: OracleMesh, p: Params, U0, Uk=None, Ukm1=None, adv=None, rtol=1e-10, atol=0.0,
           max_it=30, line_search=True) -> NewtonResult:
    """Newton's method (Sec. 4.1) with a direct sparse solve of J dU = -F.

    U0 is made consistent (Dirichlet values, hanging interpolation) first.  Backtracking
    line search: halve alpha until ||F(U + alpha dU)|| <= (1 - 1e-4 alpha) ||F(U)||.
    """
    U = mesh.make_consistent(U0, p)
    F = mesh.residual(p, U, Uk, Ukm1, adv)
    f0 = np.linalg.norm(F)
    norms = [f0]
    it = 0
    while norms[-1] > max(rtol * f0, atol) and it < max_it:
        J = mesh.jacobian(p, U, Uk, Ukm1, adv)
        dU = spla.spsolve(J.tocsc(), -F.reshape(-1)).reshape(-1, 3)
        alpha = 1.0
        while True:
            Ut = U + alpha * dU
            Ft = mesh.residual(p, Ut, Uk, Ukm1, adv)
            ft = np.linalg.norm(Ft)
            if not line_search or ft <= (1.0 - 1e-4 * alpha) * norms[-1] or alpha < 1e-4:
                break
            alpha *= 0.5
        U, F = Ut, Ft
        norms.append(ft)
        it += 1
    return NewtonResult(U, norms, norms[-1] <= max(rtol * f0, atol), it)


def bdf_coefficients(step_index: int, order: int = 2):
    """(beta0, beta1, beta2) of constant-step BDF; BDF1 on the first step."""
    if order == 1 or step_index == 0:
        return (1.0, -1.0, 0.0)
    return (1.5, -2.0, 0.5)


def mms_run(octants, eps: float, dt: float, n_steps: int, steady: bool = False, rtol: float = 1e-11):
    """Manufactured-solution run (Sec. 5.1) on the mesh of ``octants`` (uniform in the paper).

    PNP only: the manufactured velocity (u, v) of Eq. manufac_sol is the advection
    field (interpolated at the nodes; in the transient run the extrapolation
    2 v^k - v^{k-1} of the nodal velocity history).  Dirichlet data on every face.
    Returns (mesh, U_final, exact_final, t_final).
    """
    dim = octants.dim
    mesh = OracleMesh(octants)
    bt = np.ones((2 * dim, 3), np.int32)
    bv = np.zeros((2 * dim, 3))

    def exact(t):
        vals, _ = mms_eval(dim, eps, t, steady, mesh.x)
        return vals[:, :3].copy(), vals[:, 3:3 + dim].copy()

    if steady:
        p = Params(eps=eps, steady=True, mms=True, bc_type=bt, bc_val=bv)
        U0 = np.zeros((mesh.n_nodes, 3))
        _, vel = exact(0.0)
        res = newton(mesh, p, U0, adv=vel, rtol=rtol)
        return mesh, res.U, exact(0.0)[0], 0.0
    U_prev, v_prev = exact(-dt)
    U_cur, v_cur = exact(0.0)
    t = 0.0
    for k in range(n_steps):
        t_new = (k + 1) * dt
        beta = bdf_coefficients(k)
        # velocity at t^{k+1}: extrapolation of the nodal history (Eq. averaging1)
        vt = 2.0 * v_cur - v_prev
        p = Params(eps=eps, dt=dt, beta=beta, t=t_new, mms=True, bc_type=bt, bc_val=bv)
        res = newton(mesh, p, 2.0 * U_cur - U_prev if k else U_cur, U_cur, U_prev, vt, rtol=rtol)
        U_prev, U_cur = U_cur, res.U
        v_prev, v_cur = v_cur, exact(t_new)[1]
        t = t_new
    return mesh, U_cur, exact(t)[0], t


def stencil_offsets(dim: int = 3):
    """The 27 (9 in 2D) lattice offsets in {-1,0,1}^dim, x fastest."""
    r = [-1, 0, 1]
    if dim == 3:
        return np.array([(x, y, z) for z in r for y in r for x in r], np.int64)
    return np.array([(x, y) for y in r for x in r], np.int64)


def stencil_features(mesh: OracleMesh, levels, Uk, Ukm1, uz_k=None, uz_km1=None):
    """Raw network inputs of every non-hanging node: the fields (c+, c-, phi, u_z) of the
    last two time levels at the 3x3x3 lattice around the node with spacing equal to the
    finest incident element, points clamped to the domain, values of the Q1 fields there.
    Returns (node ids, features [n, 216]) with feature index ((step*4 + field)*27 + point),
    step 0 = U^k, step 1 = U^{k-1}.
    """
    nodes = np.nonzero(mesh.hanging == 0)[0]
    hmin = mesh.node_sizes(levels)
    off = stencil_offsets(mesh.dim)
    npt = off.shape[0]
    size = 1 << mesh.max_level
    pts = mesh.ijk[nodes][:, None, :] + hmin[nodes][:, None, None] * off[None, :, :]
    pts = np.clip(pts, 0, size).reshape(-1, mesh.dim)
    feats = np.zeros((nodes.size, 8 * npt))
    zero = np.zeros(mesh.n_nodes)
    for step, (U, uz) in enumerate(((Uk, uz_k), (Ukm1, uz_km1))):
        vals = mesh.eval_points(U, pts).reshape(nodes.size, npt, 3)
        U4 = np.zeros((mesh.n_nodes, 3))
        U4[:, 0] = zero if uz is None else uz
        vz = mesh.eval_points(U4, pts).reshape(nodes.size, npt, 3)[:, :, 0]
        for f in range(3):
            feats[:, (step * 4 + f) * npt:(step * 4 + f + 1) * npt] = vals[:, :, f]
        feats[:, (step * 4 + 3) * npt:(step * 4 + 4) * npt] = vz
    return nodes, feats


def l2_error(mesh: OracleMesh, U, Uex):
    """Discrete L2 error on a uniform grid: sqrt(h^d sum_i |U_i - Uex_i|^2) per field."""
    h = 1.0 / (1 << mesh.max_level)
    d = U - Uex
    return np.sqrt(h ** mesh.dim * np.sum(d**2, axis=0))


def ns_mms_eval(p: NsParams, dim: int, t: float, x: np.ndarray):
    """Manufactured (u, v, w, p) [n, 4] of Eq. manufac_sol and the momentum forcing [n, 3]."""
    n = x.shape[0]
    x3 = np.zeros((n, 3)); x3[:, : x.shape[1]] = x
    vals = np.zeros((n, 4)); forc = np.zeros((n, 3))
    pc = p.to_c()
    lib().ora_ns_mms(C.byref(pc), dim, t, n, _p(x3, C.c_double), _p(vals, C.c_double), _p(forc, C.c_double))
    return vals, forc


@dataclasses.dataclass
class CoupledResult:
    X: np.ndarray          # (v, p) at t^{k+1}, [n, 4]
    U: np.ndarray          # (c+, c-, phi) at t^{k+1}, [n, 3]
    newton_its: list


def coupled_step(mesh: OracleMesh, p: Params, nsp: NsParams, Uk, Ukm1, Vk, Vkm1, n_block: int = 1,
                 start: str = "previous", rtol: float = 1e-10, line_search: bool = True) -> CoupledResult:
    """One NS-PNP time step by block iteration (Sec. 4.1): the linear NS block from the
    latest PNP state (U^k in the first pass), then PNP Newton with the new velocity as
    advection; repeated n_block times.  p and nsp carry the step's dt and BDF
    coefficients; the NS advection is v~ = 2 v^k - v^{k-1} (Eq. averaging1).
    """
    Uk = mesh._z(Uk); Ukm1 = mesh._z(Ukm1)
    vk = mesh._vel3(Vk); vkm1 = mesh._vel3(Vkm1)
    adv = 2.0 * vk - vkm1
    U = Uk.copy() if start == "previous" else 2.0 * Uk - Ukm1
    body = Uk
    its = []
    X = None
    for _ in range(n_block):
        X = mesh.ns_solve(nsp, adv, vk, vkm1, body)
        # every pass meets rtol ||F(U^k)|| (with this pass's advection), whatever its start
        f_ref = np.linalg.norm(mesh.residual(p, mesh.make_consistent(Uk, p), Uk, Ukm1, X[:, :3]))
        res = newton(mesh, p, U, Uk, Ukm1, adv=X[:, :3], rtol=rtol, atol=rtol * f_ref, line_search=line_search)
        U = res.U
        body = U
        its.append(res.iterations)
    return CoupledResult(X, U, its)
