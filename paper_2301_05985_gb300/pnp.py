"""Thin ctypes binding of the C ABI in ``include/pnp.h`` (argument marshalling only).

Every computation runs in ``_build/libpnp_gb300.so``; this module only converts Python
arguments (numpy arrays on the host, torch CUDA tensors on the device) into pointers
and sizes, checks status codes and raises ``PnpError`` with the library's message.
There is no fallback: if the library is missing, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpnp_gb300.so")

# enums (include/pnp.h)
PNP_OK, PNP_ERR_ARG, PNP_ERR_MESH, PNP_ERR_MESH_UNBALANCED, PNP_ERR_NAN = 0, 1, 2, 3, 4
PNP_ERR_KRYLOV_MAXIT, PNP_ERR_NEWTON_DIVERGED, PNP_ERR_CUDA, PNP_ERR_DEVICE_FLAG = 5, 6, 7, 8
PNP_ERR_NOMEM, PNP_ERR_STATE = 9, 10
PNP_C_PLUS, PNP_C_MINUS, PNP_PHI = 0, 1, 2
PNP_NATURAL, PNP_DIRICHLET = 0, 1
PNP_F64, PNP_F32 = 0, 1
PNP_DEVICE, PNP_HOST = 0, 1
PNP_FIELD_U, PNP_FIELD_U_PREV, PNP_FIELD_U_PREV2 = 0, 1, 2
PNP_FIELD_ADVECTION, PNP_FIELD_VELOCITY, PNP_FIELD_VELOCITY_PREV = 3, 4, 5
PNP_FIELD_NS = 6
PNP_NS_VX, PNP_NS_VY, PNP_NS_VZ, PNP_NS_P = 0, 1, 2, 3
PNP_START_PREVIOUS, PNP_START_EXTRAPOLATE, PNP_START_LEARNED = 0, 1, 2


class PnpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[pnp status {code}] {msg}")
        self.code = code


class pnp_params(C.Structure):
    _fields_ = [
        ("eps", C.c_double), ("dt", C.c_double), ("C_I", C.c_double),
        ("beta0", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double),
        ("steady", C.c_int32), ("bdf_order", C.c_int32),
        ("newton_rtol", C.c_double), ("newton_atol", C.c_double),
        ("newton_max_it", C.c_int32), ("line_search", C.c_int32),
        ("gmres_restart", C.c_int32), ("gmres_max_it", C.c_int32),
        ("gmres_rtol", C.c_double),
        ("precision", C.c_int32), ("start_mode", C.c_int32),
        ("ew_eta_max", C.c_double), ("ew_eta_min", C.c_double),
        ("monitor", C.c_int32), ("f64_fallback", C.c_int32),
        ("gmres_cgs2", C.c_int32), ("dt_retries", C.c_int32),
        ("gmres_inner", C.c_int32), ("newton_ew_f64", C.c_int32),
        ("mg_levels", C.c_int32), ("mg_smooth", C.c_int32), ("mg_omega", C.c_double),
        ("mg_coarse_its", C.c_int32), ("ns_blocks", C.c_int32),
        ("ns_Sc", C.c_double), ("ns_kappa", C.c_double), ("ns_rtol", C.c_double), ("ns_atol", C.c_double),
        ("ns_inner_rtol", C.c_double), ("ns_max_it", C.c_int32), ("ns_pin", C.c_int32),
        ("ns_mg_levels", C.c_int32), ("ns_inner_max_it", C.c_int32),
        ("ns_fgmres", C.c_int32), ("pad4_", C.c_int32),
    ]


class pnp_ns_stats(C.Structure):
    _fields_ = [
        ("status", C.c_int32), ("refinements", C.c_int32), ("inner_its", C.c_int32),
        ("matvecs32", C.c_int32), ("matvecs64", C.c_int32), ("singular_blocks", C.c_int32),
        ("floor_stop", C.c_int32), ("mg_fallbacks", C.c_int32),
        ("krylov_fallbacks", C.c_int32), ("pad_", C.c_int32),
        ("res0", C.c_double), ("res_final", C.c_double), ("wall_ms", C.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class pnp_solve_stats(C.Structure):
    _fields_ = [
        ("status", C.c_int32), ("newton_its", C.c_int32), ("krylov_its", C.c_int32),
        ("residual_evals", C.c_int32), ("jv_evals", C.c_int32), ("start_used", C.c_int32),
        ("f64_fallbacks", C.c_int32), ("substeps", C.c_int32),
        ("res0", C.c_double), ("res_final", C.c_double),
        ("res_start_extrapolated", C.c_double), ("res_start_learned", C.c_double),
        ("wall_ms", C.c_double), ("res_ref", C.c_double),
        ("mg_fallbacks", C.c_int32), ("pad_", C.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class pnp_train_cfg(C.Structure):
    _fields_ = [("steps", C.c_int32), ("batch", C.c_int32), ("lr", C.c_double), ("beta1", C.c_double),
                ("beta2", C.c_double), ("adam_eps", C.c_double), ("seed", C.c_uint64)]


class pnp_train_stats(C.Structure):
    _fields_ = [("loss_first", C.c_double), ("loss_last", C.c_double), ("wall_ms", C.c_double),
                ("samples", C.c_int64), ("steps", C.c_int32), ("pad_", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


PNP_MLP_PARAMS = 61187

_lib = None
_vp, _i64, _i32, _d = C.c_void_p, C.c_int64, C.c_int32, C.c_double
_P = C.POINTER

# name -> (restype, argtypes)
SIGNATURES = {
    "pnp_last_error": (C.c_char_p, []),
    "pnp_version": (C.c_char_p, []),
    "pnp_params_default": (None, [_P(pnp_params)]),
    "pnp_mesh_create": (C.c_int, [C.c_int, C.c_int, _i64, _vp, _vp, _P(_vp)]),
    "pnp_mesh_create_periodic": (C.c_int, [C.c_int, C.c_int, _i64, _vp, _vp, C.c_int, _P(_vp)]),
    "pnp_mesh_create_refined": (C.c_int, [C.c_int, C.c_int, _i64, _vp, _vp, _vp, C.c_int, _P(_vp)]),
    "pnp_mesh_destroy": (None, [_vp]),
    "pnp_mesh_coarsen": (C.c_int, [_vp, C.c_int, _P(_vp)]),
    "pnp_mesh_transfer": (C.c_int, [_vp, _vp, _P(_i64), _vp, _vp, _vp, _vp]),
    "pnp_element_gradient": (C.c_int, [_vp, _vp, _vp]),
    "pnp_mesh_info": (C.c_int, [_vp, _P(C.c_int), _P(C.c_int), _P(_i64), _P(_i64), _P(_i64)]),
    "pnp_mesh_node_coords": (C.c_int, [_vp, _vp]),
    "pnp_mesh_hanging": (C.c_int, [_vp, _vp]),
    "pnp_mesh_elements": (C.c_int, [_vp, _vp, _vp]),
    "pnp_mesh_patch_stats": (C.c_int, [_vp, _vp]),
    "pnp_ctx_create": (C.c_int, [_vp, _P(pnp_params), _vp, _P(_vp)]),
    "pnp_ctx_destroy": (None, [_vp]),
    "pnp_set_params": (C.c_int, [_vp, _P(pnp_params)]),
    "pnp_get_params": (C.c_int, [_vp, _P(pnp_params)]),
    "pnp_set_bc": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, _d]),
    "pnp_set_field": (C.c_int, [_vp, C.c_int, _vp, C.c_int]),
    "pnp_get_field": (C.c_int, [_vp, C.c_int, _vp, C.c_int]),
    "pnp_make_consistent": (C.c_int, [_vp]),
    "pnp_residual": (C.c_int, [_vp, _vp, _vp]),
    "pnp_jv": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int]),
    "pnp_linearize": (C.c_int, [_vp, _vp]),
    "pnp_jv_linearized": (C.c_int, [_vp, _vp, _vp]),
    "pnp_block_diag": (C.c_int, [_vp, _vp, _vp]),
    "pnp_block_diag_f32": (C.c_int, [_vp, _vp, _vp]),
    "pnp_boundary_flux": (C.c_int, [_vp, _vp, C.c_int, _vp]),
    "pnp_plane_average": (C.c_int, [_vp, _vp, C.c_int, _i64, _vp]),
    "pnp_norm2": (C.c_int, [_vp, _vp, _i64, _P(_d)]),
    "pnp_gmres": (C.c_int, [_vp, _vp, _vp, _vp, _d, C.c_int, _P(pnp_solve_stats)]),
    "pnp_newton_solve": (C.c_int, [_vp, _P(pnp_solve_stats)]),
    "pnp_time_step": (C.c_int, [_vp, _P(pnp_solve_stats)]),
    "pnp_ns_set_bc": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int, _d]),
    "pnp_ns_residual": (C.c_int, [_vp, _vp, _vp]),
    "pnp_ns_matvec": (C.c_int, [_vp, _vp, _vp, C.c_int]),
    "pnp_ns_block_diag": (C.c_int, [_vp, _vp]),
    "pnp_ns_solve": (C.c_int, [_vp, _P(pnp_ns_stats)]),
    "pnp_coupled_step": (C.c_int, [_vp, _P(pnp_solve_stats), _P(pnp_ns_stats)]),
    "pnp_step_count": (C.c_int, [_vp, _P(_i64)]),
    "pnp_set_step_count": (C.c_int, [_vp, _i64]),
    "pnp_set_wait_limit": (C.c_int, [_vp, _i64]),
    "pnp_reset_history": (C.c_int, [_vp]),
    "pnp_profile_enable": (C.c_int, [_vp, C.c_int]),
    "pnp_profile_read": (C.c_int, [_vp, C.c_int, _P(_d), _P(_i64), _P(_d), _P(_d)]),
    "pnp_kernel_launches": (_i64, []),
    "pnp_graph_captures": (_i64, []),
    "pnp_mlp_init": (C.c_int, [_vp, C.c_uint64]),
    "pnp_mlp_set_weights": (C.c_int, [_vp, _vp, _i64]),
    "pnp_mlp_get_weights": (C.c_int, [_vp, _vp, _i64]),
    "pnp_mlp_set_normalization": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "pnp_mlp_get_normalization": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "pnp_mlp_add_trajectory": (C.c_int, [_vp, _vp, _i64, _vp]),
    "pnp_mlp_clear_data": (C.c_int, [_vp]),
    "pnp_mlp_train": (C.c_int, [_vp, _P(pnp_train_cfg), _P(pnp_train_stats)]),
    "pnp_mlp_features": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "pnp_mlp_forward": (C.c_int, [_vp, _vp, _i64, _vp]),
    "pnp_mlp_loss_grad": (C.c_int, [_vp, _vp, _vp, _i64, _vp, _P(_d)]),
    "pnp_mlp_forward_noalloc": (C.c_int, [_vp, _vp, _i64, _vp, _vp]),
    "pnp_mlp_adam_step": (C.c_int, [_vp, _vp, _P(pnp_train_cfg)]),
    "pnp_mlp_get_adam_state": (C.c_int, [_vp, _vp, _vp, _P(_i64)]),
}

PNP_NOALLOC_MAX_ROWS = 4096


def mlp_forward_noalloc(params, X, Y, stream: int = 0):
    """Allocation-free network forward (no context); params/X/Y device FP32 tensors."""
    check(lib().pnp_mlp_forward_noalloc(_ptr(params), _ptr(X), int(X.shape[0]), _ptr(Y), C.c_void_p(stream)))
    return Y

PNP_PROF_RESIDUAL, PNP_PROF_JV64, PNP_PROF_JV32, PNP_PROF_BLOCKDIAG = 0, 1, 2, 3
PNP_PROF_ORTHO, PNP_PROF_PRECOND, PNP_PROF_MLP = 4, 5, 6
PNP_PROF_ORTHO_UPDATE, PNP_PROF_INNER, PNP_PROF_MG = 7, 8, 9
PNP_PROF_NS, PNP_PROF_NS32, PNP_PROF_NS_KRYLOV, PNP_PROF_KINDS = 10, 11, 12, 13
PROF_NAMES = ["residual64", "jv64", "jv32", "blockdiag", "ortho_dot", "precond", "mlp", "ortho_update", "inner_ortho",
              "mg_coarse", "ns64", "ns32", "ns_krylov"]


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            if hasattr(L, name):
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
        _lib = L
    return _lib


def register(name, restype, argtypes):
    """Declare the signature of an additional entry point (used by sibling modules)."""
    SIGNATURES[name] = (restype, argtypes)
    if _lib is not None and hasattr(_lib, name):
        fn = getattr(_lib, name)
        fn.restype = restype
        fn.argtypes = argtypes


def check(rc: int):
    if rc != PNP_OK:
        raise PnpError(rc, lib().pnp_last_error().decode())


def default_params(**kw) -> pnp_params:
    p = pnp_params()
    lib().pnp_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(f"pnp_params has no field {k}")
        setattr(p, k, v)
    return p


def _ptr(x):
    """Pointer of a torch tensor (device or host) or numpy array."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if not x.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return x.data_ptr()


class Mesh:
    """Q1 mesh of a 2:1-balanced octree (owns a pnp_mesh handle).  ``octants.periodic``
    (bit k: axis k periodic, default 0) selects periodic sides.  With ``target_levels``
    (uint8 per octant) the octants are first refined to those levels and 2:1 balanced
    (pnp_mesh_create_refined); ``elements()`` then returns the resulting leaves."""

    def __init__(self, octants=None, target_levels=None, _handle=None):
        if _handle is not None:
            self._wrap(_handle)
            return
        a = np.ascontiguousarray(octants.anchors, dtype=np.int32)
        lv = np.ascontiguousarray(octants.levels, dtype=np.uint8)
        h = C.c_void_p()
        self.periodic = int(getattr(octants, "periodic", 0))
        if target_levels is None:
            check(lib().pnp_mesh_create_periodic(octants.dim, octants.max_level, octants.n, a.ctypes.data,
                                                 lv.ctypes.data, self.periodic, C.byref(h)))
        else:
            t = np.ascontiguousarray(target_levels, dtype=np.uint8)
            if t.shape != (octants.n,):
                raise ValueError("target_levels needs one level per octant")
            check(lib().pnp_mesh_create_refined(octants.dim, octants.max_level, octants.n, a.ctypes.data,
                                                lv.ctypes.data, t.ctypes.data, self.periodic, C.byref(h)))
        self._wrap(h)

    def _wrap(self, h):
        self.periodic = getattr(self, "periodic", 0)
        self.h = h
        d, L = C.c_int(), C.c_int()
        ne, nn, nh = C.c_int64(), C.c_int64(), C.c_int64()
        check(lib().pnp_mesh_info(h, C.byref(d), C.byref(L), C.byref(ne), C.byref(nn), C.byref(nh)))
        self.dim, self.max_level = d.value, L.value
        self.n_elem, self.n_nodes, self.n_hanging = ne.value, nn.value, nh.value
        self.ijk = np.zeros((self.n_nodes, self.dim), np.int32)
        check(lib().pnp_mesh_node_coords(h, self.ijk.ctypes.data))
        hf = np.zeros(self.n_nodes, np.uint8)
        check(lib().pnp_mesh_hanging(h, hf.ctypes.data))
        self.hanging = hf.astype(bool)

    def coarsen(self, cap_level: int) -> "Mesh":
        """The octree with every leaf finer than cap_level replaced by its ancestor there."""
        h = C.c_void_p()
        check(lib().pnp_mesh_coarsen(self.h, int(cap_level), C.byref(h)))
        return Mesh(_handle=h)

    def transfer(self, coarse: "Mesh"):
        """Prolongation CSR (ptr, col, w) from `coarse` to this mesh and the injection map."""
        nnz = C.c_int64()
        check(lib().pnp_mesh_transfer(self.h, coarse.h, C.byref(nnz), None, None, None, None))
        ptr = np.zeros(self.n_nodes + 1, np.int64)
        col = np.zeros(nnz.value, np.int32)
        w = np.zeros(nnz.value, np.float32)
        inj = np.zeros(coarse.n_nodes, np.int32)
        check(lib().pnp_mesh_transfer(self.h, coarse.h, C.byref(nnz), ptr.ctypes.data, col.ctypes.data,
                                      w.ctypes.data, inj.ctypes.data))
        return ptr, col, w, inj

    def patch_stats(self) -> dict:
        s = np.zeros(7, np.int64)
        check(lib().pnp_mesh_patch_stats(self.h, s.ctypes.data))
        keys = ["patches", "max_nodes", "max_colors", "shared_nodes", "partials", "slots", "violations"]
        return dict(zip(keys, s.tolist()))

    def elements(self):
        a = np.zeros((self.n_elem, self.dim), np.int32)
        lv = np.zeros(self.n_elem, np.uint8)
        check(lib().pnp_mesh_elements(self.h, a.ctypes.data, lv.ctypes.data))
        return a, lv

    def close(self):
        if getattr(self, "h", None):
            lib().pnp_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """A solver context on the current CUDA device (owns a pnp_ctx handle).

    ``stream`` is a raw cudaStream_t handle (int); torch users pass
    ``torch.cuda.current_stream().cuda_stream``.
    """

    def __init__(self, mesh: Mesh, params: pnp_params, stream: int = 0):
        h = C.c_void_p()
        check(lib().pnp_ctx_create(mesh.h, C.byref(params), C.c_void_p(stream), C.byref(h)))
        self.h = h
        self.mesh = mesh
        self.dim = mesh.dim
        self.n_nodes = mesh.n_nodes

    def close(self):
        if getattr(self, "h", None):
            lib().pnp_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # parameters / BCs / fields
    def set_params(self, p: pnp_params):
        check(lib().pnp_set_params(self.h, C.byref(p)))

    def get_params(self) -> pnp_params:
        p = pnp_params()
        check(lib().pnp_get_params(self.h, C.byref(p)))
        return p

    def set_bc(self, face: int, field: int, kind: int, value: float):
        check(lib().pnp_set_bc(self.h, face, field, kind, value))

    def set_bcs(self, bcs):
        for f in range(bcs.types.shape[0]):
            for k in range(3):
                self.set_bc(f, k, int(bcs.types[f, k]), float(bcs.values[f, k]))

    def set_field(self, which: int, x, where: int | None = None):
        if where is None:
            where = PNP_HOST if isinstance(x, np.ndarray) else PNP_DEVICE
        if isinstance(x, np.ndarray):
            x = np.ascontiguousarray(x, dtype=np.float64)
        check(lib().pnp_set_field(self.h, which, _ptr(x), where))

    def get_field(self, which: int, out=None, where: int | None = None):
        ncomp = 4 if which == PNP_FIELD_NS else (self.dim if which >= PNP_FIELD_ADVECTION else 3)
        if out is None:
            out = np.zeros((self.n_nodes, ncomp))
        if where is None:
            where = PNP_HOST if isinstance(out, np.ndarray) else PNP_DEVICE
        check(lib().pnp_get_field(self.h, which, _ptr(out), where))
        return out

    def make_consistent(self):
        check(lib().pnp_make_consistent(self.h))

    # operators (device pointers: torch CUDA tensors)
    def residual(self, U, F):
        check(lib().pnp_residual(self.h, _ptr(U), _ptr(F)))
        return F

    def jv(self, U, V, JV, precision: int = PNP_F64):
        check(lib().pnp_jv(self.h, _ptr(U), _ptr(V), _ptr(JV), precision))
        return JV

    def linearize(self, U):
        check(lib().pnp_linearize(self.h, _ptr(U)))

    def jv_linearized(self, V, JV):
        check(lib().pnp_jv_linearized(self.h, _ptr(V), _ptr(JV)))
        return JV

    def block_diag(self, U, D):
        """D [n][9]: FP64 blocks, or FP32 blocks (FP32 arithmetic) when D is float32."""
        fn = lib().pnp_block_diag_f32 if str(D.dtype) == "torch.float32" else lib().pnp_block_diag
        check(fn(self.h, _ptr(U), _ptr(D)))
        return D

    def boundary_flux(self, U, face: int) -> np.ndarray:
        """[int_face n.(grad c+ + c+ grad phi), int_face n.(grad c- - c- grad phi)] over a
        boundary face (outward normal n); U a device FP64 [n][3] tensor."""
        out = np.zeros(2)
        check(lib().pnp_boundary_flux(self.h, _ptr(U), int(face), out.ctypes.data))
        return out

    def boundary_current(self, U, face: int) -> float:
        """Net species flux through a face, j = -(flux_+ - flux_-) / |face| (Sec. 5.2)
        on the unit domain."""
        f = self.boundary_flux(U, face)
        return -(f[0] - f[1])

    def element_gradient(self, U, G):
        """G [n_elem][3] (device FP64): |grad c+|, |grad c-|, |grad phi| at element centres."""
        check(lib().pnp_element_gradient(self.h, _ptr(U), _ptr(G)))
        return G

    def plane_average(self, U, axis: int, coord: int) -> np.ndarray:
        """Averages of (c+, c-, phi) over the plane x_axis = coord 2^-max_level."""
        out = np.zeros(3)
        check(lib().pnp_plane_average(self.h, _ptr(U), int(axis), int(coord), out.ctypes.data))
        return out

    def averaged_profile(self, U, axis: int, coords) -> np.ndarray:
        """[len(coords)][3] plane averages along `axis` (the x-averaged profiles of
        Sec. 5.2 when `axis` is the wall-normal axis and `coords` its node levels)."""
        return np.array([self.plane_average(U, axis, int(z)) for z in coords])

    def norm2(self, x) -> float:
        r = C.c_double()
        check(lib().pnp_norm2(self.h, _ptr(x), int(x.numel()), C.byref(r)))
        return r.value

    def gmres(self, U, b, x, rtol: float, precision: int = PNP_F64, raise_on_error=True):
        st = pnp_solve_stats()
        rc = lib().pnp_gmres(self.h, _ptr(U), _ptr(b), _ptr(x), rtol, precision, C.byref(st))
        if raise_on_error:
            check(rc)
        return st

    def newton_solve(self, raise_on_error=True) -> pnp_solve_stats:
        st = pnp_solve_stats()
        rc = lib().pnp_newton_solve(self.h, C.byref(st))
        if raise_on_error:
            check(rc)
        return st

    def time_step(self, raise_on_error=True) -> pnp_solve_stats:
        st = pnp_solve_stats()
        rc = lib().pnp_time_step(self.h, C.byref(st))
        if raise_on_error:
            check(rc)
        return st

    def reset_history(self):
        check(lib().pnp_reset_history(self.h))

    # ---------------------------------------------------------------- Navier-Stokes
    def ns_set_bc(self, face: int, slot: int, typ: int, value: float = 0.0):
        check(lib().pnp_ns_set_bc(self.h, face, slot, typ, float(value)))

    def ns_set_bcs(self, types, values):
        """types / values: [2*dim, 4] per face and slot (v_x, v_y, v_z, p)."""
        for f in range(len(types)):
            for k in range(4):
                self.ns_set_bc(f, k, int(types[f][k]), float(values[f][k]))

    def ns_residual(self, X, F):
        check(lib().pnp_ns_residual(self.h, _ptr(X), _ptr(F)))
        return F

    def ns_matvec(self, X, Y, precision: int = PNP_F64):
        check(lib().pnp_ns_matvec(self.h, _ptr(X), _ptr(Y), precision))
        return Y

    def ns_block_diag(self, D):
        check(lib().pnp_ns_block_diag(self.h, _ptr(D)))
        return D

    def ns_solve(self, raise_on_error=True) -> pnp_ns_stats:
        st = pnp_ns_stats()
        rc = lib().pnp_ns_solve(self.h, C.byref(st))
        if raise_on_error:
            check(rc)
        return st

    def coupled_step(self, raise_on_error=True):
        """One NS-PNP step (block iteration): (PNP stats, NS stats)."""
        st, nst = pnp_solve_stats(), pnp_ns_stats()
        rc = lib().pnp_coupled_step(self.h, C.byref(st), C.byref(nst))
        if raise_on_error:
            check(rc)
        return st, nst

    def set_wait_limit(self, polls: int):
        check(lib().pnp_set_wait_limit(self.h, int(polls)))

    def set_step_count(self, k: int):
        check(lib().pnp_set_step_count(self.h, int(k)))

    def step_count(self) -> int:
        k = C.c_int64()
        check(lib().pnp_step_count(self.h, C.byref(k)))
        return k.value

    def profile_enable(self, on: bool = True):
        check(lib().pnp_profile_enable(self.h, int(on)))

    def profile_read(self) -> dict:
        out = {}
        for k, name in enumerate(PROF_NAMES):
            ms, cnt, by, fl = C.c_double(), C.c_int64(), C.c_double(), C.c_double()
            check(lib().pnp_profile_read(self.h, k, C.byref(ms), C.byref(cnt), C.byref(by), C.byref(fl)))
            out[name] = {"ms": ms.value, "count": cnt.value, "alg_bytes": by.value, "alg_flops": fl.value}
        return out


    # ---------------------------------------------------------------- learned start
    def mlp_init(self, seed: int = 0):
        check(lib().pnp_mlp_init(self.h, seed))

    def mlp_set_weights(self, params: np.ndarray):
        p = np.ascontiguousarray(params, dtype=np.float32)
        check(lib().pnp_mlp_set_weights(self.h, p.ctypes.data, p.size))

    def mlp_get_weights(self) -> np.ndarray:
        p = np.zeros(PNP_MLP_PARAMS, np.float32)
        check(lib().pnp_mlp_get_weights(self.h, p.ctypes.data, p.size))
        return p

    def mlp_set_normalization(self, in_mean, in_std, out_mean, out_std):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (in_mean, in_std, out_mean, out_std)]
        check(lib().pnp_mlp_set_normalization(self.h, *[a.ctypes.data for a in arrs]))

    def mlp_get_normalization(self):
        arrs = [np.zeros(4), np.zeros(4), np.zeros(3), np.zeros(3)]
        check(lib().pnp_mlp_get_normalization(self.h, *[a.ctypes.data for a in arrs]))
        return arrs

    def mlp_add_trajectory(self, states, uz=None):
        """states: device FP64 tensor [T, n_nodes, 3]; uz: device [T, n_nodes] or None."""
        check(lib().pnp_mlp_add_trajectory(self.h, _ptr(states), int(states.shape[0]), _ptr(uz)))

    def mlp_clear_data(self):
        check(lib().pnp_mlp_clear_data(self.h))

    def mlp_train(self, steps=2000, batch=4096, lr=1e-3, seed=0, beta1=0.9, beta2=0.999, adam_eps=1e-8):
        cfg = pnp_train_cfg(steps, batch, lr, beta1, beta2, adam_eps, seed)
        st = pnp_train_stats()
        check(lib().pnp_mlp_train(self.h, C.byref(cfg), C.byref(st)))
        return st

    def mlp_adam_step(self, grad, lr=1e-3, beta1=0.9, beta2=0.999, adam_eps=1e-8):
        """One Adam update of the parameters with a device FP32 gradient [PNP_MLP_PARAMS]."""
        cfg = pnp_train_cfg(0, 1, lr, beta1, beta2, adam_eps, 0)
        check(lib().pnp_mlp_adam_step(self.h, _ptr(grad), C.byref(cfg)))

    def mlp_adam_state(self):
        """(m, v, t): Adam moments (host FP32 [PNP_MLP_PARAMS]) and step count."""
        m = np.zeros(PNP_MLP_PARAMS, np.float32)
        v = np.zeros(PNP_MLP_PARAMS, np.float32)
        t = C.c_int64()
        check(lib().pnp_mlp_get_adam_state(self.h, m.ctypes.data, v.ctypes.data, C.byref(t)))
        return m, v, t.value

    def mlp_features(self, Uk, Ukm1, uzk=None, uzkm1=None, X=None, nodes=None):
        check(lib().pnp_mlp_features(self.h, _ptr(Uk), _ptr(Ukm1), _ptr(uzk), _ptr(uzkm1), _ptr(X), _ptr(nodes)))
        return X, nodes

    def mlp_forward(self, X, Y):
        check(lib().pnp_mlp_forward(self.h, _ptr(X), int(X.shape[0]), _ptr(Y)))
        return Y

    def mlp_loss_grad(self, X, Yt, grad):
        loss = C.c_double()
        check(lib().pnp_mlp_loss_grad(self.h, _ptr(X), _ptr(Yt), int(X.shape[0]), _ptr(grad), C.byref(loss)))
        return loss.value


def kernel_launches() -> int:
    return int(lib().pnp_kernel_launches())


def graph_captures() -> int:
    return int(lib().pnp_graph_captures())
