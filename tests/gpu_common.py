"""Shared helpers of the GPU parity tests: build/load the library, map node orders."""
import numpy as np

import oracle as O
from paper_2301_05985_gb300 import workloads as W

_built = False


def lib():
    global _built
    from paper_2301_05985_gb300 import build as B
    if not _built:
        B.build()
        _built = True
    from paper_2301_05985_gb300 import pnp
    return pnp


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU test needs CUDA"
    return torch


def perm_to_oracle(ijk_lib, ijk_ora, max_level):
    """perm[i] = oracle index of library node i (matched by integer coordinates)."""
    base = (1 << max_level) + 1
    def key(ijk):
        k = np.zeros(ijk.shape[0], np.int64)
        for a in range(ijk.shape[1]):
            k += ijk[:, a].astype(np.int64) * base**a
        return k
    kl, ko = key(ijk_lib), key(ijk_ora)
    order = np.argsort(ko)
    pos = np.searchsorted(ko[order], kl)
    perm = order[pos]
    assert np.array_equal(ko[perm], kl)
    return perm


class Pair:
    """A library context and the oracle mesh of the same octants, with node maps."""

    def __init__(self, octants, params_kw, bcs, stream=0):
        self.pnp = lib()
        self.torch = torch_cuda()
        self.oc = octants
        self.mesh = self.pnp.Mesh(octants)
        self.om = O.OracleMesh(octants)
        self.perm = perm_to_oracle(self.mesh.ijk, self.om.ijk, octants.max_level)  # lib -> oracle
        self.dim = octants.dim
        self.bcs = bcs
        self.params_kw = dict(params_kw)
        self.params = self.pnp.default_params(**params_kw)
        self.ctx = self.pnp.Context(self.mesh, self.params, stream)
        self.ctx.set_bcs(bcs)
        kw = dict(eps=params_kw["eps"], dt=params_kw.get("dt", 1.0),
                  beta=(params_kw.get("beta0", 1.0), params_kw.get("beta1", -1.0), params_kw.get("beta2", 0.0)),
                  C_I=params_kw.get("C_I", 6.0), steady=bool(params_kw.get("steady", 0)),
                  bc_type=bcs.types, bc_val=bcs.values)
        self.op = O.Params(**kw)

    # library-order arrays <-> oracle-order arrays
    def to_ora(self, x_lib):
        out = np.zeros_like(x_lib)
        out[self.perm] = x_lib
        return out

    def to_lib(self, x_ora):
        return x_ora[self.perm]

    def dev(self, x):
        return self.torch.from_numpy(np.ascontiguousarray(x)).cuda()

    def set_state(self, Uk=None, Ukm1=None, vel=None):
        n = self.mesh.n_nodes
        self.Uk = np.zeros((n, 3)) if Uk is None else Uk
        self.Ukm1 = np.zeros((n, 3)) if Ukm1 is None else Ukm1
        self.vel = np.zeros((n, self.dim)) if vel is None else vel
        self.ctx.set_field(self.pnp.PNP_FIELD_U_PREV, self.Uk)
        self.ctx.set_field(self.pnp.PNP_FIELD_U_PREV2, self.Ukm1)
        self.ctx.set_field(self.pnp.PNP_FIELD_ADVECTION, self.vel)

    def oracle_residual(self, U):
        return self.to_lib(self.om.residual(self.op, self.to_ora(U), self.to_ora(self.Uk), self.to_ora(self.Ukm1),
                                            self.to_ora(self.vel)))

    def oracle_jacobian(self, U):
        J = self.om.jacobian(self.op, self.to_ora(U), self.to_ora(self.Uk), self.to_ora(self.Ukm1),
                             self.to_ora(self.vel))
        # permute to library order: row/col index 3*i+f
        p3 = (3 * self.perm[:, None] + np.arange(3)[None, :]).reshape(-1)
        return J[p3][:, p3]

    def oracle_jv(self, U, V):
        return self.to_lib(self.om.jv(self.op, self.to_ora(U), self.to_ora(V), self.to_ora(self.Uk),
                                      self.to_ora(self.Ukm1), self.to_ora(self.vel)))

    def gpu_residual(self, U):
        Ud = self.dev(U)
        F = self.torch.zeros_like(Ud)
        self.ctx.residual(Ud, F)
        return F.cpu().numpy()

    def gpu_jv(self, U, V, precision=0):
        Ud = self.dev(U)
        if precision == 0:
            Vd = self.dev(V)
            JV = self.torch.zeros_like(Vd)
        else:
            Vd = self.dev(V.astype(np.float32))
            JV = self.torch.zeros_like(Vd)
        self.ctx.jv(Ud, Vd, JV, precision)
        return JV.cpu().numpy().astype(np.float64)


def rel_err(x, ref):
    return np.linalg.norm(x - ref) / np.linalg.norm(ref)


def field_max_err(x, ref):
    """max_i |x - ref| / max_i |ref| per field (0 where ref vanishes identically)."""
    out = []
    for f in range(3):
        s = np.abs(ref[:, f]).max()
        out.append(np.abs(x[:, f] - ref[:, f]).max() / s if s > 0 else np.abs(x[:, f]).max())
    return np.array(out)


def problem_cases():
    """(name, octants, params, bcs, transient) used by several parity tests."""
    return [
        ("2d_uniform_steady", W.uniform_octants(2, 4), dict(eps=0.05, steady=1), W.equilibrium_bcs(2, 1.0)),
        ("2d_octree_transient", W.random_balanced_octants(2, 2, 5, 0.3, 11),
         dict(eps=0.02, dt=0.01, beta0=1.5, beta1=-2.0, beta2=0.5), W.membrane_bcs(2, 5.0, 2.0)),
        ("3d_uniform_transient", W.uniform_octants(3, 3),
         dict(eps=0.01, dt=1e-3, beta0=1.5, beta1=-2.0, beta2=0.5), W.membrane_bcs(3, 20.0, 2.0)),
        ("3d_octree_transient", W.random_balanced_octants(3, 1, 4, 0.3, 12),
         dict(eps=0.03, dt=0.02, beta0=1.0, beta1=-1.0, beta2=0.0), W.membrane_bcs(3, 3.0, None)),
        ("3d_octree_steady", W.random_balanced_octants(3, 2, 4, 0.25, 13), dict(eps=0.1, steady=1),
         W.equilibrium_bcs(3, 2.0)),
    ]
