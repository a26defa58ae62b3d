"""Benchmark: NS-PNP time steps on the 3D electroconvection octree.

Workload (the 3D electroconvection configuration, octree levels 6-10): unit cube;
membrane at z = 0 (phi = 0, c+ = 2, c- zero flux), reservoir at z = 1 (phi = V, c+- = 1),
zero-flux side walls, no-slip walls for the fluid; Lambda = 5e-4, V = 40, dt = 5e-4,
Sc = 1, kappa = 0.5; c+- = 1 + seeded uniform noise of amplitude 1e-3, phi linear, fluid
at rest.  The octree is solution-adaptive (paper_2301_05985_gb300.refine): base level 6, a
PNP pre-solve (3 steps) on a level-8 band z < 0.01, then level 9 for every octant with
z_min < 0.01 and level 10 wherever max |grad c+-| at the octant centre exceeds 60 (the
Debye layer), 2:1 balanced: 5.6 M elements, 6.67 M nodes, 20.0 M PNP unknowns and 26.7 M
NS unknowns.

One step = one pnp_coupled_step (Sec. 4.1, one block iteration): the semi-implicit VMS
Navier-Stokes block (linear in v, p; FGMRES in FP64 right-preconditioned by an FP32
multigrid V-cycle on the octree hierarchy, to ||F|| <= 1e-8 ||F(X^0)||) with the body
force of U^k, then the PNP block's pnp_time_step with v^{k+1} as the advection: BDF2
(BDF1 first), Newton to ||F|| <= 1e-8 ||F(U^k)||.
  mixed (timed): inexact Newton (Eisenstat-Walker) with flexible GMRES(60) in FP64 (dots,
        orthogonalisation, basis) preconditioned by 24 steps of FP32 GMRES on J M^-1 (FP32
        J V, M the 3x3 block Jacobi); FP64 residual; learned start (network trained before
        the timed region on the first steps of this run), judged against 2 U^k - U^{k-1}.
  FP64 arms, from the state the timed steps start from (the NS block solved the same way):
        plain_same_solver: the same nested PNP solver and forcing entirely in FP64;
        plain_gmres: FP64 J V, GMRES(100) + block Jacobi to rtol 1e-8 per Newton step
        (exact Newton), previous-step start (the paper's solver settings).
  --pnp-only times the PNP block's step alone (fluid at rest).

value = seconds per step of the timed mixed steps (CUDA events on the library's stream);
replicas: the slowest rank's time over the steps all ranks took.  The J V kernel's roofline
uses the algorithmic work per unit of the FP32 J V (56 B per node, 36 B per element,
2.5 kFLOP per element); its binding bound is the larger of the HBM time and the FP32 ALU
time of that work (FP32 peak 152 SMs x 128 FMA/clk x 2 x 2.07 GHz).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
for _p in (ROOT, os.path.join(ROOT, "oracle")):
    if _p not in sys.path:
        sys.path.insert(0, _p)

METRIC = "PNP Jv GDoF/s (% HBM peak); s per PNP–NS step at rel-resid 1e-8, plain vs mixed+learned"
# ALU peaks: 152 SMs x (2 FP64 | 128 FP32) FMA per clock x 2 flop x 2.07 GHz
FP64_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# algorithmic work of the J V per unit (the FP32 / FP64 J V rows of the measurement plan)
JV_BYTES_PER_NODE = {"jv32": 56.0, "jv64": 112.0}
JV_BYTES_PER_ELEM = 36.0
JV_FLOPS_PER_ELEM = 2500.0
# arithmetic of each kernel class; for ALU classes the binding roofline is chosen per run
BOUNDS = {"residual64": "fp32", "jv64": "fp64", "jv32": "fp32", "blockdiag": "fp32", "ortho_dot": "fp64",
          "ortho_update": "fp64", "precond": "hbm", "mlp": "bf16", "inner_ortho": "hbm", "ns64": "fp32",
          "ns32": "fp32", "ns_krylov": "hbm", "mg_coarse": "hbm"}
# the Navier-Stokes block (the configurations give neither Sc nor kappa): Sc = 1, kappa = 0.5,
# multigrid-preconditioned FP32 BiCGStab under FP64 refinement, App. A's tolerances
NS_KW = dict(ns_Sc=1.0, ns_kappa=0.5, ns_mg_levels=8, mg_smooth=3, mg_omega=0.6, mg_coarse_its=32,
             ns_rtol=1e-8, ns_atol=1e-10, ns_blocks=1, ns_fgmres=50)

WORKLOADS = {
    "electroconvection": {"eps": 5e-4, "V": 40.0, "dt": 5e-4,
                          "desc": "3D electroconvection octree, levels 6-10: level 9 for z<0.01, level 10 where "
                                  "the pre-solve's |grad c| > 60 (Debye layer), 2:1 balanced"},
    "membrane": {"eps": 1e-3, "V": 20.0, "dt": 1e-3,
                 "desc": "3D membrane-band octree, base level 5, level 8 for z<0.05 (2:1 graded)"},
    "small": {"eps": 2e-3, "V": 20.0, "dt": 1e-3,
              "desc": "membrane-band octree, base level 4, level 7 for z<0.05 (profiling miniature)"},
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="electroconvection", choices=list(WORKLOADS))
    ap.add_argument("--small", action="store_true", help="alias of --workload small (profiling captures)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--plain", action="store_true",
                    help="run the FP64 comparison arms on the main workload too (they always run on the "
                         "membrane-band secondary workload)")
    ap.add_argument("--plain-steps", type=int, default=1, help="steps of each FP64 arm on the main workload")
    ap.add_argument("--e2e-steps", type=int, default=5, help="timed steps re-run end to end (the first ones)")
    ap.add_argument("--no-mg", action="store_true", help="skip the multigrid-preconditioned comparison arm")
    ap.add_argument("--mg-steps", type=int, default=5, help="steps of the multigrid arm")
    ap.add_argument("--no-sweep", action="store_true", help="skip the J V sweep on the uniform level-7 cube")
    ap.add_argument("--no-secondary", action="store_true", help="skip the membrane-band secondary run")
    ap.add_argument("--no-learned", action="store_true", help="mixed mode without training the learned start")
    ap.add_argument("--record-steps", type=int, default=0,
                    help="trajectory steps recorded for training (0: the warm-up steps are the recording)")
    ap.add_argument("--train-steps", type=int, default=600, help="Adam steps of the learned start")
    ap.add_argument("--profile-steps", type=int, default=3, help="further steps timed per kernel class")
    ap.add_argument("--pnp-only", action="store_true",
                    help="time the PNP block's step alone (fluid at rest, no Navier-Stokes block)")
    a = ap.parse_args()
    if a.small:
        a.workload = "small"
    return a


def build_workload(pnp, torch, name):
    """Octants (and target levels) of a workload; the refinement recipe runs its pre-solve."""
    from paper_2301_05985_gb300 import workloads as W
    if name == "electroconvection":
        from paper_2301_05985_gb300 import refine as R
        wl = WORKLOADS[name]
        t0 = time.perf_counter()
        oc, target, info = R.gradient_refined_octants(pnp, torch, torch.cuda.current_stream().cuda_stream,
                                                      R.RefineRecipe(), wl["eps"], wl["V"], wl["dt"])
        info["build_s"] = time.perf_counter() - t0
        return oc, target, info
    if name == "membrane":
        return W.membrane_band_octants(5, 8, 0.05), None, {}
    return W.membrane_band_octants(4, 7, 0.05), None, {}


def mode_params(pnp, wl, mode, learned=True):
    p = _mode_params(pnp, wl, mode, learned)
    for k, v in NS_KW.items():
        setattr(p, k, v)
    return p


def _mode_params(pnp, wl, mode, learned=True):
    if mode == "mixed":
        return pnp.default_params(eps=wl["eps"], dt=wl["dt"], precision=pnp.PNP_F32,
                                  start_mode=pnp.PNP_START_LEARNED if learned else pnp.PNP_START_EXTRAPOLATE,
                                  newton_rtol=1e-8, gmres_restart=60, gmres_max_it=3000, dt_retries=2,
                                  gmres_inner=24)
    if mode == "mixed_mg":
        return pnp.default_params(eps=wl["eps"], dt=wl["dt"], precision=pnp.PNP_F32,
                                  start_mode=pnp.PNP_START_EXTRAPOLATE, newton_rtol=1e-8, gmres_restart=60,
                                  gmres_max_it=3000, dt_retries=2, gmres_inner=24, mg_levels=8, mg_smooth=3,
                                  mg_omega=0.6, mg_coarse_its=32)
    if mode == "same64":
        return pnp.default_params(eps=wl["eps"], dt=wl["dt"], precision=pnp.PNP_F64,
                                  start_mode=pnp.PNP_START_EXTRAPOLATE, newton_rtol=1e-8, gmres_restart=60,
                                  gmres_max_it=3000, dt_retries=2, gmres_inner=24, newton_ew_f64=1)
    return pnp.default_params(eps=wl["eps"], dt=wl["dt"], precision=pnp.PNP_F64, start_mode=pnp.PNP_START_PREVIOUS,
                              newton_rtol=1e-8, gmres_rtol=1e-8, gmres_restart=100, gmres_max_it=4000,
                              dt_retries=2)


def make_ctx(pnp, W, torch, mesh, wl, mode, learned=True):
    ctx = pnp.Context(mesh, mode_params(pnp, wl, mode, learned), torch.cuda.current_stream().cuda_stream)
    ctx.set_bcs(W.membrane_bcs(3, wl["V"], 2.0))
    bt = np.zeros((6, 4), np.int32)
    bt[:, :3] = pnp.PNP_DIRICHLET  # no-slip walls
    ctx.ns_set_bcs(bt, np.zeros((6, 4)))
    U0 = W.noisy_state(mesh.ijk, mesh.max_level, seed=0, amp=1e-3, phi_bottom=0.0, phi_top=wl["V"])
    ctx.set_field(pnp.PNP_FIELD_U, U0)
    ctx.make_consistent()
    ctx.reset_history()
    return ctx


def do_step(ctx, coupled, raise_on_error=True):
    """One step: the coupled NS-PNP step (its NS statistics under "ns") or the PNP step."""
    if coupled:
        st, nst = ctx.coupled_step(raise_on_error=raise_on_error)
        d = st.as_dict()
        d["ns"] = nst.as_dict()
        return d
    return ctx.time_step(raise_on_error=raise_on_error).as_dict()


def ns_summary(stats):
    """Per-step means of the NS solves of coupled steps (None for PNP-only steps)."""
    ns = [s["ns"] for s in stats if "ns" in s]
    if not ns:
        return None
    k = len(ns)
    return {"krylov_its_per_step": sum(x["inner_its"] for x in ns) / k,
            "cycles_per_step": sum(x["refinements"] for x in ns) / k,
            "fp32_fine_applications_per_step": sum(x["matvecs32"] for x in ns) / k,
            "fp64_applications_per_step": sum(x["matvecs64"] for x in ns) / k,
            "s_per_step": sum(x["wall_ms"] for x in ns) * 1e-3 / k,
            "rel_res_max": max(x["res_final"] / x["res0"] if x["res0"] > 0 else 0.0 for x in ns),
            "floor_stops": sum(int(x["floor_stop"]) for x in ns), "status": [int(x["status"]) for x in ns]}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "fallback": True}


class ClockSampler:
    """nvidia-smi sampling of SM clocks / throttle reasons while the timed region runs."""

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 4 + i and "Active" in r[4 + i]
                          and "Not" not in r[4 + i]})
        pw = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "samples": len(self.rows), "reasons": reasons}


# ----------------------------------------------------------------------------- oracle timing
def oracle_threads():
    return max(1, os.cpu_count() or 1)


class OracleTimer:
    """The FP64 oracle's residual, matrix-free J V and NS operator on the workload's own mesh
    and state, timed on the host cores: a contiguous sample of the oracle's elements split
    into equal ranges over one thread per core (ctypes releases the interpreter lock), each
    thread adding into a buffer of its own.  Scaled to the whole mesh and to a step's
    operator counts, a timing estimates what the oracle's operator evaluations alone would
    take per step.  The element-range sums reproduce the serial oracle (pinned by a CPU
    test).  The oracle's mesh is built once, outside every timing."""

    def __init__(self, oc, wl, U, Uk, Ukm1, V, sample_frac=0.125, ns_state=None):
        import oracle as O
        t0 = time.perf_counter()
        self.m = m = O.OracleMesh(oc)
        self.build_s = time.perf_counter() - t0
        perm = _perm(m.ijk, U["ijk"], oc.max_level)
        bcs = __import__("paper_2301_05985_gb300.workloads", fromlist=["x"]).membrane_bcs(3, wl["V"], 2.0)
        self.p = O.Params(eps=wl["eps"], dt=wl["dt"], beta=(1.5, -2.0, 0.5), bc_type=bcs.types, bc_val=bcs.values)
        self.Uo, self.Uko, self.Ukm1o, self.Vo = (np.ascontiguousarray(x[perm]) for x in (U["U"], Uk, Ukm1, V))
        self.ns = ns_state is not None
        if self.ns:
            self.nsp = O.NsParams(Sc=NS_KW["ns_Sc"], kappa=NS_KW["ns_kappa"], eps=wl["eps"], dt=wl["dt"],
                                  beta=(1.5, -2.0, 0.5), bc_type=np.ones((6, 4), np.int32), bc_val=np.zeros((6, 4)))
            self.Xo, self.vko, self.vkm1o = (np.ascontiguousarray(ns_state[k][perm]) for k in ("X", "vk", "vkm1"))
            self.advo = 2.0 * self.vko - self.vkm1o
        self.T = T = oracle_threads()
        self.E = E = m.n_elem
        self.Es = Es = max(T, int(E * sample_frac))
        self.cuts = np.linspace(0, Es, T + 1).astype(np.int64)
        self.bufs = [np.zeros((m.n_nodes, 3)) for _ in range(T)]
        self.bufs4 = [np.zeros((m.n_nodes, 4)) for _ in range(T)] if self.ns else None
        self.sample = (f"{Es} of {E} elements ({Es / E:.3f}) in {T} equal ranges, one thread per host core, "
                       f"scaled to the whole mesh")

    def time(self, kind):
        """Seconds of one evaluation of `kind` ("res", "jv", "ns") over the whole mesh."""
        m, cuts = self.m, self.cuts
        for b in self.bufs:
            b[:] = 0.0

        def run(i):
            if kind == "res":
                m.residual_elements(self.p, self.Uo, self.Uko, self.Ukm1o, None, cuts[i], cuts[i + 1], self.bufs[i])
            elif kind == "jv":
                m.jv_elements(self.p, self.Uo, self.Vo, self.Uko, self.Ukm1o, None, cuts[i], cuts[i + 1],
                              self.bufs[i])
            else:
                m.ns_apply_elements(self.nsp, self.Xo, self.advo, self.vko, self.vkm1o, self.Uo, False, cuts[i],
                                    cuts[i + 1], self.bufs4[i])

        th = [threading.Thread(target=run, args=(i,)) for i in range(self.T)]
        t = time.perf_counter()
        for x in th:
            x.start()
        for x in th:
            x.join()
        return (time.perf_counter() - t) * self.E / self.Es

    def step(self, n_res, n_jv, n_ns=0.0):
        """One timed sample of each operator, scaled to a step of the given counts."""
        t = {"res": self.time("res"), "jv": self.time("jv"), "ns": self.time("ns") if self.ns else 0.0}
        t["s_per_step"] = n_res * t["res"] + n_jv * t["jv"] + n_ns * t["ns"]
        return t


def oracle_timing(oc, wl, U, Uk, Ukm1, V, n_res, n_jv, sample_frac=0.125, repeats=3, ns_state=None, n_ns=0.0):
    """OracleTimer's operators, median of `repeats`, scaled to the step's counts."""
    ot = OracleTimer(oc, wl, U, Uk, Ukm1, V, sample_frac, ns_state)
    t_res = statistics.median(ot.time("res") for _ in range(repeats))
    t_jv = statistics.median(ot.time("jv") for _ in range(repeats))
    t_ns = statistics.median(ot.time("ns") for _ in range(repeats)) if ot.ns else 0.0
    dofs = 3.0 * ot.m.n_nodes
    return {"t_residual_s": t_res, "t_jv_s": t_jv, "t_ns_s": t_ns if ot.ns else None,
            "residual_gdofs": dofs / t_res / 1e9, "jv_gdofs": dofs / t_jv / 1e9,
            "s_per_step": n_res * t_res + n_jv * t_jv + n_ns * t_ns, "cores": ot.T,
            "oracle_mesh_build_s": ot.build_s, "sample": ot.sample + f", median of {repeats}"}


def _perm(ijk_ora, ijk_lib, L):
    """perm[i] = library index of oracle node i (matched by integer coordinates)."""
    base = (1 << L) + 1
    key = lambda a: sum(a[:, k].astype(np.int64) * base**k for k in range(a.shape[1]))  # noqa: E731
    kl, ko = key(ijk_lib), key(ijk_ora)
    order = np.argsort(kl)
    return order[np.searchsorted(kl[order], ko)]


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    """The oracle on this workload's mesh and state (host cores), as its arm of the
    comparison.  Each step times one sample of the oracle's residual, J V and NS operator
    (an eighth of the mesh's elements over all host cores) and scales it to the operator
    evaluations of one time step, about the counts of the library's mixed coupled step on
    this workload over 20 steps: 7 residuals, 1,650 J V, and 310 NS operator applications
    (41 FP64 and 6 per FGMRES iteration in the V-cycle on the finest mesh).  `value` is that
    estimate in s/step, `ms_per_step` the sample's own measured wall time per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import torch
    from paper_2301_05985_gb300 import pnp
    from paper_2301_05985_gb300 import workloads as W
    wl = WORKLOADS[args.workload]
    oc, target, _ = build_workload(pnp, torch, args.workload)  # input generation (octree + its pre-solve)
    mesh = pnp.Mesh(oc, target_levels=target)
    oc_full = W.Octants(3, mesh.max_level, *mesh.elements())
    L = mesh.max_level
    U = W.noisy_state(mesh.ijk, L, seed=0, amp=1e-3, phi_bottom=0.0, phi_top=wl["V"])
    Vd = W.random_direction(mesh.ijk, L, 5)
    n_res, n_jv = 7.0, 1650.0
    coupled = not args.pnp_only
    n_ns = 310.0 if coupled else 0.0
    ns_state = {"X": np.zeros((mesh.n_nodes, 4)), "vk": np.zeros((mesh.n_nodes, 3)),
                "vkm1": np.zeros((mesh.n_nodes, 3))} if coupled else None
    ot = OracleTimer(oc_full, wl, {"U": U, "ijk": mesh.ijk}, U, U, Vd, ns_state=ns_state)
    for _ in range(args.warmup):
        ot.step(n_res, n_jv, n_ns)
    t0 = time.perf_counter()
    vals = [ot.step(n_res, n_jv, n_ns)["s_per_step"] for _ in range(args.steps)]
    wall = time.perf_counter() - t0
    v = float(np.mean(vals))
    out = {"metric": METRIC, "value": v, "unit": "s/step", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": workload_config(args.workload, mesh, coupled),
           "value_note": "value = each step's timed sample scaled to the whole mesh and to a step's operator "
                         "evaluations (mean over the steps); ms_per_step = the samples' measured wall time",
           "cpu_baseline": {"kind": "oracle", "cores": ot.T, "value": v, "unit": "s/step",
                            "sample": ot.sample + f"; x {n_res:g} residuals + {n_jv:g} J V"
                                      + (f" + {n_ns:g} NS operator applications" if coupled else "")
                                      + " per step (operator evaluations only)",
                            "oracle_mesh_build_s": ot.build_s},
           "e2e": {"value": v, "unit": "s/step", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def workload_config(name, mesh, coupled=True):
    wl = WORKLOADS[name]
    cfg = {"workload": wl["desc"], "eps": wl["eps"], "V": wl["V"], "dt": wl["dt"],
           "n_elem": mesh.n_elem, "n_nodes": mesh.n_nodes, "n_hanging": mesh.n_hanging, "dofs": 3 * mesh.n_nodes}
    if coupled:
        cfg.update({"step": "NS-PNP block iteration (one pass): linear VMS Navier-Stokes, then PNP Newton",
                    "velocity": "Navier-Stokes block: Sc = 1, kappa = 0.5, no-slip walls, fluid at rest at t = 0",
                    "ns_dofs": 4 * mesh.n_nodes,
                    "ns_solver": "FGMRES(50) in FP64 (basis, two-pass Gram-Schmidt, matrix action) right-"
                                 "preconditioned by an FP32 multigrid V-cycle (8 coarser octrees, 3 block-Jacobi "
                                 "sweeps, damping 0.6, 32 on the coarsest), to 1e-8 relative / 1e-10 absolute"})
    else:
        cfg["velocity"] = "zero (the PNP block alone)"
    return cfg


# ----------------------------------------------------------------------------- helpers
def max_over_ranks(ms, dist, device):
    """The slowest rank's time (replicas: every rank times the same work)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def replica_throughput(units_per_rank, world, ms):
    """Whole-job GDoF/s: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / (ms * 1e-3) / 1e9


def replica_seconds_per_step(ms, steps, world):
    """Whole-job seconds per step: the slowest rank's time over the steps all ranks took."""
    return ms * 1e-3 / (steps * world)


def kernel_table(prof, peaks, total_ms, N, E):
    """Per class: time share, algorithmic GB/s and TFLOP/s, the roofline that binds it and
    the fraction of it.  The J V classes use the algorithmic work of the measurement plan
    (bytes per node and element, 2.5 kFLOP per element); the others the library's own
    per-launch accounting."""
    rows = {}
    for name, d in prof.items():
        if d["count"] == 0 or d["ms"] <= 0:
            continue
        t = d["ms"] * 1e-3
        if name in JV_BYTES_PER_NODE:
            by = (JV_BYTES_PER_NODE[name] * N + JV_BYTES_PER_ELEM * E) * d["count"]
            fl = JV_FLOPS_PER_ELEM * E * d["count"]
        else:
            by, fl = d["alg_bytes"], d["alg_flops"]
        gbs = by / t / 1e9
        tfl = fl / t / 1e12
        kind = BOUNDS[name]
        if kind == "hbm":
            bound, unit, ach, peak = "hbm", "GB/s", gbs, peaks["hbm_gbs"]
            src = "measured" if not peaks.get("fallback") else "fallback"
        elif kind == "bf16":
            bound, unit, ach, peak = "tensor", "TFLOP/s", tfl, peaks.get("bf16_tflops_sustained", 1700.0)
            src = "measured sustained" if not peaks.get("fallback") else "fallback"
        else:
            alu = FP64_TFLOPS if kind == "fp64" else FP32_TFLOPS
            if fl / (alu * 1e12) >= by / (peaks["hbm_gbs"] * 1e9):
                bound, unit, ach, peak = "alu", "TFLOP/s", tfl, alu
                src = f"derived {kind.upper()}: 152 SMs x {2 if kind == 'fp64' else 128} FMA/clk x 2 x 2.07 GHz"
            else:
                bound, unit, ach, peak = "hbm", "GB/s", gbs, peaks["hbm_gbs"]
                src = "measured" if not peaks.get("fallback") else "fallback"
        rows[name] = {"bound": bound, "achieved": round(ach, 4), "peak": round(peak, 3), "unit": unit,
                      "frac": round(ach / peak, 4), "peak_source": src, "launches": d["count"],
                      "avg_launch_ms": d["ms"] / d["count"], "share": round(d["ms"] / total_ms, 4),
                      "alg_bytes_per_launch": by / d["count"], "alg_flops_per_launch": fl / d["count"],
                      "alg_gbs": round(gbs, 1), "hbm_frac": round(gbs / peaks["hbm_gbs"], 4)}
    return rows


def load_traffic(workload, coupled=True):
    """Per-class DRAM traffic from the committed ncu summary, for kernels whose source is
    unchanged since the capture and whose variant the step runs (the coupled step's PNP
    solve has an advection field: four stored rows per lane; the PNP step alone three)."""
    import hashlib
    try:
        tj = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    except Exception:
        return {}
    if tj.get("workload") != workload:
        return {}
    out = {"_note": tj.get("note", "")}
    for name, e in tj.get("classes", {}).items():
        if e.get("step", "coupled") != ("coupled" if coupled else "pnp_only"):
            continue
        try:
            same = all(hashlib.sha256(open(os.path.join(ROOT, f), "rb").read()).hexdigest() == h
                       for f, h in e["sources"].items())
        except OSError:
            same = False
        if same:
            out[name] = e
    return out


def roofline(table, traffic, name="jv32", n_elem=0):
    """The roofline object of the J V class (the dominant class of the step); `traffic` is
    ncu's DRAM bytes of the class's kernel scaled to this launch by its elements."""
    if name not in table:
        name = max(table, key=lambda k: table[k]["avg_launch_ms"] * table[k]["launches"]) if table else None
    if name is None:
        return None
    rl = dict(table[name])
    rl["kernel"] = name
    e = traffic.get(name)
    rl["traffic"] = None
    if e:
        if "dram_bytes_per_element" in e and n_elem:
            rl["traffic"] = e["dram_bytes_per_element"] * n_elem
            rl["traffic_note"] = traffic.get("_note", "")
        elif "dram_bytes_per_launch" in e:
            rl["traffic"] = e["dram_bytes_per_launch"]
    return rl


def train_learned_start(pnp, torch, ctx, n_record, train_steps, coupled=True):
    """Record the first steps of this run (extrapolated start) and train the network."""
    from paper_2301_05985_gb300 import learned_start as LS
    p = ctx.get_params()
    mode = p.start_mode
    p.start_mode = pnp.PNP_START_EXTRAPOLATE
    ctx.set_params(p)
    t0 = time.perf_counter()
    S, its, uz = LS.record(pnp, torch, ctx, n_record, coupled=coupled)
    ctx.mlp_init(seed=0)
    ctx.mlp_add_trajectory(S, uz)
    st = ctx.mlp_train(steps=train_steps, batch=4096, lr=1e-3, seed=1)
    p.start_mode = mode
    ctx.set_params(p)
    del S
    return {"recorded_steps": len(its), "train_steps": train_steps, "loss_first": st.loss_first,
            "loss_last": st.loss_last, "train_s": st.wall_ms * 1e-3, "setup_s": time.perf_counter() - t0}


def snapshot(pnp, torch, ctx, N):
    """U^k, U^{k-1}, v^k, v^{k-1} and (v, p)^k on the device."""
    h = [torch.empty((N, 3), dtype=torch.float64, device="cuda") for _ in range(4)]
    h.append(torch.empty((N, 4), dtype=torch.float64, device="cuda"))
    ctx.get_field(pnp.PNP_FIELD_U_PREV, h[0], pnp.PNP_DEVICE)
    ctx.get_field(pnp.PNP_FIELD_U_PREV2, h[1], pnp.PNP_DEVICE)
    ctx.get_field(pnp.PNP_FIELD_VELOCITY, h[2], pnp.PNP_DEVICE)
    ctx.get_field(pnp.PNP_FIELD_VELOCITY_PREV, h[3], pnp.PNP_DEVICE)
    ctx.get_field(pnp.PNP_FIELD_NS, h[4], pnp.PNP_DEVICE)
    torch.cuda.synchronize()
    return h


def restore(pnp, ctx, h, step=8):
    """Resume the trajectory at the snapshot (the next step is BDF2 from it)."""
    ctx.set_field(pnp.PNP_FIELD_U_PREV, h[0], pnp.PNP_DEVICE)
    ctx.set_field(pnp.PNP_FIELD_U_PREV2, h[1], pnp.PNP_DEVICE)
    ctx.set_field(pnp.PNP_FIELD_U, h[0], pnp.PNP_DEVICE)
    ctx.set_field(pnp.PNP_FIELD_VELOCITY, h[2], pnp.PNP_DEVICE)
    ctx.set_field(pnp.PNP_FIELD_VELOCITY_PREV, h[3], pnp.PNP_DEVICE)
    ctx.set_field(pnp.PNP_FIELD_NS, h[4], pnp.PNP_DEVICE)
    ctx.set_step_count(step)


def run_arm(pnp, torch, W, mesh, wl, mode, hist, steps, coupled=True):
    """`steps` BDF2 steps of an arm from the snapshot state; time, iterations, final U."""
    ctx = make_ctx(pnp, W, torch, mesh, wl, mode)
    restore(pnp, ctx, hist)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sts = [do_step(ctx, coupled, raise_on_error=False) for _ in range(steps)]
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    U = ctx.get_field(pnp.PNP_FIELD_U)
    ctx.close()
    return {"s_per_step": t / steps, "steps": steps, "newton_its_per_step": sum(s["newton_its"] for s in sts) / steps,
            "krylov_its_per_step": sum(s["krylov_its"] for s in sts) / steps,
            "jv_per_step": sum(s["jv_evals"] for s in sts) / steps,
            "step_s": spread([s["wall_ms"] * 1e-3 for s in sts]),
            "mg_fallbacks": [int(s["mg_fallbacks"]) for s in sts],
            "status": [int(s["status"]) for s in sts], "substeps": [int(s["substeps"]) for s in sts],
            "ns": ns_summary(sts)}, U


def spread(xs):
    """Median and range of per-step times (the Krylov path varies from run to run: the
    atomic scatter reorders FP32 sums)."""
    return {"median": float(np.median(xs)), "min": float(np.min(xs)), "max": float(np.max(xs)), "n": len(xs)}


def field_errors(U, ref):
    """Relative 2-norm and max-norm differences per field (c+, c-, phi)."""
    out = {}
    for f, name in enumerate(["c+", "c-", "phi"]):
        d = U[:, f] - ref[:, f]
        out[name] = {"rel_l2": float(np.linalg.norm(d) / np.linalg.norm(ref[:, f])),
                     "rel_max": float(np.abs(d).max() / np.abs(ref[:, f]).max())}
    return out


def jv_sweep(pnp, torch, W, peaks, states=5, reps=10):
    """FP64 and FP32 J V on the uniform level-7 cube (128^3 elements, 6.44 M dofs) with the
    divergence-free Fourier velocity, Lambda = 1e-3, V = 30, at seeded states: GDoF/s, HBM
    fraction of the algorithmic bytes, the binding roofline fraction, and the FP32 error
    against the FP64 J V per field (the FP64 J V matches the oracle at this size in the
    parity tests)."""
    oc = W.uniform_octants(3, 7)
    mesh = pnp.Mesh(oc)
    N, E, L = mesh.n_nodes, mesh.n_elem, oc.max_level
    ctx = pnp.Context(mesh, pnp.default_params(eps=1e-3, dt=1e-3, beta0=1.5, beta1=-2.0, beta2=0.5),
                      torch.cuda.current_stream().cuda_stream)
    ctx.set_bcs(W.membrane_bcs(3, 30.0, 2.0))
    ctx.set_field(pnp.PNP_FIELD_ADVECTION, W.fourier_velocity(mesh.ijk, L, 3))
    res = {"mesh": "uniform level 7 (2,097,152 elements, 2,146,689 nodes)", "velocity": "Fourier, RMS 0.1",
           "states": states, "jv64": [], "jv32": [], "err32": []}
    for sd in range(states):
        Uk = W.noisy_state(mesh.ijk, L, seed=10 + sd, amp=1e-3, phi_bottom=0.0, phi_top=30.0)
        ctx.set_field(pnp.PNP_FIELD_U_PREV, Uk)
        ctx.set_field(pnp.PNP_FIELD_U_PREV2, Uk)
        Ud = torch.from_numpy(W.noisy_state(mesh.ijk, L, seed=20 + sd, amp=1e-2, phi_bottom=0.0, phi_top=30.0)).cuda()
        Vd = torch.from_numpy(W.random_direction(mesh.ijk, L, 30 + sd)).cuda()
        V32 = Vd.float()
        J64 = torch.zeros_like(Vd)
        J32 = torch.zeros_like(V32)
        for prec, V, J in ((pnp.PNP_F64, Vd, J64), (pnp.PNP_F32, V32, J32)):
            ctx.jv(Ud, V, J, prec)
            ctx.profile_enable(True)
            for _ in range(reps):
                ctx.jv(Ud, V, J, prec)
            pr = ctx.profile_read()
            ctx.profile_enable(False)
            name = "jv64" if prec == pnp.PNP_F64 else "jv32"
            t = pr[name]["ms"] / pr[name]["count"] * 1e-3
            by = JV_BYTES_PER_NODE[name] * N + JV_BYTES_PER_ELEM * E
            fl = JV_FLOPS_PER_ELEM * E
            alu = FP64_TFLOPS if name == "jv64" else FP32_TFLOPS
            tstar = max(by / (peaks["hbm_gbs"] * 1e9), fl / (alu * 1e12))
            res[name].append({"ms": t * 1e3, "gdofs": 3 * N / t / 1e9, "hbm_frac": by / t / (peaks["hbm_gbs"] * 1e9),
                              "binding_frac": tstar / t})
        a, b = J32.double().cpu().numpy(), J64.cpu().numpy()
        res["err32"].append({f: float(np.linalg.norm(a[:, i] - b[:, i]) / np.linalg.norm(b[:, i]))
                             for i, f in enumerate(["c+", "c-", "phi"])})
    for name in ("jv64", "jv32"):
        rows = res[name]
        res[name + "_mean"] = {k: float(np.mean([r[k] for r in rows])) for k in rows[0]}
    ctx.close()
    mesh.close()
    return res


# ----------------------------------------------------------------------------- main
def timed_mixed(pnp, torch, ctx, steps, stream, local, coupled):
    stats = []
    launches0 = pnp.kernel_launches()
    sys.stderr.write(f"library launches before the timed steps: {launches0}\n")
    captures0 = pnp.graph_captures()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            stats.append(do_step(ctx, coupled))
        e1.record(stream)
        torch.cuda.synchronize()
    return e0.elapsed_time(e1), stats, pnp.kernel_launches() - launches0, pnp.graph_captures() - captures0, clk


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    from paper_2301_05985_gb300 import pnp
    from paper_2301_05985_gb300 import workloads as W

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    pnp.lib()
    wl = WORKLOADS[args.workload]
    full = args.workload != "small"
    oc, target, mesh_info = build_workload(pnp, torch, args.workload)
    mesh = pnp.Mesh(oc, target_levels=target)
    N, E = mesh.n_nodes, mesh.n_elem
    ctx = make_ctx(pnp, W, torch, mesh, wl, "mixed", learned=not args.no_learned)
    stream = torch.cuda.current_stream()
    coupled = not args.pnp_only

    learned = None
    warm = args.warmup
    if not args.no_learned:
        # the warm-up steps (extrapolated start) are the recorded trajectory; one more
        # untimed step then runs the trained network's path once
        rec = args.record_steps if args.record_steps > 0 else max(args.warmup, 3)
        learned = train_learned_start(pnp, torch, ctx, rec, args.train_steps, coupled)
        warm = 1 if args.record_steps <= 0 else args.warmup
    for _ in range(warm):
        do_step(ctx, coupled)
    torch.cuda.synchronize()
    hist = snapshot(pnp, torch, ctx, N)  # the state the timed steps start from
    if dist:
        dist.barrier()
    ms, stats, launches, captures, clk = timed_mixed(pnp, torch, ctx, args.steps, stream, local, coupled)
    ms = max_over_ranks(ms, dist, "cuda")
    value = replica_seconds_per_step(ms, args.steps, world)
    gdofs_advanced = replica_throughput(3.0 * N * args.steps, world, ms)

    # per-class kernel times: further steps with the library's event pair around every launch
    ctx.profile_enable(True)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kp = max(1, min(args.profile_steps, args.steps))
    torch.cuda.synchronize()
    p0.record(stream)
    for _ in range(kp):
        do_step(ctx, coupled)
    p1.record(stream)
    torch.cuda.synchronize()
    prof_ms = p0.elapsed_time(p1)
    prof = ctx.profile_read()
    ctx.profile_enable(False)

    # end to end through the C ABI: the same steps again from the same state, the history
    # uploaded from pinned host memory and the new state read back every step
    plain_steps = max(1, min(args.plain_steps, args.steps))
    e2e_steps = max(1, min(args.e2e_steps, args.steps))
    e2e = None
    U_mixed = None
    if not args.no_e2e:
        # pinned host copies of the step's inputs (U^k, U^{k-1}, v^k, v^{k-1}, (v, p)^k) and outputs
        pin = lambda k: torch.empty((N, k), dtype=torch.float64, pin_memory=True)  # noqa: E731
        hU, hV, hX = [pin(3) for _ in range(3)], [pin(3) for _ in range(2)], [pin(4) for _ in range(2)]
        for dst, src in ((hU[0], hist[0]), (hU[1], hist[1]), (hV[0], hist[2]), (hV[1], hist[3]), (hX[0], hist[4])):
            dst.copy_(src)
        torch.cuda.synchronize()
        c0 = pnp.graph_captures()
        e2e_stats = []
        t0 = time.perf_counter()
        restore(pnp, ctx, hist)
        for k in range(e2e_steps):
            ctx.set_field(pnp.PNP_FIELD_U_PREV, hU[0], pnp.PNP_HOST)
            ctx.set_field(pnp.PNP_FIELD_U_PREV2, hU[1], pnp.PNP_HOST)
            if coupled:
                ctx.set_field(pnp.PNP_FIELD_VELOCITY, hV[0], pnp.PNP_HOST)
                ctx.set_field(pnp.PNP_FIELD_VELOCITY_PREV, hV[1], pnp.PNP_HOST)
                ctx.set_field(pnp.PNP_FIELD_NS, hX[0], pnp.PNP_HOST)
            e2e_stats.append(do_step(ctx, coupled))
            ctx.get_field(pnp.PNP_FIELD_U, hU[2], pnp.PNP_HOST)
            if coupled:
                ctx.get_field(pnp.PNP_FIELD_NS, hX[1], pnp.PNP_HOST)
                hV = [hV[1], hV[0]]
                hV[0].copy_(hX[1][:, :3])  # v^{k+1} is the next step's v^k
                hX = [hX[1], hX[0]]
            if k + 1 == plain_steps:
                U_mixed = hU[2].numpy().copy()
            hU = [hU[2], hU[0], hU[1]]
        t_e2e = time.perf_counter() - t0
        h2d = (2 * 24 + (2 * 24 + 32 if coupled else 0)) * N
        d2h = (24 + (32 if coupled else 0)) * N
        e2e = {"value": replica_seconds_per_step(1e3 * t_e2e, e2e_steps, world), "unit": "s/step",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": 1e3 * t_e2e / e2e_steps, "steps": e2e_steps, "graph_captures": pnp.graph_captures() - c0,
               "trajectory": f"the first {e2e_steps} timed steps again from the same state",
               "device_timed_same_steps_s_per_step": sum(s["wall_ms"] for s in stats[:e2e_steps]) * 1e-3 / e2e_steps,
               "step_s": spread([s["wall_ms"] * 1e-3 for s in e2e_stats]),
               "newton_its_per_step": sum(s["newton_its"] for s in e2e_stats) / e2e_steps,
               "krylov_its_per_step": sum(s["krylov_its"] for s in e2e_stats) / e2e_steps,
               "ns": ns_summary(e2e_stats)}

    peaks = measured_peaks()
    table = kernel_table(prof, peaks, prof_ms, N, E)
    rl = roofline(table, load_traffic(args.workload, coupled), "jv32", E)
    jv = dict(table.get("jv32", {}))
    if jv:
        jv["gdofs"] = 3.0 * N / (jv["avg_launch_ms"] * 1e-3) / 1e9
        tstar = max((JV_BYTES_PER_NODE["jv32"] * N + JV_BYTES_PER_ELEM * E) / (peaks["hbm_gbs"] * 1e9),
                    JV_FLOPS_PER_ELEM * E / (FP32_TFLOPS * 1e12))
        jv["binding_time_ms"] = tstar * 1e3
        jv["binding_frac"] = tstar / (jv["avg_launch_ms"] * 1e-3)

    nt = sum(s["newton_its"] for s in stats)
    kt = sum(s["krylov_its"] for s in stats)
    n_res = sum(s["residual_evals"] for s in stats) / args.steps
    n_jv = sum(s["jv_evals"] for s in stats) / args.steps
    nss = ns_summary(stats)
    n_ns = (nss["fp32_fine_applications_per_step"] + nss["fp64_applications_per_step"]) if nss else 0.0

    # FP64 arms and the multigrid-preconditioned arm from the same state (rank 0 only)
    arms = {}
    if not args.no_mg and rank == 0:
        mg_steps = max(1, min(args.mg_steps, args.steps))
        arm, _ = run_arm(pnp, torch, W, mesh, wl, "mixed_mg", hist, mg_steps, coupled)
        arm["preconditioner"] = ("geometric multigrid V-cycle (8 coarser octrees, 3 block-Jacobi sweeps, "
                                 "damping 0.6, 32 sweeps on the coarsest), inner GMRES(24) where it falls behind")
        arm["start"] = "extrapolated"
        arm["timed_mixed_same_steps_s_per_step"] = sum(s["wall_ms"] for s in stats[:mg_steps]) * 1e-3 / mg_steps
        arms["mixed_multigrid"] = arm
    if (args.plain or args.workload != "electroconvection") and rank == 0:
        arm, U_same = run_arm(pnp, torch, W, mesh, wl, "same64", hist, plain_steps, coupled)
        arms["plain_same_solver"] = arm
        arm, U_gm = run_arm(pnp, torch, W, mesh, wl, "plain", hist, plain_steps, coupled)
        arms["plain_gmres"] = arm
        if U_mixed is not None:
            arms["field_errors"] = {"steps": plain_steps, "mixed_vs_fp64_same_solver": field_errors(U_mixed, U_same),
                                    "mixed_vs_fp64_gmres": field_errors(U_mixed, U_gm),
                                    "fp64_same_solver_vs_fp64_gmres": field_errors(U_same, U_gm)}
        arms["mixed_first_steps"] = {"steps": plain_steps,
                                     "s_per_step": sum(s["wall_ms"] for s in stats[:plain_steps]) * 1e-3 / plain_steps,
                                     "newton_its_per_step": sum(s["newton_its"] for s in stats[:plain_steps]) / plain_steps,
                                     "krylov_its_per_step": sum(s["krylov_its"] for s in stats[:plain_steps]) / plain_steps}

    if rank != 0:
        return
    sweep = None
    if not args.no_sweep and full and world == 1:
        sweep = jv_sweep(pnp, torch, W, peaks)
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        Uh = hist[0].cpu().numpy()
        Vh = W.random_direction(mesh.ijk, mesh.max_level, 5)
        oc_full = W.Octants(3, mesh.max_level, *mesh.elements())
        ns_state = {"X": hist[4].cpu().numpy(), "vk": hist[2].cpu().numpy(), "vkm1": hist[3].cpu().numpy()} \
            if coupled else None
        ot = oracle_timing(oc_full, wl, {"U": Uh, "ijk": mesh.ijk}, Uh, hist[1].cpu().numpy(), Vh, n_res, n_jv,
                           ns_state=ns_state, n_ns=n_ns)
        cpu = {"value": ot["s_per_step"], "unit": "s/step", "cores": ot["cores"], "kind": "oracle",
               "sample": ot["sample"] + f"; x {n_res:.1f} residuals + {n_jv:.0f} J V"
                         + (f" + {n_ns:.0f} NS operator applications (FP64 ones and the V-cycles' on the "
                            "finest mesh)" if coupled else "")
                         + " per step (the mixed step's counts; operator evaluations only, FP64)",
               "residual_gdofs": ot["residual_gdofs"], "jv_gdofs": ot["jv_gdofs"],
               "t_residual_s": ot["t_residual_s"], "t_jv_s": ot["t_jv_s"], "t_ns_s": ot.get("t_ns_s"),
               "oracle_mesh_build_s": ot["oracle_mesh_build_s"]}
    ctx.close()
    secondary = None
    if not args.no_secondary and args.workload == "electroconvection" and world == 1:
        secondary = secondary_membrane(pnp, torch, W, peaks, coupled=coupled)

    out = {
        "metric": METRIC, "value": round(value, 6), "unit": "s/step", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {**workload_config(args.workload, mesh, coupled), "mesh_build": mesh_info,
                   "mode": "mixed FP32 J V + learned start" if learned else "mixed FP32 J V",
                   "krylov": "flexible GMRES(60) in FP64, preconditioned by 24 steps of FP32 GMRES on J M^-1 "
                             "(M block Jacobi); Eisenstat-Walker forcing",
                   "start": "learned (judged vs extrapolated)" if learned else "extrapolated",
                   "l2": "inputs larger than L2 (FP64 vectors of 3N entries, Krylov basis of 61 of them)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": rl,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "graph_captures": int(captures),
        "clocks": clk.summary(),
        "jv": jv,
        "gdofs_advanced_per_s": gdofs_advanced,
        "step_s": spread([s["wall_ms"] * 1e-3 for s in stats]),
        "newton_its_per_step": nt / args.steps, "krylov_its_per_step": kt / args.steps,
        "residual_evals_per_step": n_res, "jv_evals_per_step": n_jv,
        "ns": nss,
        "split_steps": sum(int(s["substeps"] > 1) for s in stats),
        "learned_start_used": sum(int(s["start_used"] == pnp.PNP_START_LEARNED) for s in stats),
        "learned_training": learned,
        **arms,
        "kernels": table,
        "kernel_profile": {"steps": kp, "ms_per_step": prof_ms / kp,
                           "note": "per-class times and shares from further steps with an event pair around every "
                                   "launch (eager); the timed steps replay the inner solve as a CUDA graph"},
        "jv_sweep_uniform_L7": sweep,
        "secondary_membrane_L5_8": secondary,
    }
    print(json.dumps(out))


def secondary_membrane(pnp, torch, W, peaks, warmup=3, steps=3, coupled=True):
    """The membrane-band octree (3.14 M dofs): mixed steps and both FP64 arms from the same
    state, with the per-field differences of the final states."""
    wl = WORKLOADS["membrane"]
    mesh = pnp.Mesh(W.membrane_band_octants(5, 8, 0.05))
    N = mesh.n_nodes
    ctx = make_ctx(pnp, W, torch, mesh, wl, "mixed", learned=False)
    for _ in range(warmup):
        do_step(ctx, coupled)
    hist = snapshot(pnp, torch, ctx, N)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sts = [do_step(ctx, coupled) for _ in range(steps)]
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    Um = ctx.get_field(pnp.PNP_FIELD_U)
    ctx.close()
    out = {"workload": wl["desc"], "dofs": 3 * N, "steps": steps,
           "mixed": {"s_per_step": t / steps, "newton_its_per_step": sum(s["newton_its"] for s in sts) / steps,
                     "krylov_its_per_step": sum(s["krylov_its"] for s in sts) / steps,
                     "start": "extrapolated", "ns": ns_summary(sts)}}
    arm, _ = run_arm(pnp, torch, W, mesh, wl, "mixed_mg", hist, steps, coupled)
    out["mixed_multigrid"] = arm
    arm, Us = run_arm(pnp, torch, W, mesh, wl, "same64", hist, steps, coupled)
    out["plain_same_solver"] = arm
    arm, Ug = run_arm(pnp, torch, W, mesh, wl, "plain", hist, steps, coupled)
    out["plain_gmres"] = arm
    out["field_errors"] = {"mixed_vs_fp64_same_solver": field_errors(Um, Us), "mixed_vs_fp64_gmres": field_errors(Um, Ug)}
    mesh.close()
    return out


if __name__ == "__main__":
    main()
