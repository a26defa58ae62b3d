"""Benchmark: BDF time steps of the VMS PNP block on the 3D near-membrane octree.

Workload (the transient membrane configuration): unit cube, octree base level 5,
level 8 for every octant with z_min < 0.05, 2:1 graded (971,776 elements, 1,047,407
nodes, 3.14 M unknowns c+, c-, phi); Lambda = 1e-3, V = 20, dt = 1e-3; membrane
at z = 0 (phi = 0, c+ = 2, c- zero flux), reservoir at z = 1 (phi = V, c+- = 1),
zero-flux side walls; c+- = 1 + seeded uniform noise of amplitude 1e-3, phi linear.
The velocity is zero (no Navier-Stokes block in this library).

One step = one pnp_time_step: BDF2 (BDF1 first), Newton to ||F|| <= 1e-8 ||F(U^k)||,
GMRES with 3x3 block-Jacobi on the exact Jacobian action.  Modes:
  mixed : inexact Newton (Eisenstat-Walker) with flexible GMRES(60) in FP64 (dots,
          orthogonalisation, basis), preconditioned by 24 steps of FP32 GMRES on J M^-1
          (FP32 J V, M the 3x3 block Jacobi); FP64 residual; learned start (network
          trained, before the timed region, on the first steps of this run's own
          trajectory), judged against the extrapolated start 2 U^k - U^{k-1}.
  plain : FP64 J V, GMRES(100) rtol 1e-8 per Newton step, previous-step start (the
          paper's); timed for comparison from the same state as the first mixed step.

value = unknowns advanced per second = 3 N x steps / time (GDoF/s), timed with CUDA
events on the library's stream.  Kernel rooflines come from the library's own event
timing of each launch class during the timed region, against the roofline that bounds
the class: FP64 or FP32 ALU (peaks derived from 152 SMs x 2 FP64 / 128 FP32 FMA per
clock x 2.07 GHz), HBM or BF16 tensor (measured peaks).
"""
from __future__ import annotations

import argparse
import json
import os
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
EPS, VOLT, DT = 1e-3, 20.0, 1e-3
# ALU peaks: 152 SMs x (2 FP64 | 128 FP32) FMA per clock x 2 flop x 2.07 GHz
FP64_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# arithmetic of each kernel class; for ALU classes the binding roofline is chosen per run
# from the algorithmic flops and bytes (kernel_table)
BOUNDS = {"residual64": "fp64", "jv64": "fp64", "jv32": "fp32", "blockdiag": "fp32", "ortho_dot": "fp64",
          "ortho_update": "fp64", "precond": "hbm", "mlp": "bf16", "inner_ortho": "hbm"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="mixed", choices=["mixed", "plain"])
    ap.add_argument("--small", action="store_true", help="level 4-7 miniature (profiling captures)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-mode comparison step")
    ap.add_argument("--no-learned", action="store_true", help="mixed mode without training the learned start")
    ap.add_argument("--inner", type=int, default=None, help="inner FP32 GMRES steps of the flexible outer GMRES (mixed)")
    ap.add_argument("--restart", type=int, default=None, help="outer GMRES restart length (mixed)")
    ap.add_argument("--record-steps", type=int, default=8, help="trajectory steps recorded for training")
    ap.add_argument("--train-steps", type=int, default=400, help="Adam steps of the learned start")
    return ap.parse_args()


def workload_octants(small: bool):
    from paper_2301_05985_gb300 import workloads as W
    return W.membrane_band_octants(4, 7, 0.05) if small else W.membrane_band_octants(5, 8, 0.05)


INNER, RESTART = 24, 60  # mixed mode: inner FP32 GMRES steps, outer restart


def mode_params(pnp, mode, inner=None, restart=None):
    if mode == "mixed":
        inner = INNER if inner is None else inner
        restart = RESTART if restart is None else restart
        return pnp.default_params(eps=EPS, dt=DT, precision=pnp.PNP_F32, start_mode=pnp.PNP_START_LEARNED,
                                  newton_rtol=1e-8, gmres_restart=restart, gmres_max_it=3000, dt_retries=2,
                                  gmres_inner=inner)
    return pnp.default_params(eps=EPS, dt=DT, precision=pnp.PNP_F64, start_mode=pnp.PNP_START_PREVIOUS,
                              newton_rtol=1e-8, gmres_rtol=1e-8, gmres_restart=100, gmres_max_it=4000,
                              dt_retries=2)


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


def setup_ctx(pnp, W, torch, oc, mode, inner=None, restart=None):
    mesh = pnp.Mesh(oc)
    ctx = pnp.Context(mesh, mode_params(pnp, mode, inner, restart), torch.cuda.current_stream().cuda_stream)
    ctx.set_bcs(W.membrane_bcs(3, VOLT, 2.0))
    U0 = W.noisy_state(mesh.ijk, oc.max_level, seed=0, amp=1e-3, phi_bottom=0.0, phi_top=VOLT)
    ctx.set_field(pnp.PNP_FIELD_U, U0)
    ctx.make_consistent()
    ctx.reset_history()
    return mesh, ctx


def cpu_baseline_oracle(n_steps: int = 1):
    """The FP64 oracle (single-threaded C++ + SciPy sparse direct solve) on a bounded
    sample: the same physics on the level 3-5 miniature of the membrane octree."""
    import oracle as O
    from paper_2301_05985_gb300 import workloads as W
    oc = W.membrane_band_octants(3, 5, 0.05)
    m = O.OracleMesh(oc)
    bcs = W.membrane_bcs(3, VOLT, 2.0)
    U = W.noisy_state(m.ijk, oc.max_level, seed=0, amp=1e-3, phi_bottom=0.0, phi_top=VOLT)
    p = O.Params(eps=EPS, dt=DT, beta=(1.0, -1.0, 0.0), bc_type=bcs.types, bc_val=bcs.values)
    U = m.make_consistent(U, p)
    Uk = Ukm1 = U
    t0 = time.perf_counter()
    for k in range(n_steps):
        beta = O.bdf_coefficients(k)
        p = O.Params(eps=EPS, dt=DT, beta=beta, bc_type=bcs.types, bc_val=bcs.values)
        res = O.newton(m, p, Uk, Uk, Ukm1, None, rtol=1e-8)
        Ukm1, Uk = Uk, res.U
    t = time.perf_counter() - t0
    return {"value": 3 * m.n_nodes * n_steps / t / 1e9, "unit": "GDoF/s", "cores": 1, "kind": "oracle",
            "sample": f"{n_steps} BDF step(s) of the same physics on the level 3-5 miniature of the membrane "
                      f"octree ({m.n_elem} elements, {m.n_nodes} nodes), oracle Newton with direct sparse "
                      f"solves, {t:.1f} s"}


def workload_config(small: bool):
    """The workload both arms name (the reference arm times the oracle on a bounded sample
    of it, described in its cpu_baseline)."""
    return {"workload": ("membrane-band octree L4-7 miniature" if small else
                         "3D membrane-band octree, base level 5, level 8 for z<0.05 (2:1 graded)"),
            "eps": EPS, "V": VOLT, "dt": DT, "velocity": "zero (no NS block)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for _ in range(args.warmup):
        pass  # the oracle has nothing to warm up
    vals = []
    t0 = time.perf_counter()
    cb = None
    for _ in range(args.steps):
        cb = cpu_baseline_oracle(1)
        vals.append(cb["value"])
    t = time.perf_counter() - t0
    v = float(np.mean(vals))
    out = {"metric": METRIC, "value": v, "unit": "GDoF/s", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": workload_config(args.small),
           "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": cb["sample"], "value": v},
           "e2e": {"value": v, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def ctx_krylov_desc(p, mode):
    if mode == "plain":
        return f"GMRES({p.gmres_restart}) + block Jacobi, FP64 J V, rtol {p.gmres_rtol:g}"
    if p.gmres_inner > 0:
        return (f"flexible GMRES({p.gmres_restart}) in FP64, preconditioned by {p.gmres_inner} steps of FP32 "
                f"GMRES on J M^-1 (M block Jacobi); Eisenstat-Walker forcing")
    return f"GMRES({p.gmres_restart}) + block Jacobi, FP32 J V, FP64 dots; Eisenstat-Walker forcing"


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


def load_traffic(small: bool):
    """Per-class DRAM traffic from the committed ncu summary, for kernels whose source
    is unchanged since the capture."""
    import hashlib
    try:
        tj = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    except Exception:
        return {}
    if tj.get("workload") != ("small" if small else "full"):
        return {}
    out = {}
    for name, e in tj.get("classes", {}).items():
        try:
            same = all(hashlib.sha256(open(os.path.join(ROOT, f), "rb").read()).hexdigest() == h
                       for f, h in e["sources"].items())
        except OSError:
            same = False
        if same:
            out[name] = e
    return out


def residual_kind():
    """The residual runs in double-float arithmetic on the FP32 pipe unless
    PNP_RESIDUAL_ARITH=f64 (or the one-thread-per-element kernel) selects FP64."""
    f64 = os.environ.get("PNP_RESIDUAL_ARITH") == "f64" or os.environ.get("PNP_ELEMENT_KERNEL") == "thread"
    return "fp64" if f64 else "fp32"


def kernel_table(prof, peaks, total_ms):
    """Per class: time share, algorithmic GB/s and TFLOP/s, and the fraction of the
    roofline that bounds it."""
    rows = {}
    for name, d in prof.items():
        if d["count"] == 0 or d["ms"] <= 0:
            continue
        t = d["ms"] * 1e-3
        gbs = d["alg_bytes"] / t / 1e9
        tfl = d["alg_flops"] / t / 1e12
        kind = residual_kind() if name == "residual64" else BOUNDS[name]
        if kind == "hbm":
            bound, unit, ach, peak = "hbm", "GB/s", gbs, peaks["hbm_gbs"]
            src = "measured" if not peaks.get("fallback") else "fallback"
        elif kind == "bf16":
            bound, unit, ach, peak = "tensor", "TFLOP/s", tfl, peaks.get("bf16_tflops_sustained", 1700.0)
            src = "measured sustained" if not peaks.get("fallback") else "fallback"
        else:
            alu = FP64_TFLOPS if kind == "fp64" else FP32_TFLOPS
            # the roofline that binds: the larger of the ALU time and the HBM time of the
            # algorithmic work (a stored linearisation can move a kernel from ALU to HBM)
            if d["alg_flops"] / (alu * 1e12) >= d["alg_bytes"] / (peaks["hbm_gbs"] * 1e9):
                bound, unit, ach, peak = "alu", "TFLOP/s", tfl, alu
                src = f"derived {kind.upper()}: 152 SMs x {2 if kind == 'fp64' else 128} FMA/clk x 2 x 2.07 GHz"
            else:
                bound, unit, ach, peak = "hbm", "GB/s", gbs, peaks["hbm_gbs"]
                src = "measured" if not peaks.get("fallback") else "fallback"
        rows[name] = {"bound": bound, "achieved": round(ach, 4), "peak": round(peak, 3), "unit": unit,
                      "frac": round(ach / peak, 4), "peak_source": src, "launches": d["count"],
                      "avg_launch_ms": d["ms"] / d["count"], "share": round(d["ms"] / total_ms, 4),
                      "alg_bytes_per_launch": d["alg_bytes"] / d["count"],
                      "alg_flops_per_launch": d["alg_flops"] / d["count"],
                      "alg_gbs": round(gbs, 1), "hbm_frac": round(gbs / peaks["hbm_gbs"], 4)}
    return rows


def roofline(table, traffic):
    """The dominant class's roofline object (largest device time)."""
    if not table:
        return None
    name = max(table, key=lambda k: table[k]["avg_launch_ms"] * table[k]["launches"])
    rl = dict(table[name])
    rl["kernel"] = name
    e = traffic.get(name)
    rl["traffic"] = None
    if e:
        if "dram_bytes_per_launch" in e:
            rl["traffic"] = e["dram_bytes_per_launch"]
        elif "dram_per_requested" in e:  # launches of varying size: DRAM bytes per requested byte
            rl["traffic"] = e["dram_per_requested"] * rl["alg_bytes_per_launch"]
            rl["traffic_note"] = "ncu DRAM bytes per L2-requested byte x this run's algorithmic bytes per launch"
    return rl


def train_learned_start(pnp, torch, ctx, n_record, train_steps):
    """Record the first steps of this run (extrapolated start) and train the network."""
    from paper_2301_05985_gb300 import learned_start as LS
    p = ctx.get_params()
    mode = p.start_mode
    p.start_mode = pnp.PNP_START_EXTRAPOLATE
    ctx.set_params(p)
    t0 = time.perf_counter()
    S, its = LS.record(pnp, torch, ctx, n_record)
    ctx.mlp_init(seed=0)
    ctx.mlp_add_trajectory(S)
    st = ctx.mlp_train(steps=train_steps, batch=4096, lr=1e-3, seed=1)
    p.start_mode = mode
    ctx.set_params(p)
    return {"recorded_steps": len(its), "train_steps": train_steps, "loss_first": st.loss_first,
            "loss_last": st.loss_last, "train_s": st.wall_ms * 1e-3, "setup_s": time.perf_counter() - t0}


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
    oc = workload_octants(args.small)
    mesh, ctx = setup_ctx(pnp, W, torch, oc, args.mode, args.inner, args.restart)
    N = mesh.n_nodes
    stream = torch.cuda.current_stream()

    learned = None
    if args.mode == "mixed" and not args.no_learned:
        learned = train_learned_start(pnp, torch, ctx, args.record_steps, args.train_steps)
    stats = []
    for _ in range(args.warmup):
        ctx.time_step()
    torch.cuda.synchronize()
    # the state the timed region starts from (for the plain-mode comparison)
    hist = [torch.empty((N, 3), dtype=torch.float64, device="cuda") for _ in range(2)]
    ctx.get_field(pnp.PNP_FIELD_U_PREV, hist[0], pnp.PNP_DEVICE)
    ctx.get_field(pnp.PNP_FIELD_U_PREV2, hist[1], pnp.PNP_DEVICE)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches0 = pnp.kernel_launches()
    captures0 = pnp.graph_captures()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            stats.append(ctx.time_step().as_dict())
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = pnp.kernel_launches() - launches0
    captures = pnp.graph_captures() - captures0
    # per-class kernel times: K further steps with the library's event pair around every
    # launch (eager launches: the inner solve's graph replays only while profiling is off)
    ctx.profile_enable(True)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    p0.record(stream)
    for _ in range(args.steps):
        ctx.time_step()
    p1.record(stream)
    torch.cuda.synchronize()
    prof_ms = p0.elapsed_time(p1)
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    ms = max_over_ranks(ms, dist, "cuda")
    value = replica_throughput(3.0 * N * args.steps, world, ms)

    # end to end through the C ABI with the state held in pinned host memory
    e2e = None
    if not args.no_e2e:
        hU = [torch.empty((N, 3), dtype=torch.float64, pin_memory=True) for _ in range(3)]
        ctx.get_field(pnp.PNP_FIELD_U_PREV, hU[0], pnp.PNP_HOST)
        ctx.get_field(pnp.PNP_FIELD_U_PREV2, hU[1], pnp.PNP_HOST)
        torch.cuda.synchronize()
        c_e2e0 = pnp.graph_captures()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.set_field(pnp.PNP_FIELD_U_PREV, hU[0], pnp.PNP_HOST)
            ctx.set_field(pnp.PNP_FIELD_U_PREV2, hU[1], pnp.PNP_HOST)
            ctx.time_step()
            ctx.get_field(pnp.PNP_FIELD_U, hU[2], pnp.PNP_HOST)
            hU = [hU[2], hU[0], hU[1]]
        t_e2e = time.perf_counter() - t0
        e2e_captures = pnp.graph_captures() - c_e2e0
        e2e = {"value": 3.0 * N * args.steps * world / t_e2e / 1e9, "unit": "GDoF/s",
               "h2d_bytes_per_step": 2 * 24 * N, "d2h_bytes_per_step": 24 * N,
               "ms_per_step": 1e3 * t_e2e / args.steps, "graph_captures": e2e_captures}

    # plain-mode comparison: one step from the state the timed mixed steps started from
    plain = None
    if not args.no_plain and rank == 0 and args.mode == "mixed":
        mesh_p, ctx_p = setup_ctx(pnp, W, torch, oc, "plain")
        p = ctx_p.get_params()
        p.bdf_order = 1
        ctx_p.set_params(p)
        ctx_p.time_step()  # one cheap BDF1 step so that the next one is BDF2 (history loaded below)
        p.bdf_order = 2
        ctx_p.set_params(p)
        ctx_p.set_field(pnp.PNP_FIELD_U_PREV, hist[0], pnp.PNP_DEVICE)
        ctx_p.set_field(pnp.PNP_FIELD_U_PREV2, hist[1], pnp.PNP_DEVICE)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = ctx_p.time_step().as_dict()
        torch.cuda.synchronize()
        plain = {"s_per_step": time.perf_counter() - t0, "newton_its": st["newton_its"],
                 "krylov_its": st["krylov_its"], "substeps": st["substeps"],
                 "state": "same state as the first timed mixed step",
                 "mixed_first_step": {"s": stats[0]["wall_ms"] * 1e-3, "newton_its": stats[0]["newton_its"],
                                      "krylov_its": stats[0]["krylov_its"]}}
        ctx_p.close()

    peaks = measured_peaks()
    table = kernel_table(prof, peaks, prof_ms)
    rl = roofline(table, load_traffic(args.small))
    jv_name = "jv32" if args.mode == "mixed" else "jv64"
    jv = prof[jv_name]
    jv_row = dict(table.get(jv_name, {}))
    if jv["ms"] > 0:
        jv_row.update({"name": jv_name, "gdofs": 3.0 * N * jv["count"] / (jv["ms"] * 1e-3) / 1e9})

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline_oracle(2)
    nt = sum(s["newton_its"] for s in stats)
    kt = sum(s["krylov_its"] for s in stats)
    out = {
        "metric": METRIC, "value": round(value, 6), "unit": "GDoF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if args.mode == "mixed" else "f64", "data": "synthetic",
        "config": {**workload_config(args.small),
                   "n_elem": mesh.n_elem, "n_nodes": N, "n_hanging": mesh.n_hanging, "dofs": 3 * N,
                   "mode": args.mode,
                   "krylov": ctx_krylov_desc(ctx.get_params(), args.mode),
                   "start": ("learned (judged vs extrapolated)" if learned else
                             "extrapolated" if args.mode == "mixed" else "previous step"),
                   "l2": "inputs larger than L2 (3.1M-dof FP64 vectors 25 MB each, Krylov basis up to 1.5 GB)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": rl,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "graph_captures": int(captures),
        "graph_captures_total": int(pnp.graph_captures()),
        "launches_before_timed": int(launches0),
        "clocks": clk.summary(),
        "newton_its_per_step": nt / args.steps, "krylov_its_per_step": kt / args.steps,
        "split_steps": sum(int(s["substeps"] > 1) for s in stats),
        "learned_start_used": sum(int(s["start_used"] == pnp.PNP_START_LEARNED) for s in stats),
        "s_per_step": ms * 1e-3 / args.steps,
        "jv_kernel": jv_row,
        "kernels": table,
        "kernel_profile": {"steps": args.steps, "ms_per_step": prof_ms / args.steps,
                           "note": "per-class times and shares from K further steps with an event pair around "
                                   "every launch (eager); the timed steps replay the inner solve as a CUDA graph"},
        "learned_training": learned,
        "plain_step": plain,
    }
    print(json.dumps(out))


if __name__ == "__main__":
    main()
