"""Host checks of the arithmetic behind bench.py's JSON line: the roofline of the J V class
from the measurement plan's work per unit, the kernel classes' bounds and shares, the
gating of the committed ncu traffic on the kernel's source, the replica aggregation and the
clock summary."""
import json
import os
import shutil

import pytest

import bench as B

N, E = 6_667_082, 5_595_136  # the electroconvection octree
PEAKS = {"hbm_gbs": 6790.3, "bf16_tflops_sustained": 1720.7}


def test_jv_roofline_follows_the_measurement_plan():
    """56 B per node + 36 B per element and 2.5 kFLOP per element over the launch time; the
    binding bound is the FP32 ALU time (30 us per million elements against 14 us of bytes)."""
    prof = {"jv32": {"ms": 0.748 * 100, "count": 100, "alg_bytes": 0.0, "alg_flops": 0.0}}
    t = B.kernel_table(prof, PEAKS, total_ms=0.748 * 100 / 0.38, N=N, E=E)["jv32"]
    assert t["bound"] == "alu" and t["unit"] == "TFLOP/s"
    assert t["alg_bytes_per_launch"] == pytest.approx(56.0 * N + 36.0 * E)
    assert t["alg_flops_per_launch"] == pytest.approx(2500.0 * E)
    tflops = 2500.0 * E / 0.748e-3 / 1e12
    assert t["achieved"] == pytest.approx(tflops, rel=1e-4)
    assert t["peak"] == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12, rel=1e-4)
    assert t["frac"] == pytest.approx(tflops / (152 * 128 * 2 * 2.07e9 / 1e12), abs=1e-4)
    assert t["frac"] == pytest.approx(0.2322, abs=1e-4)  # the bench line of 0.748 ms per launch
    assert t["hbm_frac"] == pytest.approx((56.0 * N + 36.0 * E) / 0.748e-3 / 6790.3e9, abs=1e-4)
    assert t["share"] == pytest.approx(0.38, abs=1e-4)


def test_classes_take_their_own_bound():
    """An HBM class is measured against the copy bandwidth, an FP64 class whose flops take
    longer than its bytes against the FP64 peak, the network against the BF16 peak."""
    prof = {"inner_ortho": {"ms": 2.0, "count": 4, "alg_bytes": 4 * 3.0e9, "alg_flops": 4 * 1e9},
            "ortho_dot": {"ms": 1.0, "count": 2, "alg_bytes": 2 * 1e6, "alg_flops": 2 * 5e8},
            "mlp": {"ms": 1.0, "count": 1, "alg_bytes": 1e8, "alg_flops": 6.8e11},
            "ns32": {"ms": 0.0, "count": 0, "alg_bytes": 0.0, "alg_flops": 0.0}}
    t = B.kernel_table(prof, PEAKS, total_ms=10.0, N=N, E=E)
    assert "ns32" not in t  # classes that did not run are left out
    io = t["inner_ortho"]
    assert io["bound"] == "hbm" and io["frac"] == pytest.approx(3.0e9 / 0.5e-3 / 6790.3e9, abs=1e-4)
    od = t["ortho_dot"]
    assert od["bound"] == "alu" and od["peak"] == pytest.approx(152 * 2 * 2 * 2.07e9 / 1e12, rel=1e-3)
    assert t["mlp"]["bound"] == "tensor" and t["mlp"]["frac"] == pytest.approx(680.0 / 1720.7, abs=1e-4)
    assert sum(r["share"] for r in t.values()) == pytest.approx(0.4, abs=1e-3)


SRC_ROOT = B.ROOT


def _copy_sources(dst, tj, change=None):
    for f in tj["classes"]["jv32"]["sources"]:
        os.makedirs(os.path.join(dst, os.path.dirname(f)), exist_ok=True)
        shutil.copy(os.path.join(SRC_ROOT, f), os.path.join(dst, f))
        if f == change:
            with open(os.path.join(dst, f), "a") as fh:
                fh.write("\n// changed\n")


def test_traffic_is_used_only_for_the_captured_source(tmp_path, monkeypatch):
    """The committed DRAM bytes per element stand for the kernel as captured: a changed
    source, another workload or the other step variant gives no traffic."""
    tj = json.load(open(os.path.join(B.ROOT, "profiles", "traffic.json")))
    os.makedirs(tmp_path / "profiles")
    shutil.copy(os.path.join(B.ROOT, "profiles", "traffic.json"), tmp_path / "profiles" / "traffic.json")
    _copy_sources(str(tmp_path), tj)
    monkeypatch.setattr(B, "ROOT", str(tmp_path))
    tr = B.load_traffic(tj["workload"], coupled=True)
    assert "jv32" in tr
    table = B.kernel_table({"jv32": {"ms": 7.48, "count": 10, "alg_bytes": 0.0, "alg_flops": 0.0}}, PEAKS, 20.0, N, E)
    rl = B.roofline(table, tr, "jv32", n_elem=E)
    assert rl["traffic"] == pytest.approx(tj["classes"]["jv32"]["dram_bytes_per_element"] * E)
    assert "jv32" not in B.load_traffic(tj["workload"], coupled=False)
    assert B.load_traffic("membrane", coupled=True) == {}
    first = next(iter(tj["classes"]["jv32"]["sources"]))
    _copy_sources(str(tmp_path), tj, change=first)
    assert "jv32" not in B.load_traffic(tj["workload"], coupled=True)
    assert B.roofline(table, B.load_traffic(tj["workload"], True), "jv32", n_elem=E)["traffic"] is None


def test_replica_aggregation():
    """Whole-job figures: the units all ranks processed, and the steps all ranks took, over
    the slowest rank's time."""
    assert B.replica_throughput(3.0e9, 2, 1000.0) == pytest.approx(6.0)
    assert B.replica_seconds_per_step(6600.0, 20, 1) == pytest.approx(0.33)
    assert B.replica_seconds_per_step(6600.0, 20, 2) == pytest.approx(0.165)
    assert B.max_over_ranks(12.5, None, "cpu") == 12.5


def test_clock_summary_reports_throttle_reasons():
    cs = B.ClockSampler(0)
    assert cs.summary()["reasons"] == ["unavailable"]
    cs.rows = [["2070", "2070", "900.5", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
               ["1965", "2070", "1390.2", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
               ["2070", "2070", "1000.0", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]]
    s = cs.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"] and s["power_w_max"] == pytest.approx(1390.2)


def test_reference_arm_line_keeps_the_contract():
    """The reference arm (the oracle on the host cores) on the small workload: one JSON line
    with the contract's keys, its cpu_baseline and e2e describing the same value, and
    ms_per_step x steps within the process's own wall time."""
    import subprocess
    import sys
    import time
    t0 = time.perf_counter()
    r = subprocess.run([sys.executable, os.path.join(B.ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "small", "--steps", "2", "--warmup", "1"], cwd=B.ROOT, capture_output=True, text=True,
                       timeout=600)
    wall = time.perf_counter() - t0
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "s/step" and d["higher_is_better"] is False
    assert d["steps"] == 2 and d["warmup"] == 1 and d["value"] > 0
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["kind"] == "oracle"
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "s/step", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["ms_per_step"] * d["steps"] * 1e-3 <= wall
