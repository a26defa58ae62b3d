"""GPU parity of the kernel paths that an environment variable selects instead of the default.

The library reads these switches once per process, so each case runs a child pytest with
the variable set, on the same oracle parity tests as the default path and at the same
tolerances (FP64 1e-12 relative, whole vector and per field; FP32 2e-5 per field):

* PNP_ELEMENT_KERNEL=thread: one thread per element with the modal sum factorisation
  (residual and J V, FP64 and FP32) instead of one lane group per element;
* PNP_RESIDUAL_ARITH=f64: the residual (and the FP64 rows of the Navier-Stokes block) in
  FP64 arithmetic instead of double-float pairs;
* PNP_INNER_GRAPH=0: the inner FP32 Krylov solve launched eagerly instead of replayed as
  a CUDA graph.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

CASES = {
    "PNP_ELEMENT_KERNEL=thread": ("test_gpu_parity.py",
                                  "residual_f64 or jv_f64 or jv_f32 or exact_derivative or hanging_values "
                                  "or newton_equilibrium or bdf_time_steps"),
    "PNP_RESIDUAL_ARITH=f64": ("test_gpu_parity.py",
                               "residual_f64 or exact_derivative or hanging_values or newton_equilibrium "
                               "or bdf_time_steps"),
    "PNP_INNER_GRAPH=0": ("test_gpu_parity.py", "fp32_gmres or bdf_time_steps"),
    "PNP_RESIDUAL_ARITH=f64 (NS)": ("test_gpu_ns.py", "residual_and_matrix or solve_matches"),
}


@pytest.mark.parametrize("setting", list(CASES))
def test_alternate_path_matches_oracle(setting):
    var, val = setting.split(" ")[0].split("=")
    fname, expr = CASES[setting]
    env = dict(os.environ)
    env[var] = val
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
           os.path.join(HERE, fname), "-k", expr]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, f"{setting}: child pytest failed\n{tail}"
    assert " passed" in r.stdout and " failed" not in r.stdout, tail
