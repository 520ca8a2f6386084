"""Host-side contract checks, no GPU needed: the benchmark's reference arm prints the agreed JSON
line, and without a GPU the product path fails loudly instead of computing on the host."""
import ctypes as C
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def test_reference_arm_json_line():
    """`bench.py --impl reference` (the oracle timed on the host cores) prints one JSON line with
    the base contract's keys and the same metric and workload as the GPU arm's default."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    import bench
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == "s/step" and line["higher_is_better"] is False
    assert line["config"]["workload"] == bench.workload_name(bench.WORKLOADS["big"])      # the default workload
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == (os.cpu_count() or 1) and cb["value"] == line["value"]
    assert cb["extrapolated"] is True and cb["sample"].startswith("extrapolated")
    assert line["e2e"] == {"value": line["value"], "unit": "s/step", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


@pytest.mark.skipif(_has_gpu(), reason="checks the behaviour without a GPU")
def test_no_host_fallback_without_gpu():
    """Without a GPU, creating a solver through the C ABI returns STDG_ECUDA (no host path), and
    the benchmark exits non-zero without printing a result line."""
    from paper_1601_07384_gb300.build import build
    build()
    import numpy as np
    import paper_1601_07384_gb300 as g
    from paper_1601_07384_gb300 import _lib
    from inputs import kuhn_mesh
    v, t = kuhn_mesh(2, seed=0)
    mesh, ref = g.Mesh(v, t), g.Reference(1, 0)
    h = C.c_void_p()
    st = _lib.load().stdg_solver_create(mesh._h, ref._h, 0.01, None, None, C.byref(h))
    assert st == -3                                # STDG_ECUDA
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--workload", "tiny", "--steps", "1",
                          "--warmup", "0", "--no-compare", "--no-cpu-baseline"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode != 0
    assert not any(ln.startswith("{") and '"value"' in ln for ln in out.stdout.splitlines())
