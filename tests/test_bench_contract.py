"""bench.py's JSON contract on CPU: the reference arm (the oracle timed on the
host cores) prints one line with the keys, units and types the driver reads;
and host-side C-ABI argument checks of the profiling switch."""
import ctypes
import json
import os
import subprocess
import sys

import pytest

from paper_2002_05018_gb300 import d3m

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "1",
                          "--steps", "1", "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 3
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["data"] == "synthetic"
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["unit"] == "GFLOP/s"
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_set_profile_argument_checks():
    lib = d3m.load()
    assert lib.d3m_set_profile(None, 1) == d3m.D3M_EINVAL
    from paper_2002_05018_gb300 import workloads as W
    s = d3m.Solver.from_workload(W.tiny(4, 4, 4, 2, 1, 1, seed=1))  # host-only context: no CUDA call
    s.set_profile(True)
    s.set_profile(False)
    s.close()
