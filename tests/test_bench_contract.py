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
    """The reference arm (the CPU oracle) prints the contract's line with the
    same config as the GPU arm, and never loads the product library."""
    code = ("import runpy, sys; sys.argv = ['bench.py', '--impl', 'reference', '--config', '1', '--steps', '1', "
            "'--warmup', '3']; runpy.run_path('bench.py', run_name='__main__'); "
            "print('LIBD3M_LOADED', any('libd3m' in ln for ln in open('/proc/self/maps')))")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    assert "LIBD3M_LOADED False" in out.stdout
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    from paper_2002_05018_gb300 import workloads as W
    w = W.make(1)
    sv = d3m.Solver.from_workload(w)   # host-only set-up: the exported structure gives the same arena
    arena = bench.front_arena_bytes(sv.structure(d3m.SN_RANGE), sv.structure(d3m.SN_STRUCT))
    sv.close()
    assert d["config"] == bench.bench_config(w, 1, arena)
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


def _fake_run(ms_panel, ms_update):
    prof = {"ms_update": ms_update, "ms_panel": ms_panel, "ms_assemble": 1.0, "ms_inverse": 2.0, "ms_fwd": 3.0,
            "ms_bwd": 4.0, "ms_residual": 0.5, "flops_update": 4.0e11, "flops_panel": 1.0e10}
    stats = {"n_levels": 28, "tuned_levels_tc": 0, "tuned_levels_cs2": 3, "ms_tuning": 200.0}
    return dict(factor_flops=6.8e11, factor_ms=70.0, solve_ms=45.0, iters=3, max_resid=3e-11, step_ms=115.0,
                prof=prof, stats=stats)


def test_precision_summary_roofline_keys():
    sys.path.insert(0, ROOT)
    import bench
    for ms_panel, ms_update, dom in ((40.0, 30.0, "panel"), (20.0, 30.0, "update")):
        sub = bench.precision_summary(_fake_run(ms_panel, ms_update), 80.55, "float", 2, 64)
        other = "update" if dom == "panel" else "panel"
        roof, roof2 = sub["roofline"], sub["roofline_" + other]
        for r in (roof, roof2):
            for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
                assert k in r
            assert r["unit"] == "TFLOP/s" and r["peak"] == 80.55
            assert abs(r["frac"] - r["achieved"] / 80.55) < 1e-3
        ms, fl = (ms_panel, 1.0e10) if dom == "panel" else (ms_update, 4.0e11)
        assert abs(roof["achieved"] - fl / (ms * 1e-3) / 1e12) < 1e-3
        assert roof["ms_per_step"] == ms
        # traffic data exist for workload 2's update class only
        assert (roof["traffic"] is not None) == (dom == "update")
        assert sub["solve_rhs_per_s"] == round(64 / 45e-3, 1)
        assert sub["schedule"]["doubled_cluster_levels"] == 3
    # another workload never picks up workload 2's traffic figure
    sub5 = bench.precision_summary(_fake_run(20.0, 30.0), 80.55, "float", 5, 128)
    assert sub5["roofline"]["traffic"] is None
