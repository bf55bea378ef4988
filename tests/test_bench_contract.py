"""bench.py's JSON contract on CPU: the reference arm (the oracle timed on the
host cores) prints one line with the keys, units and types the driver reads;
and host-side C-ABI argument checks of the profiling switch."""
import ctypes
import json
import os
import subprocess
import sys

import numpy as np
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


def test_reference_arm_seed_and_log(tmp_path):
    """--seed is accepted and --log appends each printed line to a JSONL
    file; the seed reaches the workload generator (workload 2's cut jitter
    differs between seeds)."""
    log = tmp_path / "runs.jsonl"
    outs = []
    for seed in (2, 7):
        code = ("import runpy, sys; sys.argv = ['bench.py', '--impl', 'reference', '--config', '1', '--seed', "
                f"'{seed}', '--steps', '1', '--warmup', '3', '--log', '{log}']; "
                "runpy.run_path('bench.py', run_name='__main__')")
        out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600, cwd=ROOT)
        assert out.returncode == 0, out.stderr[-2000:]
        outs.append([ln for ln in out.stdout.splitlines() if ln.startswith("{")][0])
    logged = log.read_text().splitlines()
    assert logged == outs
    from paper_2002_05018_gb300 import workloads as W
    a, b = W.make(2, seed=2), W.make(2, seed=7)
    assert any(not np.array_equal(x, y) for x, y in ((a.cx, b.cx), (a.cy, b.cy), (a.cz, b.cz)))


def test_reference_arm_on_a_general_mesh():
    """--element mesh: the reference arm runs the oracle on the Delaunay form
    of the workload and reports the same config the GPU arm would."""
    code = ("import runpy, sys; sys.argv = ['bench.py', '--impl', 'reference', '--config', '1', '--element', "
            "'mesh', '--order', '2', '--steps', '1', '--warmup', '3']; runpy.run_path('bench.py', run_name='__main__')")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["value"] > 0 and "Delaunay mesh" in d["config"]["workload"] and "order 2" in d["config"]["workload"]


def test_set_profile_argument_checks():
    lib = d3m.load()
    assert lib.d3m_set_profile(None, 1) == d3m.D3M_EINVAL
    from paper_2002_05018_gb300 import workloads as W
    s = d3m.Solver.from_workload(W.tiny(4, 4, 4, 2, 1, 1, seed=1))  # host-only context: no CUDA call
    s.set_profile(True)
    s.set_profile(False)
    s.close()


def _fake_run(ms_panel, ms_update, ms_tc=0.0):
    prof = {"ms_update": ms_update, "ms_panel": ms_panel, "ms_assemble": 1.0, "ms_inverse": 2.0, "ms_tc": ms_tc,
            "ms_fwd": 3.0, "ms_bwd": 4.0, "ms_residual": 0.5, "flops_update": 4.0e11, "flops_panel": 1.0e10,
            "flops_tc": 6.0e11}
    stats = {"n_levels": 28, "tuned_levels_tc": 0, "tuned_levels_cs2": 3, "ms_tuning": 200.0}
    return dict(factor_flops=6.8e11, factor_ms=70.0, solve_ms=45.0, iters=3, max_resid=3e-11, step_ms=115.0,
                prof=prof, stats=stats)


def test_precision_summary_roofline_keys():
    """The dominant class (by profiled time) gets "roofline", every other class
    "roofline_<class>", each against the peak of its own pipe; the tensor-core
    class reports its fraction of the BF16x3 ceiling as well."""
    sys.path.insert(0, ROOT)
    import bench
    peaks = {"alu": 80.55, "tensor": 900.0}
    for ms_panel, ms_update, ms_tc, dom in ((40.0, 30.0, 5.0, "panel"), (20.0, 30.0, 5.0, "update"),
                                            (20.0, 3.0, 25.0, "tc")):
        sub = bench.precision_summary(_fake_run(ms_panel, ms_update, ms_tc), peaks, "float", 2, 64)
        others = [c for c in ("panel", "update", "tc") if c != dom]
        for r in [sub["roofline"]] + [sub["roofline_" + c] for c in others]:
            for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
                assert k in r
            assert r["unit"] == "TFLOP/s" and r["traffic"] is None
            assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-3
        roof = sub["roofline"]
        ms, fl = {"panel": (ms_panel, 1.0e10), "update": (ms_update, 4.0e11), "tc": (ms_tc, 6.0e11)}[dom]
        assert abs(roof["achieved"] - fl / (ms * 1e-3) / 1e12) < 1e-3
        assert roof["ms_per_step"] == ms
        tc = roof if dom == "tc" else sub["roofline_tc"]
        assert tc["bound"] == "tensor" and tc["peak"] == 900.0
        assert abs(tc["frac_of_bf16x3_ceiling"] - 6 * tc["frac"]) < 4e-3
        assert sub["solve_rhs_per_s"] == round(64 / 45e-3, 1)
        assert sub["schedule"]["doubled_cluster_levels"] == 3
    # a run without deferred levels (fp64 leg) reports no tensor-core class
    sub = bench.precision_summary(_fake_run(40.0, 30.0, 0.0), peaks, "double", 2, 64)
    assert "roofline_tc" not in sub and sub["roofline"]["bound"] == "alu"
