#!/usr/bin/env python
"""D^3M benchmark on GB300: factor GFLOP/s and solve RHS/s, FP64 vs mixed+refine.

Workload (default): 32^3 bricks (104,544 edges) in a 3-wavelength box, lossy
dielectric sphere eps_r = 4 - 0.1j, 4x4x2 subdomains with seeded +-3-cell
jittered cuts, 64 plane waves on a seeded 8x8 angle grid (workloads.make(2)).

One step = the whole hot path on that batch: d3m_factor (interior fronts,
interface fronts giving -K_D, block LDL^T of K) + d3m_solve of the 64 RHS
(substitution, recovery of E, and for mixed precision fp64 refinement until
||A x - f||_inf / ||f||_inf <= 1e-10).  value = algorithmic flops of the step
(factor + one substitution pass; refinement passes are not credited) / step
time, with the inputs resident in HBM.  e2e: the same, through d3m_solve_host
with pinned host RHS and solution (H2D + D2H inside the timed region).
N > 1 (torchrun): every rank runs its own replica (weak scaling, no
collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D3M factor GFLOP/s & solve RHS/s, FP64 vs mixed+refine at resid<=1e-10"
SM_COUNT, FP32_LANES, SM_MAX_GHZ = 152, 128, 2.070
FP64_PER_SM_CLK = 4.0  # 2 DFMA per clock per SM (GB300), measured: 1.20 TFLOP/s at ~1.9 GHz


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9], parts[4]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [r[0] for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": reasons}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(ws, v, op):
    """All-reduce of one float over the ranks (NCCL on the GPU, gloo on CPU)."""
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def _max_over_ranks(ws, v):
    import torch.distributed as dist
    return v if ws == 1 else _reduce(ws, v, dist.ReduceOp.MAX)


def _sum_over_ranks(ws, v):
    import torch.distributed as dist
    return v if ws == 1 else _reduce(ws, v, dist.ReduceOp.SUM)


def run_precision(w, prec, steps, warmup, ws, stream, rhs_dev, sample_clocks=False, dev_index=0, cache=None):
    """Times `steps` steps (factor + solve) of one precision, then runs the same
    steps again with the library's per-kernel-class CUDA events on (eager
    launches) for the kernel breakdown and the roofline.  Returns a dict."""
    import torch
    from paper_2002_05018_gb300 import d3m
    s = d3m.Solver.from_workload(w, precision=prec, stream=stream, profile=False,
                                 autotune_cache=None if cache is None else f"{cache}.{'mixed' if prec else 'fp64'}")
    st0 = s.stats()
    factor_flops = st0["flops_interior"] + st0["flops_domain"] + st0["flops_k"]
    r = rhs_dev.shape[1]
    with torch.cuda.stream(stream):
        x = torch.empty((r, w.n_edges), dtype=torch.complex128, device="cuda").t()
    for _ in range(warmup):
        s.factor()
        s.solve(rhs_dev, x)
    _barrier(ws)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    acc = {k: 0.0 for k in ("ms_update", "ms_panel", "ms_assemble", "ms_inverse", "ms_fwd", "ms_bwd",
                            "ms_residual", "flops_update", "flops_panel")}
    launches = 0
    infos = []
    sampler = ClockSampler(dev_index) if sample_clocks else None
    if sampler:
        sampler.__enter__()
    t_wall = time.perf_counter()
    for i in range(steps):
        ev[i][0].record(stream)
        s.factor()
        stf = s.stats()
        ev[i][1].record(stream)
        _, info = s.solve(rhs_dev, x)
        ev[i][2].record(stream)
        sts = s.stats()
        launches += stf["launches_factor"] + sts["launches_solve"]
        infos.append(info)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    _barrier(ws)
    clocks = None
    if sampler:
        sampler.__exit__()
        clocks = sampler.summary()
    # kernel breakdown: the same steps with events around every kernel group
    s.set_profile(True)
    for i in range(steps):
        s.factor()
        stf = s.stats()
        s.solve(rhs_dev, x)
        sts = s.stats()
        for k in ("ms_update", "ms_panel", "ms_assemble", "ms_inverse", "flops_update", "flops_panel"):
            acc[k] += stf[k]
        for k in ("ms_fwd", "ms_bwd", "ms_residual"):
            acc[k] += sts[k]
    torch.cuda.synchronize()
    s.set_profile(False)
    fac_ms = [a.elapsed_time(b) for a, b, _ in ev]
    sol_ms = [b.elapsed_time(c) for _, b, c in ev]
    step_ms = [f + q for f, q in zip(fac_ms, sol_ms)]
    stats = s.stats()
    solve_flops_1 = stats["solve_flops"] / max(1, infos[-1]["iters"] + 1)
    out = dict(solver=s, x=x, factor_flops=factor_flops, solve_flops=solve_flops_1,
               factor_ms=statistics.mean(fac_ms), solve_ms=statistics.mean(sol_ms),
               step_ms=statistics.mean(step_ms), max_step_ms=max(step_ms), wall_s=t_wall,
               iters=max(i["iters"] for i in infos), max_resid=max(i["max_resid"] for i in infos),
               launches=launches, clocks=clocks, stats=stats,
               prof={k: v / steps for k, v in acc.items()})
    return out


def e2e_mixed(s, w, f_host, steps, warmup, ws, stream):
    """factor + d3m_solve_host with pinned host RHS / solution (copies timed)."""
    import torch
    r = f_host.shape[1]
    rhs = torch.from_numpy(f_host.T.copy()).pin_memory().t()
    xh = torch.empty((r, w.n_edges), dtype=torch.complex128).pin_memory().t()
    for _ in range(max(1, warmup // 2)):
        s.factor()
        s.solve_host(rhs, xh)
    _barrier(ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    for _ in range(steps):
        e0.record(stream)
        s.factor()
        s.solve_host(rhs, xh)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    _barrier(ws)
    return statistics.mean(ms), rhs.numel() * 16, xh.numel() * 16


_CPU_CTX = {}


def _cpu_context(w):
    """Oracle decomposition plus the library's per-front algorithmic flops."""
    key = (w.name, w.seed)
    if key not in _CPU_CTX:
        import numpy as np
        from oracle import decomp
        from paper_2002_05018_gb300 import d3m
        dec = decomp.decompose(w)
        s = d3m.Solver.from_workload(w)
        rng = s.structure(d3m.SN_RANGE)
        kind = s.structure(d3m.SN_KIND)
        st = s.structure(d3m.SN_STRUCT)
        s.close()
        n = len(rng)
        p = (rng[:, 1] - rng[:, 0]).astype(float)
        m = p + np.diff(st[: n + 1])
        # exact count used by the library: sum_{k<p} (m-k-1)(m-k)/2 complex MACs, 8 flops each
        fl = np.array([8.0 * sum(0.5 * (mm - kk - 1) * (mm - kk) for kk in range(int(pp)))
                       for mm, pp in zip(m, p)])
        _CPU_CTX[key] = (dec, kind, fl)
    return _CPU_CTX[key]


def cpu_baseline_sample(w, budget_s=20.0, subs=None):
    """The oracle's main step 1 (domain matrices K_D via sparse LU of A_i) on a
    bounded number of subdomains of the same workload; rate in GFLOP/s using
    the library's algorithmic flop count of those subdomains' fronts."""
    import numpy as np
    from oracle import decomp
    dec, kind, fl = _cpu_context(w)
    order = subs if subs is not None else list(range(len(dec.subs)))
    done, flops, t0 = [], 0.0, time.perf_counter()
    for q in order:
        sd = dec.subs[q]
        import scipy.sparse.linalg as spla
        D = decomp.D_matrix(dec, sd).tocsc()
        cols = np.flatnonzero(np.diff(D.indptr))
        Dc = D[:, cols].toarray().astype(np.complex128)
        lu = spla.splu(sd.A.tocsc())
        KD = Dc.T @ lu.solve(Dc)
        del KD
        done.append(q)
        sel = (kind[:, 1] == q) & (kind[:, 0] <= 1)
        flops += fl[sel].sum()
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return flops / dt / 1e9, dict(cores=os.cpu_count(), sample=(
        f"oracle main step 1 (SciPy sparse LU of A_i, K_D = D_i^T A_i^-1 D_i) on {len(done)} of "
        f"{len(dec.subs)} subdomains of {w.name}; flops = the library's algorithmic count of those "
        f"subdomains' fronts; {dt:.1f} s"), seconds=dt)


_ROOF_KERNELS = {
    "update": ("k_update (trailing/Schur update of the fronts, rank-kb complex SYRK-like)", "ms_update",
               "flops_update"),
    "panel": ("k_panel_cl + k_l21 (restricted Bunch-Kaufman panel of the pivot rows, update-row solve)",
              "ms_panel", "flops_panel"),
}


def _roofline(prof, peak_alu_tflops, cls, traffic=None):
    """Algorithmic flops of a kernel class (the library's counts) over its
    CUDA-event time in the profiled steps, against the ALU peak."""
    name, kms, kfl = _ROOF_KERNELS[cls]
    ms = prof[kms]
    achieved = prof[kfl] / (ms * 1e-3) / 1e12 if ms > 0 else 0.0
    return {"kernel": name, "bound": "alu", "achieved": round(achieved, 3), "peak": round(peak_alu_tflops, 2),
            "unit": "TFLOP/s", "frac": round(achieved / peak_alu_tflops, 4), "traffic": traffic,
            "ms_per_step": round(ms, 3)}


def _load_traffic(name):
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d.get(name)
    return None


def precision_summary(r, alu, prec_tag, config, nrhs):
    """The per-precision sub-object of the JSON line from one run_precision
    result: step/factor/solve figures, the profiled kernel split, the tuned
    schedule, and rooflines for the kernel class with the most time
    ("roofline") and for the other class."""
    dom = "panel" if r["prof"]["ms_panel"] >= r["prof"]["ms_update"] else "update"
    other = "update" if dom == "panel" else "panel"
    return {"factor_gflops": round(r["factor_flops"] / (r["factor_ms"] * 1e-3) / 1e9, 2),
            "factor_ms": round(r["factor_ms"], 3),
            "solve_rhs_per_s": round(nrhs / (r["solve_ms"] * 1e-3), 1),
            "solve_ms": round(r["solve_ms"], 3), "refine_steps": r["iters"],
            "max_resid": r["max_resid"], "ms_per_step": round(r["step_ms"], 3),
            "kernel_ms": {k: round(v, 3) for k, v in r["prof"].items() if k.startswith("ms_")},
            "schedule": {"levels": r["stats"]["n_levels"],
                         "tcgen05_update_levels": r["stats"]["tuned_levels_tc"],
                         "doubled_cluster_levels": r["stats"]["tuned_levels_cs2"],
                         "tuning_ms": round(r["stats"]["ms_tuning"], 1)},
            "roofline": _roofline(r["prof"], alu, dom, _load_traffic(f"config{config}:{dom}<{prec_tag}>")),
            "roofline_" + other: _roofline(r["prof"], alu, other, _load_traffic(f"config{config}:{other}<{prec_tag}>")),
            "kernel_timing": "per-kernel-class CUDA events in a second, profiled run of the same steps "
                             "(the timed steps replay the captured factor graph without events)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--autotune-cache", default=None,
                    help="file prefix for the tuned factor schedules (read when they match, else written); "
                         "lets a profiler run reuse the schedule of a plain run")
    args = ap.parse_args()
    ws, rank, local = _dist()
    from paper_2002_05018_gb300 import workloads as W
    w = W.make(args.config)
    workload = (f"config{args.config}: {w.nx}x{w.ny}x{w.nz} bricks ({w.n_edges} edges), "
                f"{w.lx:g}x{w.ly:g}x{w.lz:g} wavelengths, {'x'.join(map(str, w.partition))} subdomains "
                f"(cuts {[int(v) for v in w.cx]}/{[int(v) for v in w.cy]}/{[int(v) for v in w.cz]}), {w.nrhs} plane waves")
    if args.impl == "reference":
        if rank != 0:
            return
        rates = []
        t0 = time.perf_counter()
        budget = max(5.0, 120.0 / max(1, args.steps + args.warmup))
        nsub = len(w.cx) - 1
        nsubs = (len(w.cx) - 1) * (len(w.cy) - 1) * (len(w.cz) - 1)
        for i in range(args.warmup + args.steps):
            rate, meta = cpu_baseline_sample(w, budget_s=budget, subs=[i % nsubs])
            if i >= args.warmup:
                rates.append((rate, meta))
        v = statistics.mean(r for r, _ in rates)
        wall = time.perf_counter() - t0
        line = {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "GFLOP/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(1000 * statistics.mean(m["seconds"] for _, m in rates), 1),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
                "data": "synthetic", "config": {"workload": workload, "sample": "one subdomain per step"},
                "cpu_baseline": {"value": round(v, 3), "unit": "GFLOP/s", "cores": os.cpu_count(),
                                 "kind": "oracle", "sample": rates[-1][1]["sample"]},
                "e2e": {"value": round(v, 3), "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0},
                "wall_s": round(wall, 1)}
        print(json.dumps(line))
        return

    import torch
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.cuda.current_device()
    from paper_2002_05018_gb300 import d3m
    stream = torch.cuda.Stream()
    f_host = None
    # RHS on the host once (d3m_rhs_planewave), then resident on the device
    probe = d3m.Solver.from_workload(w)
    f_host = probe.rhs_planewave(w.khat_pol6())
    probe.close()
    with torch.cuda.stream(stream):
        rhs_dev = torch.tensor(f_host.T.copy(), device="cuda").t()
    torch.cuda.synchronize()

    mixed = run_precision(w, d3m.MIXED, args.steps, args.warmup, ws, stream, rhs_dev, sample_clocks=(rank == 0),
                          dev_index=dev, cache=args.autotune_cache)
    e2e_ms, h2d, d2h = e2e_mixed(mixed["solver"], w, f_host, args.steps, args.warmup, ws, stream)
    mixed["solver"].close()
    del mixed["solver"], mixed["x"]
    torch.cuda.empty_cache()
    fp64 = None
    if not args.no_fp64:
        fp64 = run_precision(w, d3m.FP64, args.steps, args.warmup, ws, stream, rhs_dev, cache=args.autotune_cache)
        fp64["solver"].close()
        del fp64["solver"], fp64["x"]
        torch.cuda.empty_cache()

    step_flops = mixed["factor_flops"] + mixed["solve_flops"]
    t_step = _max_over_ranks(ws, mixed["step_ms"])
    value = _sum_over_ranks(ws, step_flops) / (t_step * 1e-3) / 1e9
    t_e2e = _max_over_ranks(ws, e2e_ms)
    e2e_value = _sum_over_ranks(ws, step_flops) / (t_e2e * 1e-3) / 1e9
    peaks, peak_kind = _peaks()
    alu32 = SM_COUNT * FP32_LANES * 2 * SM_MAX_GHZ / 1e3
    alu64 = SM_COUNT * FP64_PER_SM_CLK * SM_MAX_GHZ / 1e3

    def summary(r, alu, prec_tag):
        return precision_summary(r, alu, prec_tag, args.config, w.nrhs)

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline:
        rate, meta = cpu_baseline_sample(w, budget_s=20.0)
        cpu = {"value": round(rate, 3), "unit": "GFLOP/s", "cores": meta["cores"], "kind": "oracle",
               "sample": meta["sample"]}
    mix = summary(mixed, alu32, "float")
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "GFLOP/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_step, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64 factors + c128 residual/refinement (mixed); c128 (fp64 leg)",
        "data": "synthetic",
        "config": {"workload": workload, "nrhs": w.nrhs, "precision": "mixed+refine (headline)",
                   "l2": "inputs larger than L2 (factor arena %.1f GB)" % (mixed["stats"]["arena_bytes"] / 1e9),
                   "step": "d3m_factor + d3m_solve(64 RHS) incl. refinement to resid<=1e-10",
                   "value_def": "algorithmic flops (factor + one substitution pass) / step time"},
        "roofline": mix["roofline"],
        "e2e": {"value": round(e2e_value, 2), "unit": "GFLOP/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(mixed["launches"]),
        "clocks": mixed["clocks"],
        "cpu_baseline": cpu,
        "mixed": mix,
        "fp64": summary(fp64, alu64, "double") if fp64 else None,
        "peaks": {"source": peak_kind, "fp32_alu_tflops": round(alu32, 2), "fp64_alu_tflops": round(alu64, 3),
                  "hbm_gbs": peaks.get("hbm_gbs")},
    }
    if line["fp64"]:
        line["mixed_speedup_vs_fp64"] = round(fp64["step_ms"] / mixed["step_ms"], 2)
    print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
