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


def run_precision(w, prec, steps, warmup, ws, stream, rhs_dev, sample_clocks=False, dev_index=0, cache=None,
                  update_kernel=0, solve_kernel=0):
    """Times `steps` steps (factor + solve) of one precision, then runs the same
    steps again with the library's per-kernel-class CUDA events on (eager
    launches) for the kernel breakdown and the roofline.  Returns a dict."""
    import torch
    from paper_2002_05018_gb300 import d3m
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    s = d3m.Solver.from_workload(w, precision=prec, stream=stream, profile=False, update_kernel=update_kernel,
                                 solve_kernel=solve_kernel,
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
    # device memory held by this context after its first factor + solve (the
    # library allocates with cudaMalloc, outside torch's allocator)
    device_bytes = free0 - torch.cuda.mem_get_info()[0]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    acc = {k: 0.0 for k in ("ms_update", "ms_panel", "ms_assemble", "ms_inverse", "ms_tc", "ms_fwd", "ms_bwd",
                            "ms_residual", "flops_update", "flops_panel", "flops_tc")}
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
        for k in ("ms_update", "ms_panel", "ms_assemble", "ms_inverse", "ms_tc", "flops_update", "flops_panel",
                  "flops_tc"):
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
               step_ms_each=[round(v, 3) for v in step_ms], factor_ms_each=[round(v, 3) for v in fac_ms],
               step_ms=statistics.mean(step_ms), max_step_ms=max(step_ms), wall_s=t_wall,
               iters=max(i["iters"] for i in infos), max_resid=max(i["max_resid"] for i in infos),
               launches=launches, clocks=clocks, stats=stats, device_bytes=device_bytes,
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


# ------------------------------------------------------------ CPU oracle baseline
def front_arena_bytes(rng, st):
    """8 sum m^2 (complex64 fronts) from the exported supernode ranges and
    update-row offsets."""
    import numpy as np
    n = len(rng)
    m = (rng[:, 1] - rng[:, 0]) + np.diff(st[: n + 1])
    return int(8 * (m.astype(np.int64) ** 2).sum())


def oracle_front_flops(dec):
    """The metric's algorithmic flop count per front, from the oracle's own
    ordering and supernodal symbolic factorisation (no library involved):
    eliminating p pivots of a front of order m costs sum_{k<p} (m-k)(m-k-1)/2
    complex MACs = C(m+1, 3) - C(m-p+1, 3), 8 real flops each.  Returns
    (kind, owner, flops) per front (kind 0 interior, 1 interface dofs, 2 K)
    and the complex64 front storage 8 sum m^2 in bytes."""
    import numpy as np
    from oracle import ordering
    plan = ordering.build_plan(dec)
    r, c = ordering.saddle_pattern(dec, plan)
    ordering.symbolic_merge(plan, r, c)
    p = (plan.sn_end - plan.sn_start).astype(float)
    m = p + np.array([len(st) for st in plan.struct], float)
    c3 = lambda n: n * (n - 1.0) * (n - 2.0) / 6.0
    return plan.sn_kind, plan.sn_owner, 8.0 * (c3(m + 1.0) - c3(m - p + 1.0)), int(8 * (m.astype(np.int64) ** 2).sum())


def _kd_columns(args):
    """Worker (spawned process): the oracle's main step 1 on a slice of the
    multiplier columns of one subdomain."""
    from oracle import d3m as od3m
    A, Dc, which = args
    KD = od3m.domain_matrix(A, Dc, which=which)
    return float(abs(KD).max()) if KD.size else 0.0


class OracleStep1:
    """Bounded CPU sample of the oracle's D^3M path: its main step 1 (dense
    domain matrix K_D of a subdomain by SciPy sparse LU, the dominant cost of
    the oracle's factorisation) for one subdomain at a time, its multiplier
    columns split over a pool of spawned worker processes (one per host core).
    Each subdomain is credited with the algorithmic flops of its fronts
    (interior + interface dofs) from the oracle's own symbolic factorisation."""

    def __init__(self, w, workers=None):
        import multiprocessing as mp
        import numpy as np
        from oracle import decomp
        self.w = w
        self.dec = decomp.decompose(w)
        kind, owner, fl, self.arena_bytes = oracle_front_flops(self.dec)
        self.flops = [float(fl[(kind <= 1) & (owner == q)].sum()) for q in range(len(self.dec.subs))]
        self.workers = workers or os.cpu_count() or 1
        # one BLAS thread per worker process (the workers already use every core)
        keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
        saved = {k: os.environ.get(k) for k in keys}
        os.environ.update({k: "1" for k in keys})
        try:
            self.pool = mp.get_context("spawn").Pool(self.workers)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        A0 = self.dec.subs[0].A
        self.pool.map(_kd_columns, [(A0, np.zeros((A0.shape[0], 1)), None)] * self.workers)  # warm the workers

    def run(self, q):
        """Step 1 of subdomain q; returns (seconds, flops)."""
        import numpy as np
        from oracle import decomp
        sd = self.dec.subs[q]
        t0 = time.perf_counter()
        D = decomp.D_matrix(self.dec, sd).tocsc()
        cols = np.flatnonzero(np.diff(D.indptr))
        Dc = D[:, cols].toarray()
        chunks = [c for c in np.array_split(np.arange(Dc.shape[1]), self.workers) if len(c)]
        self.pool.map(_kd_columns, [(sd.A, Dc, c) for c in chunks])
        return time.perf_counter() - t0, self.flops[q]

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline_sample(w, budget_s=20.0):
    """The oracle sample (OracleStep1) over subdomains 0, 1, ... until
    budget_s seconds have passed; rate in GFLOP/s of the metric's count."""
    o = OracleStep1(w)
    done, secs, flops = 0, 0.0, 0.0
    try:
        for q in range(len(o.dec.subs)):
            t, f = o.run(q)
            secs += t
            flops += f
            done += 1
            if secs > budget_s:
                break
    finally:
        o.close()
    return flops / secs / 1e9, dict(cores=o.workers, seconds=secs, sample=(
        f"oracle main step 1 (K_D = D_i^T A_i^-1 D_i by SciPy sparse LU) on {done} of {len(o.dec.subs)} "
        f"subdomains of {w.name}, multiplier columns split over {o.workers} spawned processes; flops = the "
        f"metric's algorithmic count of those subdomains' fronts from the oracle's own symbolic "
        f"factorisation; {secs:.1f} s"))


# kernel classes of the factorisation: (kernel names, time key, algorithmic
# flop key, bound, peak key)
_ROOF_KERNELS = {
    "update": ("k_update (right-looking trailing update after each panel: whole trailing triangle on FMA "
               "levels, the pivot block only on deferred levels)", "ms_update", "flops_update", "alu", "alu"),
    "panel": ("k_panel_cl + k_l21 (restricted Bunch-Kaufman panel of the pivot rows, update-row solve)",
              "ms_panel", "flops_panel", "alu", "alu"),
    "tc": ("k_tc_split + k_tc_gemm (deferred Schur products C = F22 - L21 W21^T, complex BF16x3 on tcgen05, "
           "TMA-staged)", "ms_tc", "flops_tc", "tensor", "tensor"),
}


def _roofline(prof, peaks, cls, traffic=None):
    """Algorithmic flops of a kernel class (8 real flops per complex MAC, the
    library's counts) over its CUDA-event time in the profiled steps, against
    the peak of the pipe it runs on (peaks: {"alu": ..., "tensor": ...})."""
    name, kms, kfl, bound, pk = _ROOF_KERNELS[cls]
    ms = prof.get(kms, 0.0)
    peak = peaks[pk]
    achieved = prof.get(kfl, 0.0) / (ms * 1e-3) / 1e12 if ms > 0 else 0.0
    out = {"kernel": name, "bound": bound, "achieved": round(achieved, 3), "peak": round(peak, 2),
           "unit": "TFLOP/s", "frac": round(achieved / peak, 4) if peak else None, "traffic": traffic,
           "ms_per_step": round(ms, 3)}
    if cls == "tc" and peak:
        # BF16x3 complex: 6 bf16 products per real product, 4 real products
        # per complex MAC, i.e. 6 tensor flops per algorithmic flop; the
        # ceiling of this scheme is peak / 6
        out["frac_of_bf16x3_ceiling"] = round(6.0 * achieved / peak, 4)
    return out


def _load_traffic(name):
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d.get(name)
    return None


def precision_summary(r, peaks, prec_tag, config, nrhs):
    """The per-precision sub-object of the JSON line from one run_precision
    result: step/factor/solve figures, the profiled kernel split, the tuned
    schedule, and rooflines for the kernel class with the most time
    ("roofline") and for each other class ("roofline_<class>")."""
    classes = [c for c in _ROOF_KERNELS if r["prof"].get(_ROOF_KERNELS[c][1], 0.0) > 0 or c != "tc"]
    dom = max(classes, key=lambda c: r["prof"].get(_ROOF_KERNELS[c][1], 0.0))
    roofs = {"roofline_" + c: _roofline(r["prof"], peaks, c, _load_traffic(f"config{config}:{c}<{prec_tag}>"))
             for c in classes if c != dom}
    return {"factor_gflops": round(r["factor_flops"] / (r["factor_ms"] * 1e-3) / 1e9, 2),
            "factor_ms": round(r["factor_ms"], 3),
            "solve_rhs_per_s": round(nrhs / (r["solve_ms"] * 1e-3), 1),
            "solve_ms": round(r["solve_ms"], 3), "refine_steps": r["iters"],
            "max_resid": r["max_resid"], "ms_per_step": round(r["step_ms"], 3),
            "ms_each_step": r.get("step_ms_each"), "factor_ms_each_step": r.get("factor_ms_each"),
            "device_gb": (round(r["device_bytes"] / 1e9, 2) if r.get("device_bytes") is not None else None),
            "kernel_ms": {k: round(v, 3) for k, v in r["prof"].items() if k.startswith("ms_")},
            "schedule": {"levels": r["stats"]["n_levels"],
                         "tcgen05_update_levels": r["stats"]["tuned_levels_tc"],
                         "doubled_cluster_levels": r["stats"]["tuned_levels_cs2"],
                         "tuning_ms": round(r["stats"]["ms_tuning"], 1)},
            "roofline": _roofline(r["prof"], peaks, dom, _load_traffic(f"config{config}:{dom}<{prec_tag}>")),
            **roofs,
            "kernel_timing": "per-kernel-class CUDA events in a second, profiled run of the same steps "
                             "(the timed steps replay the captured factor graph without events)"}


def bench_config(w, config, arena_bytes):
    """The `config` object of the JSON line (the same for both arms);
    arena_bytes = 8 sum m^2 over the fronts (complex64 front storage)."""
    el = getattr(w, "element", "brick")
    if el == "mesh":
        return {"workload": (f"config{config} box as a Delaunay mesh of {(w.nx + 1) * (w.ny + 1) * (w.nz + 1)} "
                             f"jittered points ({w.n_cells} tetrahedra, order {w.order}, {w.n_edges} dofs), "
                             f"{w.lx:g}x{w.ly:g}x{w.lz:g} wavelengths, {'x'.join(map(str, w.partition))} "
                             f"coordinate-box subdomains, {w.nrhs} plane waves"),
                "nrhs": w.nrhs, "precision": "mixed+refine (headline)",
                "l2": ("every step refactors the whole front arena (%.2f GB in complex64; L2 is 0.13 GB)"
                       % (arena_bytes / 1e9)),
                "step": f"d3m_factor + d3m_solve({w.nrhs} RHS) incl. refinement to resid<=1e-10",
                "value_def": "algorithmic flops (factor + one substitution pass) / step time"}
    cells = "bricks" if el == "brick" else "cells x 6 jittered tetrahedra"
    return {"workload": (f"config{config}: {w.nx}x{w.ny}x{w.nz} {cells} ({w.n_edges} edges), "
                         f"{w.lx:g}x{w.ly:g}x{w.lz:g} wavelengths, {'x'.join(map(str, w.partition))} subdomains "
                         f"(cuts {[int(v) for v in w.cx]}/{[int(v) for v in w.cy]}/{[int(v) for v in w.cz]}), "
                         f"{w.nrhs} plane waves"),
            "nrhs": w.nrhs, "precision": "mixed+refine (headline)",
            "l2": ("every step refactors the whole front arena (%.2f GB in complex64; L2 is 0.13 GB)"
                   % (arena_bytes / 1e9)),
            "step": f"d3m_factor + d3m_solve({w.nrhs} RHS) incl. refinement to resid<=1e-10",
            "value_def": "algorithmic flops (factor + one substitution pass) / step time"}


def _emit(line, log_path):
    """Print the run's JSON line; with --log also append it to that file."""
    text = json.dumps(line)
    print(text)
    if log_path:
        with open(log_path, "a") as fh:
            fh.write(text + "\n")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--update-kernel", type=int, default=0, choices=[0, 1, 2],
                    help="mixed update scheme: 0 per-level autotuned (default), 1 right-looking FMA, "
                         "2 deferred tensor-core Schur products on every level (for profiling a small workload)")
    ap.add_argument("--ncu-range", action="store_true",
                    help="after the timed steps, run one more mixed step (factor graph + solve) between "
                         "cudaProfilerStart/Stop, for ncu --profile-from-start off")
    ap.add_argument("--solve-kernel", type=int, default=0, choices=[0, 1],
                    help="mixed substitution products: 0 tensor cores (default), 1 fp32 FMA (profiling)")
    ap.add_argument("--nrhs", type=int, default=0,
                    help="replace the workload's plane waves by this many seeded random ones "
                         "(profiling the substitution of a small workload with many right-hand sides)")
    ap.add_argument("--autotune-cache", default=None,
                    help="file prefix for the tuned factor schedules (read when they match, else written); "
                         "lets a profiler run reuse the schedule of a plain run")
    ap.add_argument("--seed", type=int, default=None,
                    help="seed of the synthetic workload (default: the workload's index, as everywhere else)")
    ap.add_argument("--log", default=None,
                    help="also append the JSON line to this file (one run per line)")
    ap.add_argument("--element", default="brick", choices=["brick", "tet", "mesh"],
                    help="tet: the same workload on six jittered tetrahedra per cell; mesh: its box as a "
                         "Delaunay mesh of the jittered lattice points (general connectivity), the same "
                         "subdomain counts as equal coordinate cuts, the same plane waves")
    ap.add_argument("--order", type=int, default=1, choices=[1, 2, 3],
                    help="--element mesh: 2 = complete first-order elements (two dofs per edge), "
                         "3 = curl-complete second order (also two per face)")
    args = ap.parse_args()
    ws, rank, local = _dist()
    from paper_2002_05018_gb300 import workloads as W
    w = W.make(args.config, seed=args.seed)
    if args.nrhs > 0:
        w = W.with_waves(w, args.nrhs, seed=args.config)
    if args.element == "tet":
        w = W.tetrahedral(w, 0.1)
    elif args.element == "mesh":
        import dataclasses
        wm = W.delaunay(w.nx, w.ny, w.nz, *w.partition, seed=args.config, h=w.lx / w.nx, order=args.order)
        w = dataclasses.replace(wm, k=w.k, khat=w.khat, pol=w.pol)
    if args.impl == "reference":
        # the reference arm is the CPU oracle (no GPU, no library): rank 0 only
        if rank != 0:
            return
        t0 = time.perf_counter()
        o = OracleStep1(w)
        samples = []
        nsub = len(o.dec.subs)
        try:
            for i in range(args.warmup + args.steps):
                t, f = o.run(i % nsub)
                if i >= args.warmup:
                    samples.append((t, f, i % nsub))
        finally:
            o.close()
        secs = sum(t for t, _, _ in samples)
        v = sum(f for _, f, _ in samples) / secs / 1e9
        sample = (f"per step: oracle main step 1 (K_D = D_i^T A_i^-1 D_i by SciPy sparse LU) of one subdomain "
                  f"of {w.name} (round robin), multiplier columns split over {o.workers} spawned processes; "
                  f"flops = the metric's algorithmic count of that subdomain's fronts from the oracle's own "
                  f"symbolic factorisation; {len(samples)} steps, {secs:.1f} s")
        line = {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "GFLOP/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(1000 * secs / max(1, len(samples)), 1),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
                "data": "synthetic", "config": bench_config(w, args.config, o.arena_bytes),
                "cpu_baseline": {"value": round(v, 3), "unit": "GFLOP/s", "cores": o.workers,
                                 "kind": "oracle", "sample": sample},
                "e2e": {"value": round(v, 3), "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0},
                "wall_s": round(time.perf_counter() - t0, 1)}
        _emit(line, args.log)
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
    arena_c64 = front_arena_bytes(probe.structure(d3m.SN_RANGE), probe.structure(d3m.SN_STRUCT))
    probe.close()
    with torch.cuda.stream(stream):
        rhs_dev = torch.tensor(f_host.T.copy(), device="cuda").t()
    torch.cuda.synchronize()

    mixed = run_precision(w, d3m.MIXED, args.steps, args.warmup, ws, stream, rhs_dev, sample_clocks=(rank == 0),
                          dev_index=dev, cache=args.autotune_cache, update_kernel=args.update_kernel,
                          solve_kernel=args.solve_kernel)
    if args.ncu_range:
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStart()
        mixed["solver"].factor()
        mixed["solver"].solve(rhs_dev, mixed["x"])
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStop()
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

    # the tensor-core class runs bf16 products inside the long factor step:
    # the sustained measured bf16 peak
    bf16 = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops")

    def summary(r, alu, prec_tag):
        return precision_summary(r, {"alu": alu, "tensor": bf16}, prec_tag, args.config, w.nrhs)

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
        "config": bench_config(w, args.config, arena_c64),
        "roofline": mix["roofline"],
        "e2e": {"value": round(e2e_value, 2), "unit": "GFLOP/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(mixed["launches"]),
        "clocks": mixed["clocks"],
        "cpu_baseline": cpu,
        "mixed": mix,
        "fp64": summary(fp64, alu64, "double") if fp64 else None,
        "peaks": {"source": peak_kind, "fp32_alu_tflops": round(alu32, 2), "fp64_alu_tflops": round(alu64, 3),
                  "hbm_gbs": peaks.get("hbm_gbs"), "bf16_tensor_tflops": round(bf16, 1),
                  "bf16_source": "MEASURED_PEAKS bf16_tflops_sustained (cuBLAS bf16 GEMM under the power cap)"},
    }
    if line["fp64"]:
        line["mixed_speedup_vs_fp64"] = round(fp64["step_ms"] / mixed["step_ms"], 2)
    _emit(line, args.log)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
