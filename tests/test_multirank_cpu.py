"""Multi-rank path on CPU (gloo, world size 2): bench.py's replica accounting.

Each rank builds its own replica's host plan (d3m_setup makes no CUDA call)
and reports a per-rank time; the job value divides the units summed over the
ranks by the maximum time over the ranks, with a barrier around the timed
region and no collective on the data path (replicas only)."""
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    from paper_2002_05018_gb300 import d3m, workloads as W
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    bench._barrier(ws)
    w = W.tiny(6 + 2 * rank, 6, 4, 2, 2, 1, seed=rank)  # each replica its own problem
    s = d3m.Solver.from_workload(w)
    st = s.stats()
    flops = st["flops_interior"] + st["flops_domain"] + st["flops_k"]
    s.close()
    t_ms = 10.0 * (rank + 1)  # a rank-dependent "step time"
    bench._barrier(ws)
    t_max = bench._max_over_ranks(ws, t_ms)
    f_sum = bench._sum_over_ranks(ws, flops)
    rec = {"rank": rank, "flops": flops, "t_max": t_max, "f_sum": f_sum}
    with open(f"{out}.{rank}", "w") as fh:
        json.dump(rec, fh)
    dist.destroy_process_group()


def test_replica_accounting_gloo(tmp_path):
    ws = 2
    out = str(tmp_path / "rank")
    mp.spawn(_rank_main, args=(ws, _free_port(), out), nprocs=ws, join=True)
    recs = [json.load(open(f"{out}.{r}")) for r in range(ws)]
    assert all(r["t_max"] == 20.0 for r in recs)  # max over ranks
    total = sum(r["flops"] for r in recs)
    assert all(abs(r["f_sum"] - total) <= 1e-9 * total for r in recs)  # units summed over ranks
    assert recs[0]["flops"] != recs[1]["flops"]  # independent replicas (different sizes)
