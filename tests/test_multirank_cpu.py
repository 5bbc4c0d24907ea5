"""The multi-rank path of the benchmark on CPU: two gloo ranks, as torchrun
launches them.  Segments are independent (Sec. 3.2), so each rank searches
its own segment with no collective on the data path; ranks meet only for the
timing (a barrier and the max over ranks)."""

import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist
    import bench
    import oracle
    import synth
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    res = {"rank": rank}
    # timing: every rank gets the slowest rank's time
    res["max_ms"] = bench.max_over_ranks(10.0 + rank, dist, "cpu")
    res["rate"] = bench.job_rate(world, 3, 1000, res["max_ms"])
    # work: rank r's own segment (the tiny workload with the rank's seed)
    spec = synth.config("tiny")
    spec.seed = bench.rank_seed(spec.seed, rank)
    seg = synth.make_segment(spec, nint=48)
    op = oracle.OraclePlan(seg["ant_uvw"], seg["freq_hz"], spec.inttime_s, spec.npix, spec.cell_rad, spec.dm_list,
                           spec.dt_list, spec.threshold, edge=spec.edge)
    _, st = oracle.search_segment(op, seg["vis"], images=[(0, 0, t) for t in range(3)], with_stats=True)
    res["peaks"] = [st[(0, 0, t)].peak for t in range(3)]
    res["checksum"] = float(np.abs(seg["vis"]).sum())
    dist.barrier()
    # the reference arm runs on rank 0 only; other ranks return at once
    class A:
        config = "tiny"
    if rank != 0:
        res["reference_rc"] = bench.run_reference(A(), rank, world)
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(res, f)


def test_two_gloo_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    r = [json.load(open(tmp_path / f"rank{k}.json")) for k in range(world)]
    assert r[0]["max_ms"] == r[1]["max_ms"] == 11.0
    assert r[0]["rate"] == r[1]["rate"] == pytest.approx(2 * 3 * 1000 / 0.011)
    # independent units: the ranks' segments and results differ
    assert r[0]["checksum"] != r[1]["checksum"]
    assert r[0]["peaks"] != r[1]["peaks"]
    assert r[1]["reference_rc"] == 0


def test_rank_seeds_and_rates_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert [bench.rank_seed(101, k) for k in range(4)] == [101, 1101, 2101, 3101]
    assert bench.max_over_ranks(5.0, None, "cpu") == 5.0
    # weak scaling: per-rank work fixed, the job rate grows with the ranks
    assert bench.job_rate(4, 2, 100, 1000.0) == 4 * bench.job_rate(1, 2, 100, 1000.0)
