"""bench.py host logic on the CPU: argument handling, the reference arm's
JSON line, and the replica aggregation over two gloo ranks."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_whole_job_rate():
    import bench
    assert bench.whole_job_rate(100.0, 10, 4, 2.0) == 2000.0


def test_algorithmic_bytes_cover_every_kernel():
    """Every kernel the library marks in a profiled solve has a byte formula."""
    import re
    import bench
    names = set()
    for f in os.listdir(os.path.join(ROOT, "paper_2301_01356_gb300", "csrc")):
        if f.endswith(".cu"):
            src = open(os.path.join(ROOT, "paper_2301_01356_gb300", "csrc", f)).read()
            names |= set(re.findall(r'L\.mark\("(k_[a-z0-9_]+)"\)', src))
    assert len(names) > 30
    skip = {"k_cc_pick_big", "k_rmq_level", "k_bcc_base", "k_batch_stats", "k_pos_pick_big", "k_finish"}
    missing = [k for k in sorted(names - skip) if bench.algorithmic_bytes(k, 1000, 4000, 10, 4, 16) is None]
    assert not missing, missing


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(1.0 + rank, world)
    bench.barrier(world)
    q.put((rank, t, bench.whole_job_rate(10.0, 5, world, t)))
    dist.destroy_process_group()


def test_replica_aggregation_gloo():
    import multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(60)
    assert [t for _, t, _ in out] == [2.0, 2.0]          # max over ranks
    assert all(v == 10.0 * 5 * 2 / 2.0 for _, _, v in out)


def test_reference_arm_line():
    out = subprocess.check_output([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                                   "--workload", "uniform64k", "--steps", "2", "--warmup", "3"], text=True)
    line = json.loads(out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "undirected edges/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0


def test_rejects_short_warmup():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--warmup", "1"], capture_output=True)
    assert r.returncode != 0


def test_cpu_baseline_sample_is_bounded():
    """The oracle baseline runs on the full graph where that takes seconds, and on
    the same recipe at a smaller scale for the R-MAT rows (minutes at full size)."""
    import bench
    from paper_2301_01356_gb300 import graphgen as gg
    g = gg.workload_uniform_64k()
    same, desc = bench.cpu_sample("uniform64k", g)
    assert same is g and "full" in desc
    small, desc = bench.cpu_sample("rmat24", None)
    assert small.n == 1 << bench.CPU_SAMPLE_SCALE and small.m > 0
    assert f"scale {bench.CPU_SAMPLE_SCALE}" in desc


def test_batch_chunks():
    """Splitting a bucket into chunks keeps every graph once, in order, and each
    chunk within the arc cap unless it is a single graph above the cap."""
    import numpy as np
    from paper_2301_01356_gb300.batch import chunks
    arcs = np.array([5, 3, 9, 2, 2, 12, 1, 4, 4], np.int64)
    idx = np.array([0, 2, 3, 4, 5, 6, 8])
    parts = chunks(idx, arcs, 10)
    assert np.array_equal(np.concatenate(parts), idx)
    for p in parts:
        assert arcs[p].sum() <= 10 or p.size == 1
    assert [list(p) for p in parts] == [[0], [2], [3, 4], [5], [6, 8]]
    assert chunks(np.array([], np.int64), arcs, 10) == []
    assert [list(p) for p in chunks(idx, arcs, 1 << 40)] == [list(idx)]
