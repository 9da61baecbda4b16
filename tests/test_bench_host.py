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


def test_phase_bytes_and_assignment():
    """The per-phase algorithmic bytes add up to the whole solve's, each arc pass
    carries its phase's adjacency term, and the profiled launch list is split into
    Algorithm 1's phases in launch order."""
    import bench
    n, nnz, ncc, B = 1000, 8000, 10, 8
    pb = bench.phase_bytes(n, nnz, ncc, B)
    A = 2 * (n - ncc)
    assert set(pb) == set(bench.PHASES)
    assert sum(pb.values()) == 4 * B * n + 21 * nnz + 48 * A + (16 + 16 + 40 + 28 + 12) * n
    for k, ph in (("k_cc_hook", "first_cc"), ("k_w12", "tagging"), ("k_last_cc_cross", "last_cc")):
        assert bench.algorithmic_bytes(k, n, nnz, ncc, B) >= B * n + 4 * nnz
    assert bench.algorithmic_bytes("k_edge_out", n, nnz, ncc, B) == B * n + 9 * nnz
    rows = [("k_cc_init", 1), ("k_cc_hook", 1), ("k_uf_compress", 1), ("k_link", 1), ("k_jump", 1),
            ("k_first_of", 1), ("k_rmq_query", 1), ("k_ext_compact", 1), ("k_mark_big", 1),
            ("k_final_label", 1), ("k_ap_keys", 1), ("k_edge_out", 1), ("k_finish", 1)]
    assert bench.phases_of(rows) == ["first_cc"] * 3 + ["rooting"] * 2 + ["tagging"] * 2 + ["last_cc"] * 3 + \
        ["outputs"] * 3


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


def test_clock_sampler_parses_reasons():
    """The clocks object reports the median SM clock under load, the maximum, and
    every throttle reason seen active in any sample."""
    import bench

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    s = bench.ClockSampler(0)
    s.file.write("0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                 "0, 1800, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active\n"
                 "0, 1900, 2070, 1200.0, 0x0, Active, Not Active, Not Active, Not Active\n"
                 "garbage line\n")
    s.proc = Done()
    c = s.stop()
    assert c["sm_mhz"] == 1900.0 and c["sm_max_mhz"] == 2070.0 and c["samples"] == 3
    assert c["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_traffic_is_tied_to_the_kernel_definition(tmp_path, monkeypatch):
    """With func=, the figure stays valid while only other code in the file changes,
    and is dropped once the captured kernel's own text changes."""
    import bench
    src = tmp_path / "paper_2301_01356_gb300" / "csrc"
    src.mkdir(parents=True)
    body = ("template <int K>\n__global__ void __launch_bounds__(256) k_x(int *a)\n{\n    a[0] = K;\n}\n"
            "\n__global__ void k_y(int *a)\n{\n    a[1] = 2;\n}\n")
    (src / "k.cu").write_text(body)
    sha = bench.kernel_source_hash(str(src / "k.cu"), "k_x")
    assert sha and sha != bench.kernel_source_hash(str(src / "k.cu"), "k_y")
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.txt").write_text(
        f"kernel=k_x workload=w bytes_per_launch=77 file=k.cu func=k_x sha={sha} source=test\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_traffic("k_x", "w") == 77
    (src / "k.cu").write_text(body.replace("a[1] = 2", "a[1] = 3") + "// a comment\n")
    assert bench.load_traffic("k_x", "w") == 77
    (src / "k.cu").write_text(body.replace("a[0] = K", "a[0] = K + 1"))
    assert bench.load_traffic("k_x", "w") is None


def test_traffic_is_dropped_when_the_source_changes(tmp_path, monkeypatch):
    """The committed DRAM traffic counts only for the exact source file it was
    captured from (a hash of the file sits beside the figure)."""
    import hashlib
    import bench
    src = tmp_path / "paper_2301_01356_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "k.cu").write_text("kernel source\n")
    sha = hashlib.sha1(b"kernel source\n").hexdigest()[:12]
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.txt").write_text(
        f"kernel=k_x workload=w bytes_per_launch=123456 file=k.cu sha={sha} source=test\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_traffic("k_x", "w") == 123456
    assert bench.load_traffic("k_x", "other") is None
    (src / "k.cu").write_text("kernel source, edited\n")
    assert bench.load_traffic("k_x", "w") is None


def test_committed_traffic_matches_the_current_source():
    """profiles/traffic.txt carries a figure for the bench's dominant kernel; it is
    reported while it still matches the committed source (skipped, with the reason,
    after a kernel change that awaits a new capture)."""
    import bench
    lines = [ln for ln in open(os.path.join(ROOT, "profiles", "traffic.txt")) if ln.strip()]
    assert lines
    kv = dict(x.split("=", 1) for x in lines[0].split() if "=" in x)
    assert {"kernel", "workload", "bytes_per_launch", "file", "sha"} <= set(kv)
    got = bench.load_traffic(kv["kernel"], kv["workload"])
    if got is None:
        pytest.skip(f"traffic.txt predates the current {kv['file']}: the kernel needs a new capture")
    assert got == int(float(kv["bytes_per_launch"]))


def test_tuned_config_and_overrides():
    """The tuned configuration of a workload comes from tuning.json; knobs given on
    the command line override it; --config default ignores the tuning."""
    import argparse
    import bench
    from paper_2301_01356_gb300 import batch as B
    tuned = B.load_tuning()["graphs"]["grid4096"]["config"]
    none = dict(ruler_stride=None, cc_sample=None, chase_chains=None, cc_local=None, lcc_sample=None,
                rank_variant=None, grid_ctas=None, cc_order=None, hub_deg=None, cc_ldd=None)
    a = argparse.Namespace(config="tuned", workload="grid4096", **none)
    cfg = bench.tuned_config(a)
    assert all(cfg[k] == v for k, v in tuned.items())
    a = argparse.Namespace(config="tuned", workload="grid4096", **dict(none, ruler_stride=8))
    assert bench.tuned_config(a)["ruler_stride"] == 8
    a = argparse.Namespace(config="default", workload="grid4096", **none)
    assert bench.tuned_config(a) == dict(ruler_stride=16, cc_sample=0, chase_chains=1, cc_local=0, lcc_sample=0,
                                         rank_variant=0, grid_ctas=0, cc_order=0, hub_deg=0, cc_ldd=0)


def test_bucket_summary_groups_chunks():
    """The batch line reports one entry per size bucket, with its chunk count."""
    import types
    import numpy as np
    import bench

    def chunk(bucket, sizes, cfg):
        sub = types.SimpleNamespace(sizes=lambda s=np.array(sizes): s)
        return types.SimpleNamespace(bucket=bucket, sub=sub, cfg=cfg)
    runner = types.SimpleNamespace(buckets=[chunk(0, [1000, 5000], {"a": 1}), chunk(2, [200000], {"b": 2}),
                                            chunk(2, [900000, 150000], {"b": 2})])
    out = bench.bucket_summary(runner)
    assert out == [{"n_range": [1000, 5000], "graphs": 2, "chunks": 1, "config": {"a": 1}},
                   {"n_range": [150000, 900000], "graphs": 3, "chunks": 2, "config": {"b": 2}}]
