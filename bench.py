#!/usr/bin/env python3
"""Benchmark: FAST-BCC biconnected components on one GB300 (or N replicas).

One step = one full solve (First-CC, rooting, tagging, Last-CC, heads and the
per-edge outputs) of the workload graph, already resident in HBM. The metric is
undirected edges per second. Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl fbcc|reference]

Workloads: rmat24 (default; the low-diameter power-law graph, R-MAT scale 24,
edge factor 16, the largest single graph), grid4096 (the large-diameter road-like
graph: 4096x4096 open grid, edges kept with p = 0.62, plus 0.1 % short-range
extra edges), uniform64k (the small launch-bound graph), batch (4,096 graphs per
step through the bucketed batched form), serve (the continuous-batching server
on a Poisson stream). `--impl reference` times the CPU Hopcroft-Tarjan oracle (the
only reference that exists for this method) on the same metric and workload.
The GPU path is replicated per rank (the problem does not shard): N ranks each
solve their own copy and the value is the whole job's edges per second.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2301_01356_gb300 import graphgen as gg  # noqa: E402

METRIC = "undirected edges/sec, full BCC on 1 GB300 (plain vs batched); p50/p99 ms"
UNIT = "undirected edges/s"

WORKLOADS = {
    "grid4096": (gg.workload_grid_4096, False,
                 "large-diameter road-like graph: 4096x4096 open grid, each edge kept with p=0.62, plus 0.1% "
                 "extra edges of Manhattan length 1..8, seed 2; int32 CSR"),
    "grid2896": (gg.workload_grid_2896, False,
                 "the grid4096 recipe on a 2896x2896 grid (profiler captures); int32 CSR"),
    "uniform64k": (gg.workload_uniform_64k, False,
                   "uniform random graph: n=65,536, m=196,608 distinct edges, seed 1; int32 CSR"),
    "rmat22": (gg.workload_rmat_22, True, "the rmat24 recipe at scale 22 (profiler captures); int64 offsets"),
    "rmat24": (gg.workload_rmat_24, True,
               "power-law R-MAT scale 24, edge factor 16, (a,b,c,d)=(0.57,0.19,0.19,0.05), symmetrised, seed 3; "
               "int64 offsets, int32 adjacency"),
}

L2_FLUSH_BYTES = 256 << 20   # larger than the 129 MB L2


# ---------------------------------------------------------------------------
# multi-process plumbing (replicas): plain torch.distributed, gloo on CPU tests
# ---------------------------------------------------------------------------

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, world: int) -> float:
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def whole_job_rate(units_per_rank: float, steps: int, world: int, max_seconds: float) -> float:
    """Units all ranks processed divided by the slowest rank's time."""
    return units_per_rank * steps * world / max_seconds


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({nm for r in rows for nm, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# roofline: algorithmic bytes per launch of each kernel
# ---------------------------------------------------------------------------

# Algorithm 1's steps as the profiled kernels run them: a phase starts at its first
# kernel and lasts until the next phase starts.
PHASES = ("first_cc", "rooting", "tagging", "last_cc", "outputs")
PHASE_START = {"k_cc_count": "rooting", "k_link": "rooting", "k_first_of": "tagging", "k_ext_compact": "last_cc",
               "k_tv_init": "last_cc", "k_ap_keys": "outputs"}


def phase_bytes(n: int, nnz: int, n_cc: int, off_bytes: int) -> dict:
    """Algorithmic bytes the method must move per phase of one solve: each array a
    phase needs counted once, gathers at element size, the offsets (B bytes each)
    and the adjacency (4 bytes per arc) once per arc pass. A = 2 (n - #CC) tree arcs.
      First-CC   B n + 4 nnz + 16 n     (adjacency, parent read/write, forest record)
      Rooting    48 A + 16 n            (per tree arc: build 16, link 8, rank 8, scan and
                                         scatter 16; first, last, parent, size)
      Tagging    B n + 4 nnz + 40 n     (w1/w2 write, RMQ build read, query reads and writes)
      Last-CC    B n + 4 nnz + 28 n     (five tags, union-find)
      Outputs    B n + 9 nnz + 12 n     (adjacency, edge_bcc and is_bridge written, per vertex)"""
    A, B = 2 * (n - n_cc), off_bytes
    return {"first_cc": B * n + 4 * nnz + 16 * n, "rooting": 48 * A + 16 * n,
            "tagging": B * n + 4 * nnz + 40 * n, "last_cc": B * n + 4 * nnz + 28 * n,
            "outputs": B * n + 9 * nnz + 12 * n}


def algorithmic_bytes(kernel: str, n: int, nnz: int, n_cc: int, off_bytes: int, stride: int = 0) -> int | None:
    """The share of its phase's algorithmic bytes (phase_bytes) that one launch of
    `kernel` moves: the arc pass of a phase takes the offsets, the adjacency and the
    per-arc outputs, the other kernels the per-vertex and per-tree-arc terms they
    read or write; kernels that only reshape data the method does not ask for take
    none. `stride` is unused (kept for callers)."""
    A, B = 2 * (n - n_cc), off_bytes
    arc_cc = B * n + 4 * nnz + 8 * n            # a First-CC arc pass: adjacency plus the forest record
    table = {
        # First-CC
        "k_cc_init": 4 * n, "k_uf_compress": 4 * n,
        "k_cc_hook": arc_cc, "k_cc_local": arc_cc, "k_cc_hook_rest": arc_cc, "k_cc_hook_cross": 0,
        "k_cc_sample": 0, "k_mark_big": 0, "k_cc_pick_big": 0, "k_cc_hook_chunks": 0,
        # (the LDD rounds spread the arc pass over up to 64 launches: its bytes stay with the phase)
        "k_ldd_init": 0, "k_ldd_fill": 0, "k_ldd_expand": 0, "k_ldd_chunks": 0, "k_ldd_unite": 0, "k_ldd_minroot": 0,
        "k_ldd_reroot": 0,
        # Rooting
        "k_cc_count": 0, "k_cc_place": 0, "k_permute_te": 0, "k_scan_i32": 0, "k_link": 8 * A, "k_hub_order": 0, "k_succ_rulers": 16 * A, "k_chase": 8 * A, "k_lvl_rulers": 0, "k_lvl_chase": 0,
        "k_top": 0, "k_lvl_expand": 0, "k_jump": 0, "k_comp_size": 0, "k_place_records": 8 * A, "k_preorder": 8 * A + 16 * n,
        # Tagging
        "k_first_of": 0, "k_w12": B * n + 4 * nnz + 8 * n, "k_w12_keep": B * n + 4 * nnz + 8 * n, "k_rmq_prefix": 8 * n, "k_rmq_level": 0,
        "k_rmq_query": 24 * n,
        # Last-CC
        "k_ext_compact": 0, "k_ext_halve": 0, "k_ext_finish": 0, "k_plain_label": 0,
        "k_last_cc_cross": B * n + 4 * nnz + 20 * n, "k_last_cc_cross_rest": B * n + 4 * nnz + 20 * n,
        "k_lcc_sample": 0, "k_last_cc_cross_chunks": 0, "k_pos_compress": 0, "k_pos_pick_big": 0,
        "k_final_label": 8 * n,
        # the Tarjan-Vishkin foil in place of Last-CC: its skeleton's pairs are
        # written and read once, and the union-find over n + nnz ids set up once
        "k_tv_init": 4 * (n + nnz), "k_tv_arcs": B * n + 4 * nnz + 8 * nnz, "k_tv_tree": 8 * n,
        "k_tv_unite": 8 * (nnz + n),
        # Outputs
        "k_ap_keys": 12 * n, "k_key_list": 0, "k_key_adj": 0, "k_key_scan": 0, "k_key_bits": 0, "k_scan_popc": 0, "k_rank": 0, "k_fo": 0,
        "k_edge_out": B * n + 9 * nnz, "k_edge_out_keep": B * n + 9 * nnz, "k_bcc_base": 0, "k_batch_stats": 0, "k_finish": 0,
    }
    return table.get(kernel)


def phases_of(rows) -> list:
    """The phase of every row of a profiled solve's [(kernel, ms)] launch list."""
    cur, out = PHASES[0], []
    for name, _ in rows:
        cur = PHASE_START.get(name, cur)
        out.append(cur)
    return out


def kernel_source_hash(path: str, kernel: str) -> str | None:
    """Hash of one kernel's definition (its template line, signature and body) in a
    CUDA source file, so that edits elsewhere in the file leave it unchanged."""
    try:
        src = open(path).read()
    except OSError:
        return None
    m = re.search(r"^(template <[^\n]*>\n)?__global__[^\n]*\b" + re.escape(kernel) + r"\(", src, re.M)
    end = src.find("\n}\n", m.start()) if m else -1
    if end < 0:
        return None
    return hashlib.sha1(src[m.start():end + 3].encode()).hexdigest()[:12]


def load_traffic(kernel: str, workload: str):
    """dram bytes per launch from the committed ncu summary, or None when absent
    or when the kernel's definition changed since the capture (with func=, the
    hash covers that kernel's source text; without, the whole file)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        kv = dict(x.split("=", 1) for x in line.split() if "=" in x)
        if kv.get("kernel") == kernel and kv.get("workload") == workload:
            src = os.path.join(ROOT, "paper_2301_01356_gb300", "csrc", kv.get("file", ""))
            if "func" in kv:
                now = kernel_source_hash(src, kv["func"])
            else:
                now = hashlib.sha1(open(src, "rb").read()).hexdigest()[:12] if os.path.exists(src) else None
            if now is None or now != kv.get("sha"):
                return None
            return int(float(kv["bytes_per_launch"]))
    return None


def measured_peak_gbs():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# the reference arm: the CPU oracle
# ---------------------------------------------------------------------------

def run_reference(args, world, rank):
    if rank != 0:
        return
    from oracle import ht
    if args.workload == "batch":
        bt = gg.batch(args.batch_graphs, 4, 1000, 1000000)
        # a bounded sample per step: the first 64 graphs of the batch
        sample = [bt.graph(i) for i in range(min(64, bt.G))]

        class _Sample:
            m = sum(x.m for x in sample)
            n = sum(x.n for x in sample)
        g = _Sample()
        desc = f"{bt.G} graphs of the config-4 recipe; each step solves the first {len(sample)}"
        solve = lambda: [ht.solve(x.offsets, x.adj) for x in sample]
    else:
        fn, _, desc = WORKLOADS[args.workload]
        g, sdesc = cpu_sample(args.workload, fn())
        if sdesc != f"the full {args.workload} graph":
            desc = f"{desc}; each step solves {sdesc}"
        solve = lambda: ht.solve(g.offsets, g.adj)
    ht.load()
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        solve()
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    mean = sum(times) / len(times)
    value = g.m / mean
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {desc}", "n": g.n, "m": g.m},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{desc} (single-threaded Hopcroft-Tarjan, one solve per step)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------

def tuned_config(args) -> dict:
    """The autotuner's choice for this workload (tuning.json), overridden by any knob
    given on the command line."""
    from paper_2301_01356_gb300 import batch as B
    cfg = dict(ruler_stride=16, cc_sample=0, chase_chains=1, cc_local=0, lcc_sample=0, rank_variant=0, grid_ctas=0,
               cc_order=0, hub_deg=0, cc_ldd=0)
    if args.config == "tuned":
        cfg.update(B.load_tuning().get("graphs", {}).get(args.workload, {}).get("config", {}))
    for k in ("ruler_stride", "cc_sample", "chase_chains", "cc_local", "lcc_sample", "rank_variant", "grid_ctas",
              "cc_order", "hub_deg", "cc_ldd"):
        v = getattr(args, k)
        if v is not None:
            cfg[k] = v
    return cfg


# The oracle's sample of a workload: the full graph where one single-threaded run
# takes seconds, else the same recipe at a smaller scale (the R-MAT rows: one
# oracle run on the full scale-24 graph takes minutes).
CPU_SAMPLE_SCALE = 19

# Solves in flight in the pipelined end-to-end measurement (one workspace and one
# stream each). With two, a workspace's next input copy waits for its own output
# copy and the kernels idle meanwhile; three keep them busy (grid4096: 5.66 ms per
# step with two, 4.47 ms with three; rmat24: 24.8 and 18.3 ms).
E2E_STREAMS = 3


def cpu_sample(workload: str, g):
    if workload in ("rmat22", "rmat24"):
        x = gg.rmat(CPU_SAMPLE_SCALE, 16, 0.57, 0.19, 0.19, 3)
        return x, (f"the {workload} recipe at scale {CPU_SAMPLE_SCALE} (n = {x.n:,}, m = {x.m:,}); "
                   f"the full graph takes minutes per oracle run")
    return g, f"the full {workload} graph"


def cpu_baseline(g, runs: int = 3):
    from oracle import ht
    ht.load()
    res, ts = None, []
    for _ in range(runs):
        t0 = time.perf_counter()
        res = ht.solve(g.offsets, g.adj)
        ts.append(time.perf_counter() - t0)
    return res, statistics.median(ts)


def roofline_line(kernels: dict, phase_ms: dict, n: int, nnz: int, n_cc: int, off_bytes: int,
                  ms_per_step: float, workload: str) -> dict:
    """The dominant kernel against the measured copy bandwidth (its algorithmic bytes
    per launch over its CUDA-event launch time), the whole solve (the phases' bytes
    over the timed step) and every phase (its bytes over its kernels' event times)."""
    dom = max(kernels, key=lambda k: kernels[k]["ms_per_step"])
    peak, peak_kind = measured_peak_gbs()
    ab = algorithmic_bytes(dom, n, nnz, n_cc, off_bytes)
    achieved = ab / (kernels[dom]["ms_per_launch"] / 1e3) / 1e9 if ab else None
    pb = phase_bytes(n, nnz, n_cc, off_bytes)
    solve_b = sum(pb.values())
    phases = {}
    for ph in PHASES:
        ms = phase_ms.get(ph, 0.0)
        gbs = pb[ph] / (ms / 1e3) / 1e9 if ms > 0 else None
        phases[ph] = {"ms": round(ms, 4), "bytes": pb[ph], "gbs": gbs, "frac": gbs / peak if gbs else None}
    solve_gbs = solve_b / (ms_per_step / 1e3) / 1e9
    return {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if achieved else None, "traffic": load_traffic(dom, workload),
            "algorithmic_bytes_per_launch": ab, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
            "ms_per_launch": kernels[dom]["ms_per_launch"],
            "solve_bytes": solve_b, "solve_gbs": solve_gbs, "solve_frac": solve_gbs / peak, "phases": phases}


def time_queries(torch, solver, off, adj, n: int, nnz: int, g, count: int) -> dict:
    """Biconnectivity queries on the solved workload (section 3.4's labels and heads):
    `count` vertex pairs (half the two ends of random edges, half random pairs) and
    the BCCs of `count` random vertices, timed with CUDA events after one warm-up
    call (which also builds the per-head index of the solve)."""
    from paper_2301_01356_gb300 import fbcc
    rng = np.random.default_rng(12)
    a = rng.integers(0, nnz, count // 2)
    src = (np.searchsorted(g.offsets, a, side="right") - 1).astype(np.int32)   # the arcs' sources
    u = np.concatenate([src, rng.integers(0, n, count - count // 2).astype(np.int32)])
    v = np.concatenate([g.adj[a], rng.integers(0, n, count - count // 2).astype(np.int32)])
    du, dv = torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda()
    nv = min(count, 2 * n)                       # a call lists the BCCs of at most 2 n vertices
    dw = du[:nv].contiguous()
    solver.enqueue(off, adj)
    out = torch.empty(count, dtype=torch.int32, device="cuda")
    offs = torch.empty(nv + 1, dtype=torch.int64, device="cuda")
    fbcc.fbcc_query_biconnected(solver.ws, du, dv, out)
    fbcc.fbcc_query_bcc_count(solver.ws, dw, offs)
    torch.cuda.synchronize()
    ids = torch.empty(max(int(offs[-1].item()), 1), dtype=torch.int32, device="cuda")
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record()
    fbcc.fbcc_query_biconnected(solver.ws, du, dv, out)
    e[1].record()
    fbcc.fbcc_query_bcc_count(solver.ws, dw, offs)
    fbcc.fbcc_query_bccs_of(solver.ws, dw, offs, ids)
    e[2].record()
    torch.cuda.synchronize()
    t_pair, t_list = e[0].elapsed_time(e[1]) / 1e3, e[1].elapsed_time(e[2]) / 1e3
    return {"pairs": count, "biconnected_pairs_per_s": count / t_pair,
            "pairs_sharing_a_bcc": int((out >= 0).sum().item()),
            "vertices": nv, "bccs_of_vertices_per_s": nv / t_list, "bccs_listed": int(offs[-1].item()),
            "api": "fbcc_query_biconnected; fbcc_query_bcc_count + fbcc_query_bccs_of (device arrays)"}


def time_tv_foil(torch, solver, off, adj, n: int, nnz: int, flush, reps: int = 5) -> dict:
    """The Tarjan-Vishkin foil on the same workload and workspace (the skeleton built
    explicitly in caller memory instead of Last-CC's implicit one): CUDA-event time
    per solve (L2 flushed between solves), its scratch bytes against the workspace's,
    and whether every output equals FAST-BCC's."""
    from paper_2301_01356_gb300 import fbcc
    solver.enqueue(off, adj)
    torch.cuda.synchronize()
    ref = (solver.edge_bcc[:nnz].clone(), solver.is_ap[:n].clone(), solver.is_bridge[:nnz].clone(),
           solver.bcc_head[:n].clone(), solver.stats.as_dict())
    scratch_bytes = fbcc.fbcc_tv_scratch_bytes(n, nnz)
    scratch = torch.empty(scratch_bytes, dtype=torch.uint8, device="cuda")
    m = nnz // 2
    tv = lambda: fbcc.fbcc_solve_tv(off, adj, n, m, solver.edge_bcc, solver.bcc_head, solver.is_ap,
                                     solver.is_bridge, scratch, solver.ws, None, solver.stats)
    tv()
    torch.cuda.synchronize()
    st = solver.stats.as_dict()
    nb = st["n_bcc"]
    same = (torch.equal(ref[0], solver.edge_bcc[:nnz]) and torch.equal(ref[1], solver.is_ap[:n])
            and torch.equal(ref[2], solver.is_bridge[:nnz]) and torch.equal(ref[3][:nb], solver.bcc_head[:nb])
            and all(st[k] == ref[4][k] for k in ("n_bcc", "n_ap", "n_bridge", "n_cc")))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in ev:
        flush.zero_()
        a.record()
        tv()
        b.record()
    torch.cuda.synchronize()
    ms = sorted(a.elapsed_time(b) for a, b in ev)[reps // 2]
    del scratch
    ws_bytes = fbcc.fbcc_workspace_bytes(solver.n_max, solver.nnz_max)
    return {"ms_per_solve": ms, "undirected_edges_per_s": m / (ms / 1e3), "scratch_bytes": scratch_bytes,
            "workspace_bytes": ws_bytes, "scratch_over_workspace": scratch_bytes / ws_bytes,
            "outputs_equal_fbcc": bool(same),
            "api": "fbcc_solve_tv (direct launches) on the same workspace, scratch in a caller tensor"}


def run_gpu(args, world, rank, local):
    import torch
    from paper_2301_01356_gb300 import fbcc

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (there is no CPU path)")
    torch.cuda.set_device(local)
    fn, off64, desc = WORKLOADS[args.workload]
    g = fn()
    n, nnz, m = g.n, g.nnz, g.m
    off_np = g.offsets.astype(np.int64 if off64 else np.int32)
    off = torch.from_numpy(off_np).cuda()
    adj = torch.from_numpy(g.adj).cuda()
    cfg = tuned_config(args)
    solver = fbcc.Solver(n, nnz, **cfg)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    # warm-up (also builds the captured graph)
    for _ in range(args.warmup):
        solver.enqueue(off, adj)
    torch.cuda.synchronize()
    st = solver.stats.as_dict()
    if st["device_status"] != 0:
        raise SystemExit(f"device status {st['device_status']} in warm-up")

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.zero_()                      # evict the previous step's data from L2
        ev[i][0].record(stream)
        solver.enqueue(off, adj)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    # keep the GPU busy a little longer so the clock sampler brackets the region
    t_end = time.time() + 0.3
    while time.time() < t_end:
        solver.enqueue(off, adj)
        torch.cuda.synchronize()
    clocks = sampler.stop()
    total_s = sum(step_ms) / 1e3
    max_s = max_over_ranks(total_s, world)
    value = whole_job_rate(m, args.steps, world, max_s)
    ms_sorted = sorted(step_ms)
    p50 = ms_sorted[len(ms_sorted) // 2]
    p99 = ms_sorted[min(len(ms_sorted) - 1, int(round(0.99 * (len(ms_sorted) - 1))))]

    # per-kernel times (profiled solves: an event after every kernel)
    solver.configure(profile=1, **cfg)
    prof = {}
    phase_ms = dict.fromkeys(PHASES, 0.0)
    launches_per_step = 0
    for _ in range(args.profile_steps):
        flush.zero_()
        solver.enqueue(off, adj)
        rows = fbcc.fbcc_profile(solver.ws)
        launches_per_step = len(rows)
        for (name, ms), ph in zip(rows, phases_of(rows)):
            tot, cnt = prof.get(name, (0.0, 0))
            prof[name] = (tot + ms, cnt + 1)
            phase_ms[ph] += ms / args.profile_steps
    torch.cuda.synchronize()
    solver.configure(**cfg)
    kernels = {k: {"ms_per_step": t / args.profile_steps, "launches_per_step": c // args.profile_steps,
                   "ms_per_launch": t / c} for k, (t, c) in prof.items()}
    roofline = roofline_line(kernels, phase_ms, n, nnz, st["n_cc"], off_np.itemsize, max_s * 1e3 / args.steps,
                             args.workload)

    queries = time_queries(torch, solver, off, adj, n, nnz, g, args.query_count)
    tv_foil = time_tv_foil(torch, solver, off, adj, n, nnz, flush) if n + nnz < 2**31 - 1 else None

    # end to end through the public host API: pinned host in, pinned host out
    pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
    h_off, h_adj = pin(off_np), pin(g.adj)
    h_eb = torch.empty(nnz, dtype=torch.int32).pin_memory().numpy()
    h_bh = torch.empty(n, dtype=torch.int32).pin_memory().numpy()
    h_ap = torch.empty(n, dtype=torch.uint8).pin_memory().numpy()
    h_br = torch.empty(nnz, dtype=torch.uint8).pin_memory().numpy()
    for _ in range(2):
        fbcc.fbcc_solve_host(h_off, h_adj, h_eb, h_bh, h_ap, h_br, solver.ws)
    e2e_ts = []
    barrier(world)
    for _ in range(args.steps):
        t0 = time.perf_counter()
        hs = fbcc.fbcc_solve_host(h_off, h_adj, h_eb, h_bh, h_ap, h_br, solver.ws)
        e2e_ts.append(time.perf_counter() - t0)
    e2e_sync_max = max_over_ranks(sum(e2e_ts), world)
    d2h_sync = h_eb.nbytes + h_br.nbytes + h_ap.nbytes + 4 * hs.n_bcc + ctypes.sizeof(fbcc.fbcc_stats)

    # the same, pipelined: E2E_STREAMS workspaces on as many streams, each step
    # copying its inputs in and its outputs out, so one step's copies run during
    # the others' kernels and the kernels of different steps fill each other's
    # gaps (fbcc_solve_host_async)
    extra = [fbcc.fbcc_workspace_create(n, nnz) for _ in range(E2E_STREAMS - 1)]
    for w in extra:
        fbcc.fbcc_workspace_configure(w, **cfg)
    outs = [(h_eb, h_bh, h_ap, h_br)] + [tuple(torch.empty(k, dtype=dt).pin_memory().numpy()
                                               for k, dt in ((nnz, torch.int32), (n, torch.int32),
                                                             (n, torch.uint8), (nnz, torch.uint8)))
                                         for _ in extra]
    wss = [solver.ws] + extra
    streams = [torch.cuda.Stream() for _ in wss]
    S = len(wss)
    for i in range(2 * S):
        fbcc.fbcc_solve_host_async(h_off, h_adj, *outs[i % S], wss[i % S], streams[i % S])
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for i in range(args.steps):
        # a workspace's previous step is done with its buffers before it is reused:
        # its stream orders them
        fbcc.fbcc_solve_host_async(h_off, h_adj, *outs[i % S], wss[i % S], streams[i % S])
    for q in streams:
        q.synchronize()
    e2e_max = max_over_ranks(time.perf_counter() - t0, world)
    same = all(all(np.array_equal(outs[0][j], o[j]) for j in (0, 2, 3)) and
               np.array_equal(outs[0][1][:hs.n_bcc], o[1][:hs.n_bcc]) for o in outs[1:])
    for w in extra:
        fbcc.fbcc_workspace_destroy(w)
    if not same:
        raise SystemExit("pipelined host solves disagree")
    h2d = h_off.nbytes + h_adj.nbytes
    d2h = h_eb.nbytes + h_br.nbytes + h_ap.nbytes + h_bh.nbytes

    # parity of the benchmarked configuration and the CPU baseline (one rank, N = 1 only)
    cpu = None
    parity = None
    if world == 1 and not args.no_cpu_baseline:
        sample, sdesc = cpu_sample(args.workload, g)
        exp, cpu_s = cpu_baseline(sample)
        if sample is g:
            got = {"edge_bcc": h_eb, "bcc_head": h_bh[:hs.n_bcc], "is_ap": h_ap, "is_bridge": h_br,
                   "n_bcc": hs.n_bcc, "n_ap": hs.n_ap, "n_bridge": hs.n_bridge, "n_cc": hs.n_cc}
        else:   # the sample solved on the GPU in the benchmarked configuration
            ss = fbcc.Solver(sample.n, sample.nnz, **cfg)
            got = ss.solve(torch.from_numpy(sample.offsets.astype(off_np.dtype)).cuda(),
                           torch.from_numpy(sample.adj).cuda())
            ss.close()
        parity = {"graph": sdesc, "equal": all(np.array_equal(np.asarray(got[k]), np.asarray(exp[k])) for k in
                                               ("edge_bcc", "bcc_head", "is_ap", "is_bridge", "n_bcc", "n_ap",
                                                "n_bridge", "n_cc"))}
        cpu = {"value": sample.m / cpu_s, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{sdesc}, median of 3 single-threaded Hopcroft-Tarjan runs ({cpu_s:.2f} s each)"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_s * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {desc}", "n": n, "m": m, "parallelism": f"replicas{world}",
                   "l2": "flushed between timed steps (256 MiB write)", "tuning": cfg,
                   "p50_ms": p50, "p99_ms": p99},
        "e2e": {"value": whole_job_rate(m, args.steps, world, e2e_max), "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_max * 1e3 / args.steps,
                "api": f"fbcc_solve_host_async, pinned host buffers, {E2E_STREAMS} workspaces on as many "
                       "streams (a step's copies overlap the other workspaces' kernels)",
                "sync": {"value": whole_job_rate(m, args.steps, world, e2e_sync_max), "unit": UNIT,
                         "ms_per_step": e2e_sync_max * 1e3 / args.steps, "d2h_bytes_per_step": d2h_sync,
                         "api": "fbcc_solve_host, one call at a time"}},
        "gpu_launches": launches_per_step * args.steps,
        "roofline": roofline,
        "queries": queries,
        "tv_foil": tv_foil,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "parity_vs_oracle": parity,
        "stats": {k: st[k] for k in ("n_bcc", "n_ap", "n_bridge", "n_cc")},
        "kernels": {k: round(v["ms_per_step"], 4) for k, v in sorted(kernels.items(), key=lambda kv: -kv[1]["ms_per_step"])},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    solver.close()


def run_single(args, rank, local):
    """One solve with direct launches (no graph replay, no timing loop): the
    command profilers wrap, so that every launch of one solve is captured once."""
    import torch
    from paper_2301_01356_gb300 import fbcc

    torch.cuda.set_device(local)
    fn, off64, desc = WORKLOADS[args.workload]
    g = fn()
    off = torch.from_numpy(g.offsets.astype(np.int64 if off64 else np.int32)).cuda()
    adj = torch.from_numpy(g.adj).cuda()
    cfg = dict(tuned_config(args), use_graph=-1, profile=1)
    solver = fbcc.Solver(g.n, g.nnz, **cfg)
    solver.enqueue(off, adj)
    torch.cuda.synchronize()
    rows = fbcc.fbcc_profile(solver.ws)
    st = solver.stats.as_dict()
    solver.close()
    if st["device_status"] != 0:
        raise SystemExit(f"device status {st['device_status']}")
    if rank == 0:
        print(json.dumps({"workload": args.workload, "n": g.n, "m": g.m, "tuning": tuned_config(args),
                          "launches": len(rows), "kernels": [name for name, _ in rows]}), flush=True)


def bucket_summary(runner) -> list:
    """Per size bucket: the vertex range of its graphs, their count, the number of
    chunks it was split into and its tuned configuration."""
    out = []
    for i in sorted({b.bucket for b in runner.buckets}):
        bs = [b for b in runner.buckets if b.bucket == i]
        sz = np.concatenate([b.sub.sizes() for b in bs])
        out.append({"n_range": [int(sz.min()), int(sz.max())], "graphs": int(sz.size), "chunks": len(bs),
                    "config": bs[0].cfg})
    return out


def run_batch(args, world, rank, local):
    """Config 4: thousands of graphs per launch vs a per-graph loop of the plain form."""
    import torch
    from paper_2301_01356_gb300 import batch as B, fbcc
    from oracle import ht

    torch.cuda.set_device(local)
    t0 = time.perf_counter()
    bt = gg.batch(args.batch_graphs, 4, 1000, 1000000)
    gen_s = time.perf_counter() - t0
    m_total = bt.nnz_total // 2
    runner = B.BatchRunner(bt)
    for _ in range(args.warmup):
        runner.run()
    torch.cuda.synchronize()
    st = runner.stats()
    if np.any(st[:, 4] != 0):
        raise SystemExit("device status set in the batched warm-up")
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    for a, b in ev:
        a.record()
        runner.run()
        b.record()
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    max_s = max_over_ranks(sum(step_ms) / 1e3, world)
    value = whole_job_rate(m_total, args.steps, world, max_s)
    ms_sorted = sorted(step_ms)

    # the plain form, graph by graph (same GPU, same graphs)
    B.per_graph_loop(bt, graphs=range(min(64, bt.G)))
    loop_s = B.per_graph_loop(bt)

    # one profiled solve of every chunk: its launch count, and the per-kernel times
    # of the largest chunk for the roofline
    big = max(runner.buckets, key=lambda b: b.sub.n_total)
    launches = 0
    for b in runner.buckets:
        fbcc.fbcc_workspace_configure(b.ws, profile=1, **b.cfg)
        b.launch()
        r = fbcc.fbcc_profile(b.ws)
        torch.cuda.synchronize()
        fbcc.fbcc_workspace_configure(b.ws, **b.cfg)
        launches += len(r)
        if b is big:
            rows = r
    prof = {}
    for name, ms in rows:
        t, c = prof.get(name, (0.0, 0))
        prof[name] = (t + ms, c + 1)
    phase_ms = dict.fromkeys(PHASES, 0.0)
    for (name, ms), ph in zip(rows, phases_of(rows)):
        phase_ms[ph] += ms
    n_cc_big = int(runner.stats()[big.idx, 3].sum())
    kernels = {k: {"ms_per_step": t, "ms_per_launch": t / c} for k, (t, c) in prof.items()}
    roofline = roofline_line(kernels, phase_ms, big.sub.n_total, big.sub.nnz_total, n_cc_big, 8,
                             sum(phase_ms.values()), "batch")
    roofline["traffic"] = None
    roofline["chunk_vertices"] = big.sub.n_total
    roofline["solve_basis"] = "the largest chunk's profiled solve (its kernels' event times)"

    # end to end: packed inputs from pinned host memory, outputs back to pinned host memory
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_in = [(pin(b.sub.local_off), pin(b.sub.local_adj)) for b in runner.buckets]
    h_out = [(torch.empty(b.edge_bcc.shape, dtype=torch.int32).pin_memory(),
              torch.empty(b.is_bridge.shape, dtype=torch.uint8).pin_memory(),
              torch.empty(b.is_ap.shape, dtype=torch.uint8).pin_memory(),
              torch.empty(b.stats.shape, dtype=torch.int64).pin_memory(),
              torch.empty(b.bcc_head.shape, dtype=torch.int32).pin_memory()) for b in runner.buckets]
    e2e_ts = []
    for _ in range(max(2, args.steps // 4)):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        # each chunk copies in, solves and copies out on its own stream, so one
        # chunk's copies overlap the others' kernels
        cur = torch.cuda.current_stream()
        for b, (lo, la), (eb, br, ap, sb, bh) in zip(runner.buckets, h_in, h_out):
            b.stream.wait_stream(cur)
            with torch.cuda.stream(b.stream):
                b.loff.copy_(lo, non_blocking=True)
                b.ladj.copy_(la, non_blocking=True)
            b.launch()
            with torch.cuda.stream(b.stream):
                eb.copy_(b.edge_bcc, non_blocking=True)
                br.copy_(b.is_bridge, non_blocking=True)
                ap.copy_(b.is_ap, non_blocking=True)
                sb.copy_(b.stats, non_blocking=True)
                bh.copy_(b.bcc_head, non_blocking=True)   # all n entries: n_bcc is not known yet
        torch.cuda.synchronize()
        e2e_ts.append(time.perf_counter() - t1)
    e2e_s = statistics.median(e2e_ts)
    h2d = sum(lo.numel() * 4 + la.numel() * 4 for lo, la in h_in)
    d2h = sum(eb.numel() * 4 + br.numel() + ap.numel() + sb.numel() * 8 + bh.numel() * 4
              for eb, br, ap, sb, bh in h_out)

    parity = cpu = None   # oracle parity and the CPU baseline: one rank, N = 1 only
    if world == 1 and not args.no_cpu_baseline:
        rng = np.random.default_rng(0)
        sample = rng.choice(bt.G, size=min(48, bt.G), replace=False)
        ok = True
        for g in sample:
            x = bt.graph(int(g))
            e = ht.solve(x.offsets, x.adj)
            r = runner.result(int(g))
            ok &= all(np.array_equal(np.asarray(r[k]), np.asarray(e[k])) for k in
                      ("edge_bcc", "bcc_head", "is_ap", "is_bridge", "n_bcc", "n_ap", "n_bridge", "n_cc"))
        parity = {"graphs_checked": int(sample.size), "all_equal": bool(ok)}
        t1 = time.perf_counter()
        done_m = done_g = 0
        for g in range(bt.G):
            x = bt.graph(g)
            ht.solve(x.offsets, x.adj)
            done_m += x.m
            done_g += 1
            if time.perf_counter() - t1 > args.cpu_seconds:
                break
        cs = time.perf_counter() - t1
        cpu = {"value": done_m / cs, "unit": UNIT, "cores": 1, "kind": "oracle", "graphs_per_s": done_g / cs,
               "sample": f"the first {done_g} graphs of the batch, single-threaded Hopcroft-Tarjan"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_s * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": f"batch{bt.G}: {bt.G} graphs, n log-uniform on [1e3, 1e6], uniform (degree 4-12) / "
                               "thinned grid (p 0.55-0.75) / cycle chain families round-robin, seed 4",
                   "graphs": bt.G, "n_total": bt.n_total, "m_total": m_total, "parallelism": f"replicas{world}",
                   "l2": "inputs (packed CSR, %.1f GB) larger than L2" % ((bt.n_total + bt.nnz_total) * 4 / 1e9),
                   "buckets": bucket_summary(runner),
                   "p50_ms": ms_sorted[len(ms_sorted) // 2], "p99_ms": ms_sorted[-1], "generate_s": round(gen_s, 1)},
        "graphs_per_s": whole_job_rate(bt.G, args.steps, world, max_s),
        "per_graph_loop": {"graphs_per_s": bt.G / loop_s, "value": m_total / loop_s, "unit": UNIT,
                           "seconds": loop_s, "api": "fbcc_solve per graph, direct launches"},
        "e2e": {"value": m_total / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_s * 1e3, "api": "per chunk on its own stream: pinned host copies in, "
                                                   "fbcc_solve_batch, copies out (chunks overlap)"},
        "gpu_launches": launches * args.steps,
        "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks, "parity_vs_oracle": parity,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    runner.close()


def run_serve(args, world, rank, local):
    """Config 5: Poisson arrivals, continuous batching, p50/p99 latency; then the
    same kind of requests all at once (the server's saturation throughput) and one
    at a time through the plain form (the per-request loop it must beat)."""
    import torch
    from paper_2301_01356_gb300 import fbcc, serving

    torch.cuda.set_device(local)
    t0 = time.perf_counter()
    graphs = serving.make_pool(args.pool, 5, nmax_knn=args.knn_max)
    gen_s = time.perf_counter() - t0
    pool = serving.Pool(torch, graphs)
    srv = serving.Server(pool, streams=args.streams, hbm_budget=150 << 30)
    arrivals = serving.poisson_arrivals(args.rate, args.serve_seconds, 5)
    ids = np.random.default_rng(5).integers(0, len(graphs), size=arrivals.size)
    # warm-up: every pool graph once (their CSRs become resident) and a short burst
    srv.run(np.zeros(len(graphs)), np.arange(len(graphs)))
    wa = serving.poisson_arrivals(args.rate, 1.0, 6)
    srv.run(wa, np.random.default_rng(6).integers(0, len(graphs), size=wa.size))
    sampler = ClockSampler(local)
    sampler.start()
    rep = srv.run(arrivals, ids)
    clocks = sampler.stop()
    # saturation: the first requests of the stream all at once
    k = min(arrivals.size, args.saturation_requests)
    sat = srv.run(np.zeros(k), ids[:k])
    srv.close()
    loop = serving.per_request_loop(pool, ids[:min(k, args.loop_requests)])
    # each pool graph alone (plain form) vs in the mix: a verification run keeping outputs
    check = None
    if rank == 0:
        vsrv = serving.Server(pool, streams=args.streams, keep_outputs=True)
        va = serving.poisson_arrivals(args.rate, min(1.0, args.serve_seconds), 7)
        vids = np.random.default_rng(7).integers(0, len(graphs), size=va.size)
        vsrv.run(va, vids)
        alone = fbcc.Solver(int(pool.n.max()), int(pool.nnz.max()))
        solo = {}
        ok = True
        for r, out in vsrv.outputs.items():
            g = out["graph"]
            if g not in solo:
                x = graphs[g]
                solo[g] = alone.solve(torch.from_numpy(x.offsets).cuda(), torch.from_numpy(x.adj).cuda())
            ok &= all(np.array_equal(np.asarray(out[k2]), np.asarray(solo[g][k2])) for k2 in
                      ("edge_bcc", "bcc_head", "is_ap", "is_bridge", "n_bcc", "n_ap", "n_bridge", "n_cc"))
        alone.close()
        vsrv.close()
        check = {"requests": len(vsrv.outputs), "graphs": len(solo), "equal_to_alone": bool(ok)}
    # queries from resident state (section 3.4): query requests on pool graphs, each
    # graph solved on its first query and answered from its resident state after
    qs = serving.QueryServer(pool, hbm_budget=150 << 30)
    qids = np.random.default_rng(5).integers(0, len(graphs), size=args.query_requests)
    qrep = qs.run(qids, pairs=4096, seed=5)
    qs.close()
    qrep["api"] = "serving.QueryServer: fbcc_query_biconnected on each graph's resident solved workspace"
    line = {
        "metric": METRIC, "value": rep["edges_per_s"], "unit": UNIT, "n_gpus": world, "steps": rep["requests"],
        "warmup": 1, "ms_per_step": rep["p50_ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": f"serve: Poisson {args.rate:g} req/s for {args.serve_seconds:g} s over a pool of "
                               f"{len(graphs)} graphs (config-4 families on [1e3, 1e6] and k-NN k=5 on "
                               f"[1e4, {args.knn_max:.0e}]), continuous batching on {args.streams} streams, "
                               "admission by HBM footprint within 150 GB, resident CSRs",
                   "pool_generate_s": round(gen_s, 1)},
        "serving": rep, "p50_ms": rep["p50_ms"], "p99_ms": rep["p99_ms"],
        "saturation": {"requests": sat["requests"], "graphs_per_s": sat["completed_per_s"],
                       "edges_per_s": sat["edges_per_s"], "mean_batch": sat["mean_batch"]},
        "per_request_loop": {"requests": loop["requests"], "graphs_per_s": loop["graphs_per_s"],
                             "edges_per_s": loop["edges_per_s"],
                             "api": "fbcc_solve per request on its resident CSR, outputs to pinned host memory"},
        "serving_vs_loop_graphs_per_s": sat["completed_per_s"] / loop["graphs_per_s"],
        "mix_vs_alone": check, "queries": qrep, "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="rmat24", choices=sorted(WORKLOADS) + ["batch", "serve"])
    ap.add_argument("--batch-graphs", type=int, default=4096, help="graphs in --workload batch")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="oracle time budget of the batch baseline")
    ap.add_argument("--rate", type=float, default=2000.0, help="serve: Poisson arrival rate (requests/s)")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="serve: length of the arrival stream")
    ap.add_argument("--pool", type=int, default=128, help="serve: graphs in the request pool")
    ap.add_argument("--knn-max", type=float, default=1e7, help="serve: largest k-NN graph in the pool")
    ap.add_argument("--streams", type=int, default=4, help="serve: batches in flight (one stream each)")
    ap.add_argument("--saturation-requests", type=int, default=4000,
                    help="serve: requests of the all-at-once saturation run")
    ap.add_argument("--loop-requests", type=int, default=1000, help="serve: requests of the per-request loop")
    ap.add_argument("--query-requests", type=int, default=2000,
                    help="serve: query requests (4096 vertex pairs each) answered from resident state")
    ap.add_argument("--impl", default="fbcc", choices=("fbcc", "reference"))
    ap.add_argument("--config", default="tuned", choices=("tuned", "default"),
                    help="start from the autotuner's table (paper_2301_01356_gb300/tuning.json) or the defaults")
    ap.add_argument("--ruler-stride", type=int, default=None)
    ap.add_argument("--cc-sample", type=int, default=None, help="First-CC: neighbours hooked per vertex first")
    ap.add_argument("--chase-chains", type=int, default=None, help="list ranking: walks per thread (1, 2, 4)")
    ap.add_argument("--cc-local", type=int, default=None, help="First-CC: shared-memory range in vertices (0 = off)")
    ap.add_argument("--lcc-sample", type=int, default=None, help="Last-CC: cross edges sampled per vertex (0 = off)")
    ap.add_argument("--rank-variant", type=int, default=None, help="list ranking: 0 sampled levels, 1 pointer jumping")
    ap.add_argument("--grid-ctas", type=int, default=None, help="CTAs of the persistent grid (0 = 8 per SM)")
    ap.add_argument("--cc-order", type=int, default=None, help="rooting: forest renumbered by component (1 = on)")
    ap.add_argument("--hub-deg", type=int, default=None, help="hub threshold in arcs (0 = 256, -1 = no hubs)")
    ap.add_argument("--cc-ldd", type=int, default=None, help="First-CC by LDD + union-find: 1/beta (0 = off)")
    ap.add_argument("--profile-steps", type=int, default=3)
    ap.add_argument("--query-count", type=int, default=1 << 24, help="queries timed after the solves")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--single-solve", action="store_true",
                    help="run one solve with direct launches and exit (for profilers; no timing)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    try:
        if args.impl == "reference":
            run_reference(args, world, rank)
        elif args.workload == "batch":
            run_batch(args, world, rank, local)
        elif args.workload == "serve":
            run_serve(args, world, rank, local)
        elif args.single_solve:
            run_single(args, rank, local)
        else:
            run_gpu(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
