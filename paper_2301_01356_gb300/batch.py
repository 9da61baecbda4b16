"""Batched solves: thousands of graphs of uneven sizes per launch.

The graphs of a packed :class:`graphgen.Batch` are grouped by size bucket. Each
bucket is re-packed contiguously, uploaded once, and solved by one
``fbcc_solve_batch`` call (every kernel launch covers all of the bucket's graphs).
Each bucket has its own workspace, its tuned configuration (ruler stride,
First-CC variant: see ``autotune``), its own stream and its own captured CUDA
graph, so the buckets' solves overlap on the device.

A bucket larger than ``MAX_CHUNK_ARCS`` arcs is split into chunks of consecutive
graphs, each solved like a bucket of its own (same configuration). A chunk's
copies in and out then overlap the other chunks' kernels, where one large bucket
would copy all of its input before its first kernel and all of its output after
its last.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import fbcc

# Size buckets by vertex count: [lo, hi).
BUCKETS = ((0, 10_000), (10_000, 100_000), (100_000, 1 << 62))
TUNING_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")
STATS_WORDS = 5      # one fbcc_stats is 40 bytes
MAX_CHUNK_ARCS = 1 << 26


def chunks(idx: np.ndarray, arcs: np.ndarray, cap: int) -> list:
    """Split the graph ids ``idx`` (in order) into runs whose arc counts add up to at
    most ``cap``; a graph with more than ``cap`` arcs forms a run of its own."""
    out, start, tot = [], 0, 0
    for k, g in enumerate(idx):
        a = int(arcs[g])
        if k > start and tot + a > cap:
            out.append(idx[start:k])
            start, tot = k, 0
        tot += a
    if len(idx) > start:
        out.append(idx[start:])
    return out


def load_tuning(path: str = TUNING_PATH) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def bucket_config(tuning: dict, lo: int, hi: int) -> dict:
    for b in tuning.get("buckets", []):
        if b["lo"] == lo and b["hi"] == hi:
            return dict(b["config"])
    return {}


class _Bucket:
    def __init__(self, torch, sub, idx, cfg, device):
        self.idx = idx
        self.sub = sub
        self.cfg = cfg
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
        self.vb_h, self.ab_h = sub.vtx_base, sub.arc_base
        self.vb, self.ab = dev(sub.vtx_base), dev(sub.arc_base)
        self.loff, self.ladj = dev(sub.local_off), dev(sub.local_adj)
        n, z = sub.n_total, sub.nnz_total
        self.ws = fbcc.fbcc_workspace_create(n, z)
        if cfg:
            fbcc.fbcc_workspace_configure(self.ws, **cfg)
        self.edge_bcc = torch.empty(max(z, 1), dtype=torch.int32, device=device)
        self.bcc_head = torch.empty(max(n, 1), dtype=torch.int32, device=device)
        self.is_ap = torch.empty(max(n, 1), dtype=torch.uint8, device=device)
        self.is_bridge = torch.empty(max(z, 1), dtype=torch.uint8, device=device)
        self.stats = torch.zeros(sub.G * STATS_WORDS, dtype=torch.int64, device=device)
        self.stream = torch.cuda.Stream(device=device)

    def launch(self):
        fbcc.fbcc_solve_batch(self.vb, self.ab, self.vb_h, self.ab_h, self.loff, self.ladj, self.edge_bcc,
                              self.bcc_head, self.is_ap, self.is_bridge, self.stats, self.ws, self.stream)

    def close(self):
        if self.ws:
            fbcc.fbcc_workspace_destroy(self.ws)
            self.ws = None


class BatchRunner:
    """All graphs of a batch, solved bucket by bucket (buckets overlap on streams)."""

    def __init__(self, batch, buckets=BUCKETS, tuning: dict | None = None, device="cuda", configs=None,
                 max_chunk_arcs: int = MAX_CHUNK_ARCS):
        import torch
        self.torch = torch
        self.batch = batch
        sizes = batch.sizes()
        arcs = np.diff(batch.arc_base)
        tuning = load_tuning() if tuning is None else tuning
        self.buckets = []          # one entry per chunk; .bucket is its size bucket
        for i, (lo, hi) in enumerate(buckets):
            idx = np.nonzero((sizes >= lo) & (sizes < hi))[0]
            if idx.size == 0:
                continue
            cfg = configs[i] if configs is not None else bucket_config(tuning, lo, hi)
            for part in chunks(idx, arcs, max_chunk_arcs):
                b = _Bucket(torch, batch.subset(part), part, cfg, device)
                b.bucket = i
                self.buckets.append(b)
        self.where = {}
        for bi, b in enumerate(self.buckets):
            for j, g in enumerate(b.idx):
                self.where[int(g)] = (bi, j)

    def launch(self):
        """Enqueue every bucket's solve on its own stream, after the current stream."""
        cur = self.torch.cuda.current_stream()
        for b in self.buckets:
            b.stream.wait_stream(cur)
            b.launch()

    def join(self):
        """Make the current stream wait for every bucket."""
        cur = self.torch.cuda.current_stream()
        for b in self.buckets:
            cur.wait_stream(b.stream)

    def run(self):
        self.launch()
        self.join()

    def stats(self) -> np.ndarray:
        """Per-graph stats in the batch's original order: rows n_bcc, n_ap, n_bridge, n_cc, status."""
        out = np.zeros((self.batch.G, STATS_WORDS), np.int64)
        for b in self.buckets:
            s = b.stats.cpu().numpy().reshape(b.sub.G, STATS_WORDS)
            out[b.idx] = s
        out[:, 4] &= 0xffffffff
        return out

    def result(self, g: int) -> dict:
        """Outputs of graph g (host copies)."""
        bi, j = self.where[int(g)]
        b = self.buckets[bi]
        v0, v1 = int(b.vb_h[j]), int(b.vb_h[j + 1])
        a0, a1 = int(b.ab_h[j]), int(b.ab_h[j + 1])
        st = b.stats[j * STATS_WORDS:(j + 1) * STATS_WORDS].cpu().numpy()
        nb = int(st[0])
        return {"edge_bcc": b.edge_bcc[a0:a1].cpu().numpy(), "bcc_head": b.bcc_head[v0:v0 + nb].cpu().numpy(),
                "is_ap": b.is_ap[v0:v1].cpu().numpy(), "is_bridge": b.is_bridge[a0:a1].cpu().numpy(),
                "n_bcc": nb, "n_ap": int(st[1]), "n_bridge": int(st[2]), "n_cc": int(st[3]),
                "device_status": int(st[4] & 0xffffffff)}

    def close(self):
        for b in self.buckets:
            b.close()
        self.buckets = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def per_graph_loop(batch, graphs=None, device="cuda", config=None):
    """The plain form, one fbcc_solve per graph (direct launches): the comparison point
    for the batched form. Returns the seconds all the solves took."""
    import time
    import torch
    graphs = range(batch.G) if graphs is None else graphs
    n_max = int(np.diff(batch.vtx_base).max())
    z_max = int(np.diff(batch.arc_base).max())
    s = fbcc.Solver(n_max, z_max, device=device, use_graph=-1, **(config or {}))
    offs, adjs = [], []
    for g in graphs:
        x = batch.graph(g)
        offs.append(torch.from_numpy(x.offsets).to(device))
        adjs.append(torch.from_numpy(x.adj).to(device))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for off, adj in zip(offs, adjs):
        fbcc.fbcc_solve(off, adj, off.numel() - 1, adj.numel() // 2, s.edge_bcc, s.bcc_head, s.is_ap,
                        s.is_bridge, s.ws, None, want_stats=False)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    s.close()
    return dt
