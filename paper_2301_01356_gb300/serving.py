"""Serving: continuous batching of biconnectivity requests on one GPU.

Requests (a graph each, from a pool in pinned host memory) arrive on a Poisson
clock. The loop keeps several batch *slots* in flight, each with its own stream,
workspace and device buffers, so a batch copies in, solves and copies out while
others do the same. A free slot takes the waiting requests in arrival order, as
many as fit its vertex/arc capacity, packs them (one host-to-device copy per
array and request, straight from the pinned pool into the slot's packed CSR),
solves them with one ``fbcc_solve_batch`` call and copies the outputs back; a
request is complete when its slot's copies have landed. Admission is by HBM
footprint: the slots' device bytes, sized up front, stay within the budget, and a
batch never exceeds its slot's capacity. Latency = completion minus arrival.
"""
from __future__ import annotations

import collections
import time

import numpy as np

from . import fbcc

STATS_WORDS = 5


class Slot:
    """Device and pinned host buffers for one in-flight batch."""

    def __init__(self, torch, max_n: int, max_nnz: int, max_graphs: int, device):
        self.max_n, self.max_nnz, self.max_graphs = max_n, max_nnz, max_graphs
        self.stream = torch.cuda.Stream(device=device)
        self.ws = fbcc.fbcc_workspace_create(max_n, max_nnz)
        fbcc.fbcc_workspace_configure(self.ws, use_graph=-1)
        i32, u8, i64 = torch.int32, torch.uint8, torch.int64
        self.loff = torch.empty(max(max_n, 1), dtype=i32, device=device)
        self.ladj = torch.empty(max(max_nnz, 1), dtype=i32, device=device)
        self.vb = torch.empty(max_graphs + 1, dtype=i64, device=device)
        self.ab = torch.empty(max_graphs + 1, dtype=i64, device=device)
        self.edge_bcc = torch.empty(max(max_nnz, 1), dtype=i32, device=device)
        self.bcc_head = torch.empty(max(max_n, 1), dtype=i32, device=device)
        self.is_ap = torch.empty(max(max_n, 1), dtype=u8, device=device)
        self.is_bridge = torch.empty(max(max_nnz, 1), dtype=u8, device=device)
        self.stats = torch.zeros(max_graphs * STATS_WORDS, dtype=i64, device=device)
        pin = lambda n, dt: torch.empty(max(n, 1), dtype=dt).pin_memory()
        self.h_vb, self.h_ab = pin(max_graphs + 1, i64), pin(max_graphs + 1, i64)
        self.h_edge_bcc, self.h_bcc_head = pin(max_nnz, i32), pin(max_n, i32)
        self.h_is_ap, self.h_is_bridge = pin(max_n, u8), pin(max_nnz, u8)
        self.h_stats = pin(max_graphs * STATS_WORDS, i64)
        self.done = torch.cuda.Event()
        self.requests = []      # (request index, graph id)
        self.busy = False

    def device_bytes(self) -> int:
        return (fbcc.fbcc_batch_workspace_bytes(self.max_n, self.max_nnz, self.max_graphs)
                + self.max_n * (4 + 4 + 1) + self.max_nnz * (4 + 4 + 1) + self.max_graphs * (16 + 8 * STATS_WORDS))

    def close(self):
        if self.ws:
            fbcc.fbcc_workspace_destroy(self.ws)
            self.ws = None


class Pool:
    """The graphs requests are drawn from, in pinned host memory."""

    def __init__(self, torch, graphs):
        self.graphs = graphs
        self.n = np.array([g.n for g in graphs], np.int64)
        self.nnz = np.array([g.nnz for g in graphs], np.int64)
        self.off = [torch.from_numpy(np.ascontiguousarray(g.offsets[:-1].astype(np.int32))).pin_memory()
                    for g in graphs]
        self.adj = [torch.from_numpy(np.ascontiguousarray(g.adj)).pin_memory() for g in graphs]


class Server:
    """The continuous-batching loop (see the module docstring)."""

    def __init__(self, pool: Pool, slots: int = 4, max_n: int = 1 << 24, max_nnz: int = 1 << 27,
                 max_graphs: int = 512, hbm_budget: int = 150 << 30, device="cuda", keep_outputs: bool = False):
        import torch
        self.torch = torch
        self.pool = pool
        if int(pool.n.max()) > max_n or int(pool.nnz.max()) > max_nnz:
            raise ValueError("a pool graph exceeds the slot capacity")
        self.slots = []
        used = 0
        for _ in range(slots):
            s = Slot(torch, max_n, max_nnz, max_graphs, device)
            if used + s.device_bytes() > hbm_budget and self.slots:
                s.close()
                break
            used += s.device_bytes()
            self.slots.append(s)
        self.device_bytes = used
        self.keep_outputs = keep_outputs
        self.outputs = {}

    # ---- one batch -------------------------------------------------------------
    def _launch(self, slot: Slot, batch):
        torch = self.torch
        vb = slot.h_vb.numpy()
        ab = slot.h_ab.numpy()
        vb[0] = ab[0] = 0
        for j, (_, g) in enumerate(batch):
            vb[j + 1] = vb[j] + self.pool.n[g]
            ab[j + 1] = ab[j] + self.pool.nnz[g]
        G = len(batch)
        with torch.cuda.stream(slot.stream):
            for j, (_, g) in enumerate(batch):
                slot.loff[vb[j]:vb[j + 1]].copy_(self.pool.off[g], non_blocking=True)
                slot.ladj[ab[j]:ab[j + 1]].copy_(self.pool.adj[g], non_blocking=True)
            slot.vb[:G + 1].copy_(slot.h_vb[:G + 1], non_blocking=True)
            slot.ab[:G + 1].copy_(slot.h_ab[:G + 1], non_blocking=True)
        fbcc.fbcc_solve_batch(slot.vb[:G + 1], slot.ab[:G + 1], vb[:G + 1].copy(), ab[:G + 1].copy(), slot.loff,
                              slot.ladj, slot.edge_bcc, slot.bcc_head, slot.is_ap, slot.is_bridge, slot.stats,
                              slot.ws, slot.stream)
        n, z = int(vb[G]), int(ab[G])
        with torch.cuda.stream(slot.stream):
            slot.h_stats[:G * STATS_WORDS].copy_(slot.stats[:G * STATS_WORDS], non_blocking=True)
            slot.h_is_ap[:n].copy_(slot.is_ap[:n], non_blocking=True)
            slot.h_bcc_head[:n].copy_(slot.bcc_head[:n], non_blocking=True)
            if z:
                slot.h_edge_bcc[:z].copy_(slot.edge_bcc[:z], non_blocking=True)
                slot.h_is_bridge[:z].copy_(slot.is_bridge[:z], non_blocking=True)
            slot.done.record(slot.stream)
        slot.requests = batch
        slot.busy = True

    def _collect(self, slot: Slot, now: float, complete: np.ndarray):
        for j, (r, g) in enumerate(slot.requests):
            complete[r] = now
        if self.keep_outputs:
            vb, ab = slot.h_vb.numpy(), slot.h_ab.numpy()
            st = slot.h_stats.numpy()
            for j, (r, g) in enumerate(slot.requests):
                s = st[j * STATS_WORDS:(j + 1) * STATS_WORDS]
                nb = int(s[0])
                self.outputs[r] = {
                    "graph": g,
                    "edge_bcc": slot.h_edge_bcc.numpy()[ab[j]:ab[j + 1]].copy(),
                    "bcc_head": slot.h_bcc_head.numpy()[vb[j]:vb[j] + nb].copy(),
                    "is_ap": slot.h_is_ap.numpy()[vb[j]:vb[j + 1]].copy(),
                    "is_bridge": slot.h_is_bridge.numpy()[ab[j]:ab[j + 1]].copy(),
                    "n_bcc": nb, "n_ap": int(s[1]), "n_bridge": int(s[2]), "n_cc": int(s[3]),
                    "device_status": int(s[4] & 0xffffffff)}
        slot.requests = []
        slot.busy = False

    # ---- the loop -------------------------------------------------------------
    def run(self, arrivals: np.ndarray, graph_ids: np.ndarray) -> dict:
        """Serve requests arriving at `arrivals` (seconds from the start, ascending)
        for pool graphs `graph_ids`; returns latency and throughput figures."""
        R = len(arrivals)
        complete = np.full(R, np.nan)
        waiting = collections.deque()
        nxt = 0
        queue_depth = []
        batch_sizes = []
        t0 = time.perf_counter()
        while True:
            now = time.perf_counter() - t0
            while nxt < R and arrivals[nxt] <= now:
                waiting.append((nxt, int(graph_ids[nxt])))
                nxt += 1
            for slot in self.slots:
                if slot.busy and slot.done.query():
                    self._collect(slot, time.perf_counter() - t0, complete)
            for slot in self.slots:
                if slot.busy or not waiting:
                    continue
                batch, n, z = [], 0, 0
                while waiting and len(batch) < slot.max_graphs:
                    r, g = waiting[0]
                    if n + self.pool.n[g] > slot.max_n or z + self.pool.nnz[g] > slot.max_nnz:
                        break
                    waiting.popleft()
                    batch.append((r, g))
                    n += self.pool.n[g]
                    z += self.pool.nnz[g]
                batch_sizes.append(len(batch))
                self._launch(slot, batch)
            queue_depth.append(len(waiting))
            if nxt >= R and not waiting and not any(s.busy for s in self.slots):
                break
            if not waiting and nxt < R:
                gap = arrivals[nxt] - (time.perf_counter() - t0)
                if gap > 0:
                    time.sleep(min(gap, 0.0005))
        wall = time.perf_counter() - t0
        lat = (complete - arrivals) * 1e3
        edges = float(self.pool.nnz[graph_ids].sum()) / 2
        return {
            "requests": R, "wall_s": wall, "offered_per_s": R / max(arrivals[-1], 1e-9),
            "completed_per_s": R / wall, "edges_per_s": edges / wall,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_batch": float(np.mean(batch_sizes)) if batch_sizes else 0.0, "batches": len(batch_sizes),
            "max_queue": int(max(queue_depth) if queue_depth else 0), "slots": len(self.slots),
            "device_bytes": self.device_bytes,
        }

    def close(self):
        for s in self.slots:
            s.close()
        self.slots = []


def poisson_arrivals(rate: float, seconds: float, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, size=int(rate * seconds * 1.2) + 16)
    t = np.cumsum(gaps)
    return t[t < seconds]


def make_pool(size: int, seed: int, nmin_knn: int = 10_000, nmax_knn: int = 10_000_000):
    """The request pool: the config-4 families (n on [1e3, 1e6]) and k-NN graphs (k = 5,
    n log-uniform on [nmin_knn, nmax_knn]) in equal shares."""
    from . import graphgen as gg
    per = size // 4
    b = gg.batch(3 * per, seed, 1000, 1000000)
    graphs = [b.graph(i) for i in range(b.G)]
    rng = np.random.Generator(np.random.PCG64(seed))
    for i in range(size - 3 * per):
        n = int(round(np.exp(rng.uniform(np.log(nmin_knn), np.log(nmax_knn)))))
        graphs.append(gg.knn3(n, 5, seed * 7919 + i))
    return graphs
