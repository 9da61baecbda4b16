"""Serving: continuous batching of biconnectivity requests on one GPU.

Requests (a graph each, from a pool in pinned host memory) arrive on a Poisson
clock. The server keeps several batches in flight, each on its own stream:

  - Resident graphs. A graph's CSR is uploaded to the device the first time it is
    requested and stays resident (charged to the HBM budget; the least recently
    used graphs not in flight are evicted when the budget needs the room), so a
    batch packs its requests' CSRs with device-to-device copies.
  - Admission by HBM footprint. A batch takes the waiting requests in arrival
    order while its footprint (the workspace of fbcc_batch_workspace_bytes for the
    batch's vertex, arc and graph counts, the packed CSR and the outputs) fits the
    budget next to the batches in flight and the resident graphs, and within the
    per-batch caps; a request that does not fit waits for memory to free up.
  - Intermediate arrays per batch. Each batch's workspace is carved, with
    fbcc_workspace_create_in, from a device tensor of exactly its footprint (the
    PyTorch caching allocator recycles the memory of finished batches, so the
    loop makes no cudaMalloc or cudaFree once warm), solved by one
    fbcc_solve_batch call, and its outputs copied to pinned host buffers.

A request is complete when its batch's copies have landed; latency = completion
minus arrival. The same requests can also be served one at a time with the plain
form (per_request_loop) for comparison.

Queries (QueryServer) are served from resident state: a graph's solved workspace
(labels, heads and ranks, section 3.4's representation) stays on the device after
its first query, so later "are u and v biconnected" and "BCCs of v" queries on it
need no new solve.
"""
from __future__ import annotations

import collections
import time

import numpy as np

from . import fbcc

STATS_WORDS = 5      # one fbcc_stats is 40 bytes


class Pool:
    """The graphs requests are drawn from, in pinned host memory."""

    def __init__(self, torch, graphs):
        self.graphs = graphs
        self.n = np.array([g.n for g in graphs], np.int64)
        self.nnz = np.array([g.nnz for g in graphs], np.int64)
        self.off = [torch.from_numpy(np.ascontiguousarray(g.offsets[:-1].astype(np.int32))).pin_memory()
                    for g in graphs]
        self.adj = [torch.from_numpy(np.ascontiguousarray(g.adj)).pin_memory() for g in graphs]


def batch_footprint(n: int, nnz: int, G: int) -> int:
    """Device bytes of one batch: workspace and batch staging, packed CSR, outputs,
    per-graph bases and stats."""
    return (fbcc.fbcc_batch_workspace_bytes(n, nnz, G) + 512 + n * 4 + nnz * 4 + n * 5 + nnz * 5
            + (G + 1) * 16 + G * 8 * STATS_WORDS)


class _Batch:
    pass


class Server:
    """The continuous-batching loop (see the module docstring)."""

    def __init__(self, pool: Pool, streams: int = 4, hbm_budget: int = 150 << 30, max_batch_graphs: int = 512,
                 max_batch_n: int = 1 << 24, max_batch_nnz: int = 1 << 27, device="cuda",
                 keep_outputs: bool = False, config: dict | None = None):
        import torch
        self.torch = torch
        self.pool = pool
        self.device = torch.device(device)
        self.budget = int(hbm_budget)
        self.max_batch_graphs, self.max_batch_n, self.max_batch_nnz = max_batch_graphs, max_batch_n, max_batch_nnz
        self.config = dict(config or {})
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(streams)]
        self.free = list(range(streams))
        self.pinned = [dict() for _ in range(streams)]   # per stream: reusable pinned output buffers
        self.store = collections.OrderedDict()           # graph id -> (offsets, adjacency, upload event)
        self.store_bytes = 0
        self.inflight = []
        self.used = 0                                    # device bytes of the batches in flight
        self.peak_bytes = 0
        self.keep_outputs = keep_outputs
        self.outputs = {}
        self.failed = 0                                  # requests whose solve reported a device status
        g_max = int(np.argmax(pool.nnz))
        if batch_footprint(int(pool.n[g_max]), int(pool.nnz[g_max]), 1) + self._csr_bytes(g_max) > self.budget:
            raise ValueError("the largest pool graph does not fit the HBM budget")

    # ---- resident graphs ----------------------------------------------------------
    def _csr_bytes(self, g: int) -> int:
        return int(self.pool.n[g] + self.pool.nnz[g]) * 4

    def _busy_graphs(self) -> set:
        return {g for b in self.inflight for _, g in b.requests}

    def _make_room(self, need: int) -> bool:
        """Evict least recently used resident graphs (not in flight) until `need` more
        bytes fit the budget."""
        busy = None
        while self.used + self.store_bytes + need > self.budget:
            busy = self._busy_graphs() if busy is None else busy
            victim = next((g for g in self.store if g not in busy), None)
            if victim is None:
                return False
            self.store.pop(victim)
            self.store_bytes -= self._csr_bytes(victim)
        return True

    def _resident(self, g: int, stream):
        """Graph g's device CSR, uploaded on `stream` the first time; a batch on another
        stream waits for that upload."""
        torch = self.torch
        if g in self.store:
            self.store.move_to_end(g)
            off, adj, ev = self.store[g]
            stream.wait_event(ev)
            return off, adj
        with torch.cuda.stream(stream):
            off = torch.empty(max(int(self.pool.n[g]), 1), dtype=torch.int32, device=self.device)
            adj = torch.empty(max(int(self.pool.nnz[g]), 1), dtype=torch.int32, device=self.device)
            off[:int(self.pool.n[g])].copy_(self.pool.off[g], non_blocking=True)
            adj[:int(self.pool.nnz[g])].copy_(self.pool.adj[g], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        self.store[g] = (off, adj, ev)
        self.store_bytes += self._csr_bytes(g)
        return off, adj

    # ---- one batch ----------------------------------------------------------------
    def _pinned(self, si: int, name: str, count: int, dtype):
        buf = self.pinned[si].get(name)
        if buf is None or buf.numel() < count:
            buf = self.torch.empty(max(count, 1, 0 if buf is None else 2 * buf.numel()), dtype=dtype).pin_memory()
            self.pinned[si][name] = buf
        return buf

    def _launch(self, si: int, batch, n: int, z: int, foot: int):
        torch = self.torch
        s = self.streams[si]
        G = len(batch)
        vb = np.zeros(G + 1, np.int64)
        ab = np.zeros(G + 1, np.int64)
        for j, (_, g) in enumerate(batch):
            vb[j + 1] = vb[j] + self.pool.n[g]
            ab[j + 1] = ab[j] + self.pool.nnz[g]
        b = _Batch()
        b.si, b.requests, b.vb, b.ab, b.foot = si, batch, vb, ab, foot
        i32, u8, i64 = torch.int32, torch.uint8, torch.int64
        with torch.cuda.stream(s):
            b.mem = torch.empty(fbcc.fbcc_batch_workspace_bytes(n, z, G) + 512, dtype=u8, device=self.device)
            aligned = (-b.mem.data_ptr()) % 256
            b.ws = fbcc.fbcc_workspace_create_in(b.mem[aligned:], n, z, G)
            fbcc.fbcc_workspace_configure(b.ws, use_graph=-1, **self.config)
            b.loff = torch.empty(max(n, 1), dtype=i32, device=self.device)
            b.ladj = torch.empty(max(z, 1), dtype=i32, device=self.device)
            for j, (_, g) in enumerate(batch):
                off, adj = self._resident(g, s)
                b.loff[vb[j]:vb[j + 1]].copy_(off[:vb[j + 1] - vb[j]], non_blocking=True)
                b.ladj[ab[j]:ab[j + 1]].copy_(adj[:ab[j + 1] - ab[j]], non_blocking=True)
            h_vb = self._pinned(si, "vb", G + 1, i64)
            h_ab = self._pinned(si, "ab", G + 1, i64)
            h_vb.numpy()[:G + 1] = vb
            h_ab.numpy()[:G + 1] = ab
            b.vbd = torch.empty(G + 1, dtype=i64, device=self.device)
            b.abd = torch.empty(G + 1, dtype=i64, device=self.device)
            b.vbd.copy_(h_vb[:G + 1], non_blocking=True)
            b.abd.copy_(h_ab[:G + 1], non_blocking=True)
            b.edge_bcc = torch.empty(max(z, 1), dtype=i32, device=self.device)
            b.bcc_head = torch.empty(max(n, 1), dtype=i32, device=self.device)
            b.is_ap = torch.empty(max(n, 1), dtype=u8, device=self.device)
            b.is_bridge = torch.empty(max(z, 1), dtype=u8, device=self.device)
            b.stats = torch.empty(G * STATS_WORDS, dtype=i64, device=self.device)
        fbcc.fbcc_solve_batch(b.vbd, b.abd, vb, ab, b.loff, b.ladj, b.edge_bcc, b.bcc_head, b.is_ap, b.is_bridge,
                              b.stats, b.ws, s)
        with torch.cuda.stream(s):
            b.h_stats = self._pinned(si, "stats", G * STATS_WORDS, i64)
            b.h_stats[:G * STATS_WORDS].copy_(b.stats, non_blocking=True)
            b.h_ap = self._pinned(si, "ap", n, u8)
            b.h_bh = self._pinned(si, "bh", n, i32)
            b.h_ap[:n].copy_(b.is_ap[:n], non_blocking=True)
            b.h_bh[:n].copy_(b.bcc_head[:n], non_blocking=True)
            b.h_eb = self._pinned(si, "eb", z, i32)
            b.h_br = self._pinned(si, "br", z, u8)
            if z:
                b.h_eb[:z].copy_(b.edge_bcc[:z], non_blocking=True)
                b.h_br[:z].copy_(b.is_bridge[:z], non_blocking=True)
            b.done = torch.cuda.Event()
            b.done.record(s)
        self.used += foot
        self.peak_bytes = max(self.peak_bytes, self.used + self.store_bytes)
        self.inflight.append(b)

    def _collect(self, b, now: float, complete: np.ndarray):
        st = b.h_stats.numpy()
        for j, (r, _) in enumerate(b.requests):
            complete[r] = now
            if int(st[j * STATS_WORDS + 4]) & 0xffffffff:
                self.failed += 1
        if self.keep_outputs:
            for j, (r, g) in enumerate(b.requests):
                s = st[j * STATS_WORDS:(j + 1) * STATS_WORDS]
                nb = int(s[0])
                v0, v1, a0, a1 = int(b.vb[j]), int(b.vb[j + 1]), int(b.ab[j]), int(b.ab[j + 1])
                self.outputs[r] = {
                    "graph": g,
                    "edge_bcc": b.h_eb.numpy()[a0:a1].copy(), "bcc_head": b.h_bh.numpy()[v0:v0 + nb].copy(),
                    "is_ap": b.h_ap.numpy()[v0:v1].copy(), "is_bridge": b.h_br.numpy()[a0:a1].copy(),
                    "n_bcc": nb, "n_ap": int(s[1]), "n_bridge": int(s[2]), "n_cc": int(s[3]),
                    "device_status": int(s[4] & 0xffffffff)}
        fbcc.fbcc_workspace_destroy(b.ws)
        self.used -= b.foot
        self.free.append(b.si)
        self.inflight.remove(b)   # its tensors return to the caching allocator

    def _form(self, waiting):
        """The next batch from the head of the queue, within the caps and the budget."""
        batch, n, z = [], 0, 0
        foot, new_csr, fresh = 0, 0, set()
        for r, g in waiting:
            if len(batch) >= self.max_batch_graphs:
                break
            n2, z2 = n + int(self.pool.n[g]), z + int(self.pool.nnz[g])
            if batch and (n2 > self.max_batch_n or z2 > self.max_batch_nnz):
                break
            f2 = batch_footprint(n2, z2, len(batch) + 1)
            c2 = new_csr + (self._csr_bytes(g) if g not in self.store and g not in fresh else 0)
            if not self._make_room(f2 + c2):
                break
            if g not in self.store:
                fresh.add(g)
            batch.append((r, g))
            n, z, foot, new_csr = n2, z2, f2, c2
        return batch, n, z, foot

    # ---- the loop -----------------------------------------------------------------
    def run(self, arrivals: np.ndarray, graph_ids: np.ndarray) -> dict:
        """Serve requests arriving at `arrivals` (seconds from the start, ascending)
        for pool graphs `graph_ids`; returns latency and throughput figures."""
        R = len(arrivals)
        f0 = self.failed
        complete = np.full(R, np.nan)
        waiting = collections.deque()
        nxt = 0
        depth, sizes = [], []
        t0 = time.perf_counter()
        while True:
            now = time.perf_counter() - t0
            while nxt < R and arrivals[nxt] <= now:
                waiting.append((nxt, int(graph_ids[nxt])))
                nxt += 1
            for b in list(self.inflight):
                if b.done.query():
                    self._collect(b, time.perf_counter() - t0, complete)
            while self.free and waiting:
                batch, n, z, foot = self._form(waiting)
                if not batch:
                    break          # the head request waits for memory
                for _ in batch:
                    waiting.popleft()
                sizes.append(len(batch))
                self._launch(self.free.pop(), batch, n, z, foot)
            depth.append(len(waiting))
            if nxt >= R and not waiting and not self.inflight:
                break
            if not waiting and nxt < R and not self.inflight:
                gap = arrivals[nxt] - (time.perf_counter() - t0)
                if gap > 0:
                    time.sleep(min(gap, 0.0005))
        wall = time.perf_counter() - t0
        lat = (complete - arrivals) * 1e3
        edges = float(self.pool.nnz[graph_ids].sum()) / 2
        return {
            "requests": R, "wall_s": wall, "offered_per_s": R / max(arrivals[-1], 1e-9) if R else 0.0,
            "completed_per_s": R / wall, "edges_per_s": edges / wall,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_batch": float(np.mean(sizes)) if sizes else 0.0, "batches": len(sizes),
            "max_queue": int(max(depth) if depth else 0), "streams": len(self.streams),
            "peak_device_bytes": self.peak_bytes, "resident_graphs": len(self.store),
            "resident_bytes": self.store_bytes, "budget_bytes": self.budget,
            "failed": self.failed - f0,
        }

    def close(self):
        self.torch.cuda.synchronize()
        for b in list(self.inflight):
            fbcc.fbcc_workspace_destroy(b.ws)
        self.inflight = []
        self.store.clear()


class QueryServer:
    """Biconnectivity queries (section 3.4: "are u and v biconnected", "the BCCs of
    v") answered from solved state kept on the device.

    A graph is solved on its first query into a workspace of its own; its labels,
    heads and ranks then answer every later query on it with the fbcc_query_* calls,
    without another solve. When the next graph's state would not fit the HBM budget,
    the states of the least recently queried graphs are released. Queries are
    enqueued on the current stream after the solve they read, in call order."""

    def __init__(self, pool: Pool, hbm_budget: int = 150 << 30, config: dict | None = None, device="cuda"):
        import torch
        self.torch, self.pool, self.budget, self.device = torch, pool, int(hbm_budget), device
        self.config = dict(config or {})
        self.state = collections.OrderedDict()   # graph id -> (Solver, offsets, adjacency, bytes)
        self.held = 0
        self.solves = self.hits = self.evictions = 0

    def state_bytes(self, g: int) -> int:
        """Device bytes of graph g's resident state: workspace, outputs and CSR."""
        n, z = int(self.pool.n[g]), int(self.pool.nnz[g])
        return fbcc.fbcc_workspace_bytes(n, z) + 9 * n + 5 * z + 8 * (n + 1) + 4 * z + 4096

    def solver(self, g: int):
        """Graph g's solved state, solving it (and releasing older states) when absent."""
        g = int(g)
        if g in self.state:
            self.state.move_to_end(g)
            self.hits += 1
            return self.state[g][0]
        need = self.state_bytes(g)
        if need > self.budget:
            raise MemoryError(f"graph {g} needs {need} bytes of state, over the budget of {self.budget}")
        while self.state and self.held + need > self.budget:
            _, (old, _, _, b) = self.state.popitem(last=False)
            old.close()
            self.held -= b
            self.evictions += 1
        torch = self.torch
        gr = self.pool.graphs[g]
        offs = gr.offsets.astype(np.int64 if gr.nnz >= (1 << 31) else np.int32)
        off = torch.from_numpy(offs).to(self.device, non_blocking=True)
        adj = self.pool.adj[g].to(self.device, non_blocking=True)
        s = fbcc.Solver(gr.n, gr.nnz, device=self.device, **self.config)
        st = s.enqueue(off, adj)
        torch.cuda.current_stream().synchronize()    # a failed solve must not answer queries
        if st.device_status:
            s.close()
            raise fbcc.FbccError(st.device_status, f"solve of graph {g}")
        self.state[g] = (s, off, adj, need)
        self.held += need
        self.solves += 1
        return s

    def biconnected(self, g: int, u, v):
        """Device int32 tensor: the BCC that u[i] and v[i] of graph g share, or -1."""
        return self.solver(g).biconnected(u, v)

    def bccs_of(self, g: int, v):
        """(offsets, ids) on the device: the BCCs of v[i] of graph g are ids[offsets[i]:offsets[i + 1]]."""
        return self.solver(g).bccs_of(v)

    def run(self, graph_ids: np.ndarray, pairs: int, seed: int = 0) -> dict:
        """One query request per entry of graph_ids, each `pairs` random vertex pairs of
        its graph, answered back to back with the answers copied to pinned host
        memory; the throughput, the share answered from resident state, and the
        per-request latency."""
        torch = self.torch
        rng = np.random.default_rng(seed)
        h_out = torch.empty(pairs, dtype=torch.int32).pin_memory()
        lat = []
        s0, h0 = self.solves, self.hits
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for g in graph_ids:
            n = int(self.pool.n[g])
            t1 = time.perf_counter()
            uv = torch.from_numpy(rng.integers(0, max(n, 1), size=(2, pairs), dtype=np.int32)).to(self.device)
            out = self.biconnected(int(g), uv[0], uv[1])
            h_out.copy_(out, non_blocking=True)
            torch.cuda.current_stream().synchronize()
            lat.append(time.perf_counter() - t1)
        wall = time.perf_counter() - t0
        lat = np.sort(np.array(lat)) * 1e3
        R = len(graph_ids)
        return {"requests": R, "pairs_per_request": pairs, "wall_s": wall, "requests_per_s": R / wall,
                "pairs_per_s": R * pairs / wall, "solves": self.solves - s0,
                "answered_from_resident_state": self.hits - h0,
                "p50_ms": float(lat[len(lat) // 2]), "p99_ms": float(lat[min(len(lat) - 1, int(0.99 * len(lat)))]),
                "resident_states": len(self.state), "resident_bytes": self.held, "evictions": self.evictions}

    def close(self):
        self.torch.cuda.synchronize()
        for s, _, _, _ in self.state.values():
            s.close()
        self.state.clear()
        self.held = 0


def per_request_loop(pool: Pool, graph_ids: np.ndarray, device="cuda") -> dict:
    """The plain form, one request at a time: fbcc_solve on the graph's resident CSR,
    the outputs copied to pinned host memory, and the next request after that."""
    import torch
    n_max, z_max = int(pool.n.max()), int(pool.nnz.max())
    s = fbcc.Solver(n_max, z_max, device=device, use_graph=-1)
    dev = {}
    for g in sorted(set(int(x) for x in graph_ids)):
        dev[g] = (torch.from_numpy(pool.graphs[g].offsets.astype(np.int32)).to(device), pool.adj[g].to(device))
    h_eb = torch.empty(z_max, dtype=torch.int32).pin_memory()
    h_br = torch.empty(z_max, dtype=torch.uint8).pin_memory()
    h_ap = torch.empty(n_max, dtype=torch.uint8).pin_memory()
    h_bh = torch.empty(n_max, dtype=torch.int32).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for g in graph_ids:
        off, adj = dev[int(g)]
        n, z = int(pool.n[g]), int(pool.nnz[g])
        st = s.enqueue(off, adj)
        h_eb[:z].copy_(s.edge_bcc[:z], non_blocking=True)
        h_br[:z].copy_(s.is_bridge[:z], non_blocking=True)
        h_ap[:n].copy_(s.is_ap[:n], non_blocking=True)
        h_bh[:n].copy_(s.bcc_head[:n], non_blocking=True)
        torch.cuda.current_stream().synchronize()
        if st.device_status:
            raise RuntimeError(f"device status {st.device_status}")
    wall = time.perf_counter() - t0
    s.close()
    R = len(graph_ids)
    return {"requests": R, "wall_s": wall, "graphs_per_s": R / wall,
            "edges_per_s": float(pool.nnz[graph_ids].sum()) / 2 / wall}


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
