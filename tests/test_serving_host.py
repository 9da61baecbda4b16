"""Host logic of the serving loop and of the query server, with every device call
replaced by a fake: admission by HBM footprint within the per-batch caps, LRU
eviction of resident graphs (never one in flight) and of solved states, and the
accounting of solves that report a device status."""
import collections
import types

import numpy as np
import pytest
import torch

from paper_2301_01356_gb300 import fbcc, serving


def _pool(sizes, with_graphs=False):
    n = np.array([a for a, _ in sizes], np.int64)
    z = np.array([b for _, b in sizes], np.int64)
    graphs = adj = None
    if with_graphs:
        graphs = [types.SimpleNamespace(n=int(a), nnz=int(b), offsets=np.zeros(a + 1, np.int64)) for a, b in sizes]
        adj = [torch.zeros(max(int(b), 1), dtype=torch.int32) for _, b in sizes]
    return types.SimpleNamespace(n=n, nnz=z, graphs=graphs, adj=adj)


def _server(pool, budget, graphs=512, n=1 << 24, nnz=1 << 27):
    srv = object.__new__(serving.Server)      # no streams: only the host bookkeeping runs
    srv.pool, srv.budget = pool, budget
    srv.max_batch_graphs, srv.max_batch_n, srv.max_batch_nnz = graphs, n, nnz
    srv.store = collections.OrderedDict()
    srv.store_bytes = srv.used = 0
    srv.inflight, srv.free = [], []
    srv.keep_outputs, srv.outputs, srv.failed = False, {}, 0
    return srv


def _batch(requests, foot=0, si=0):
    b = serving._Batch()
    b.requests, b.foot, b.si, b.ws = requests, foot, si, None
    return b


def test_make_room_evicts_least_recently_used_graphs_not_in_flight():
    pool = _pool([(10, 40)] * 4)                      # 200 bytes of CSR each
    srv = _server(pool, budget=1000)
    for g in (0, 1, 2, 3):
        srv.store[g] = None
        srv.store_bytes += srv._csr_bytes(g)
    srv.inflight.append(_batch([(7, 0)]))             # graph 0 is in flight
    assert srv._make_room(200) is True                # 800 + 200 fit: nothing leaves
    assert list(srv.store) == [0, 1, 2, 3]
    assert srv._make_room(500) is True                # needs 300 more: 1 and 2 leave, 0 stays
    assert list(srv.store) == [0, 3] and srv.store_bytes == 400
    srv.inflight.append(_batch([(8, 3)]))
    assert srv._make_room(700) is False               # only graphs in flight are left
    assert list(srv.store) == [0, 3]


def test_form_takes_requests_in_order_within_caps_and_budget(monkeypatch):
    monkeypatch.setattr(serving, "batch_footprint", lambda n, z, G: n + z + G)
    pool = _pool([(100, 400), (50, 100), (500, 2000), (10, 20)])
    waiting = collections.deque([(0, 0), (1, 1), (2, 2), (3, 3)])
    # the per-batch graph cap
    batch, n, z, foot = _server(pool, 1 << 20, graphs=2)._form(waiting)
    assert [g for _, g in batch] == [0, 1] and (n, z) == (150, 500) and foot == 150 + 500 + 2
    # the vertex cap stops before graph 2; the first request always goes in
    batch, n, z, _ = _server(pool, 1 << 20, n=400)._form(waiting)
    assert [g for _, g in batch] == [0, 1]
    batch, _, _, _ = _server(pool, 1 << 20, n=10)._form(waiting)
    assert [g for _, g in batch] == [0]
    # the budget: footprint plus the CSR uploads of graphs not yet resident
    srv = _server(pool, budget=(100 + 400 + 1) + 2000)
    batch, _, _, _ = srv._form(waiting)
    assert [g for _, g in batch] == [0]               # graph 1 would exceed it
    assert srv._form(collections.deque([(5, 2)]))[0] == []    # the head waits for memory


def test_collect_counts_failed_solves_and_frees_the_slot(monkeypatch):
    monkeypatch.setattr(serving.fbcc, "fbcc_workspace_destroy", lambda ws: None)
    srv = _server(_pool([(10, 40)] * 5), budget=1 << 20)
    b = _batch([(0, 3), (1, 4), (2, 3)], foot=300, si=2)
    st = np.zeros(3 * serving.STATS_WORDS, np.int64)
    st[1 * serving.STATS_WORDS + 4] = serving.fbcc.FBCC_E_ITER_LIMIT | (7 << 32)   # status in the low word
    st[2 * serving.STATS_WORDS + 4] = 7 << 32                                      # the high word is not status
    b.h_stats = torch.from_numpy(st)
    srv.used = 300
    srv.inflight.append(b)
    complete = np.full(3, np.nan)
    srv._collect(b, 1.5, complete)
    assert srv.failed == 1
    assert np.all(complete == 1.5) and srv.free == [2] and srv.used == 0 and srv.inflight == []


class _FakeSolver:
    status = {}          # n -> device status its solve reports
    made = []

    def __init__(self, n, nnz, device=None, **config):
        self.n, self.closed = n, False
        _FakeSolver.made.append(self)

    def enqueue(self, off, adj):
        return types.SimpleNamespace(device_status=_FakeSolver.status.get(self.n, 0))

    def close(self):
        self.closed = True


def _query_server(monkeypatch, pool, budget):
    monkeypatch.setattr(serving.fbcc, "Solver", _FakeSolver)
    monkeypatch.setattr(serving.fbcc, "fbcc_workspace_bytes", lambda n, z: 0)
    _FakeSolver.status, _FakeSolver.made = {}, []
    qs = serving.QueryServer(pool, hbm_budget=budget, device="cpu")
    sync = types.SimpleNamespace(synchronize=lambda: None)
    qs.torch = types.SimpleNamespace(from_numpy=torch.from_numpy,
                                     cuda=types.SimpleNamespace(current_stream=lambda: sync))
    return qs


def test_query_server_keeps_states_lru_within_the_budget(monkeypatch):
    pool = _pool([(100, 400), (200, 800), (300, 1200)], with_graphs=True)
    qs = _query_server(monkeypatch, pool, budget=0)
    sizes = [qs.state_bytes(g) for g in range(3)]
    qs.budget = sizes[0] + sizes[1] + sizes[2] - 1        # any two fit, all three do not
    s0 = qs.solver(0)
    qs.solver(1)
    assert qs.solver(0) is s0 and qs.hits == 1             # a hit moves graph 0 to the back
    qs.solver(2)                                           # graph 1, the least recently used, leaves
    assert list(qs.state) == [0, 2] and qs.evictions == 1 and qs.solves == 3
    assert _FakeSolver.made[1].closed and not s0.closed
    assert qs.held == sizes[0] + sizes[2]
    qs.budget = sizes[1] - 1
    with pytest.raises(MemoryError):
        qs.solver(1)                                       # larger than the whole budget
    assert list(qs.state) == [0, 2]


def test_query_server_refuses_a_failed_solve(monkeypatch):
    pool = _pool([(100, 400), (200, 800)], with_graphs=True)
    qs = _query_server(monkeypatch, pool, budget=1 << 40)
    qs.solver(0)
    _FakeSolver.status = {200: fbcc.FBCC_E_ITER_LIMIT}
    with pytest.raises(fbcc.FbccError) as ex:
        qs.solver(1)
    assert ex.value.status == fbcc.FBCC_E_ITER_LIMIT
    assert list(qs.state) == [0] and qs.solves == 1 and _FakeSolver.made[-1].closed
    assert qs.held == qs.state_bytes(0)
