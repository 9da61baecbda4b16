"""GPU parity at the full sizes of the benchmark workloads, element by element.

  - the power-law R-MAT scale-24 graph (260M edges, 64-bit offsets), in its tuned
    configuration and in the defaults;
  - all 4,096 graphs of the batched workload (n log-uniform on [10^3, 10^6], three
    families), solved by the bucketed batch runner exactly as the benchmark runs it;
  - a serving pool that holds a k-NN graph of 10^7 points next to the batch
    families, served by the continuous-batching loop.

Every output (edge_bcc, bcc_head, is_ap, is_bridge and the four counts) is
compared with the Hopcroft-Tarjan oracle. The oracle runs on host threads (the
ctypes call releases the GIL) while the GPU works, or over many graphs at once.
"""
import os
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from paper_2301_01356_gb300 import graphgen as gg

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

KEYS = ("edge_bcc", "bcc_head", "is_ap", "is_bridge", "n_bcc", "n_ap", "n_bridge", "n_cc")


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def assert_same(got, exp, what):
    for k in KEYS:
        assert np.array_equal(np.asarray(got[k]), np.asarray(exp[k])), f"{what}: {k} differs from the oracle"
    assert got.get("device_status", 0) == 0, f"{what}: device status {got['device_status']}"


class OracleThread(threading.Thread):
    """The oracle on one graph, on a host thread, while the caller uses the GPU."""

    def __init__(self, oracle, g):
        super().__init__(daemon=True)
        self.oracle, self.g, self.out, self.exc = oracle, g, None, None
        self.start()

    def run(self):
        try:
            self.out = self.oracle.solve(self.g.offsets, self.g.adj)
        except BaseException as e:   # re-raised in the test thread
            self.exc = e

    def result(self):
        self.join()
        if self.exc is not None:
            raise self.exc
        return self.out


def _tuned(name):
    from paper_2301_01356_gb300 import batch as B
    return dict(B.load_tuning().get("graphs", {}).get(name, {}).get("config", {}))


def test_rmat24_full_size_vs_oracle(torch_cuda, oracle):
    """C3 at full size: hubs of degree in the hundreds of thousands, 520M arcs behind
    64-bit offsets, 16.8M-position tours and RMQ arrays."""
    from paper_2301_01356_gb300 import fbcc
    g = gg.workload_rmat_24()
    ref = OracleThread(oracle, g)
    off = torch_cuda.from_numpy(g.offsets).cuda()
    adj = torch_cuda.from_numpy(g.adj).cuda()
    got = []
    for cfg in (_tuned("rmat24"), {}):
        s = fbcc.Solver(g.n, g.nnz, **cfg)
        got.append((cfg, s.solve(off, adj)))
        s.close()
    del off, adj
    exp = ref.result()
    assert exp["n_bcc"] > 1000 and exp["n_ap"] > 1000 and exp["n_bridge"] > 1000
    for cfg, r in got:
        assert_same(r, exp, f"rmat24 {cfg}")


def _bucket_host(b):
    """One bulk host copy of a chunk's outputs."""
    return {"edge_bcc": b.edge_bcc.cpu().numpy(), "bcc_head": b.bcc_head.cpu().numpy(),
            "is_ap": b.is_ap.cpu().numpy(), "is_bridge": b.is_bridge.cpu().numpy(),
            "stats": b.stats.cpu().numpy().reshape(b.sub.G, -1)}


def test_batch_4096_every_graph_vs_oracle(torch_cuda, oracle):
    """C4 at full size: every one of the 4,096 graphs, from the bucketed runner in the
    tuned per-bucket configurations, equals the oracle (and the generator's ground
    truth for the cycle chains)."""
    from paper_2301_01356_gb300 import batch as B
    bt = gg.workload_batch_4096()
    runner = B.BatchRunner(bt)
    runner.run()
    torch_cuda.cuda.synchronize()
    host = [_bucket_host(b) for b in runner.buckets]
    where = dict(runner.where)
    buckets = [(b.vb_h, b.ab_h) for b in runner.buckets]
    runner.close()

    def check(g):
        bi, j = where[g]
        h, (vb, ab) = host[bi], buckets[bi]
        v0, v1, a0, a1 = int(vb[j]), int(vb[j + 1]), int(ab[j]), int(ab[j + 1])
        st = h["stats"][j]
        nb = int(st[0])
        got = {"edge_bcc": h["edge_bcc"][a0:a1], "bcc_head": h["bcc_head"][v0:v0 + nb],
               "is_ap": h["is_ap"][v0:v1], "is_bridge": h["is_bridge"][a0:a1], "n_bcc": nb,
               "n_ap": int(st[1]), "n_bridge": int(st[2]), "n_cc": int(st[3]),
               "device_status": int(st[4] & 0xffffffff)}
        x = bt.graph(g)
        exp = oracle.solve(x.offsets, x.adj)
        assert_same(got, exp, f"batch graph {g} ({gg.Batch.FAMILIES[int(bt.family[g])]}, n={x.n})")
        if bt.truth_bcc[g] >= 0:
            assert exp["n_bcc"] == bt.truth_bcc[g] and exp["n_ap"] == bt.truth_ap[g]
        return x.m

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        edges = sum(ex.map(check, range(bt.G)))
    assert edges == bt.nnz_total // 2


def test_serving_pool_with_knn_1e7_vs_oracle(torch_cuda, oracle):
    """C5: a request pool with a k-NN graph of 10^7 points (k = 5, unit cube) beside
    the batch families; every served result equals the oracle."""
    from paper_2301_01356_gb300 import serving
    fam = gg.batch(6, 5, 1000, 1000000)
    graphs = [fam.graph(i) for i in range(fam.G)] + [gg.knn3(10_000_000, 5, 17), gg.knn3(200_000, 5, 18)]
    big = len(graphs) - 2
    refs = {big: OracleThread(oracle, graphs[big])}
    pool = serving.Pool(torch_cuda, graphs)
    srv = serving.Server(pool, streams=3, keep_outputs=True)
    arrivals = serving.poisson_arrivals(200.0, 0.5, 21)
    ids = np.random.default_rng(21).integers(0, len(graphs), size=arrivals.size)
    ids[:3] = big                                   # the 10^7 graph is requested, more than once
    ids[3:3 + len(graphs)] = np.arange(len(graphs))  # and every pool graph at least once
    rep = srv.run(arrivals, ids)
    srv.close()
    assert rep["requests"] == arrivals.size
    exp = {g: (refs[g].result() if g in refs else oracle.solve(graphs[g].offsets, graphs[g].adj))
           for g in sorted(set(int(i) for i in ids))}
    for r, out in srv.outputs.items():
        assert_same(out, exp[out["graph"]], f"request {r} (pool graph {out['graph']}, n={graphs[out['graph']].n})")
