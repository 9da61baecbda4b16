"""The serving loop: requests arriving while others are on the GPU join later
batches; every request's result equals the graph solved alone (and the oracle)."""
import numpy as np
import pytest

from paper_2301_01356_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_serving_results_equal_alone(torch_cuda, oracle):
    from paper_2301_01356_gb300 import fbcc, serving
    graphs = [gg.uniform(3000, 8000, 1), gg.grid(60, 70, p=0.6, seed=2), gg.cycle_chain(5000, 9, 3, 400, 3),
              gg.knn3(8000, 5, 4), gg.path(700), gg.from_edges(5, [], []), gg.uniform(20000, 60000, 5),
              gg.grid(120, 90, p=0.7, seed=6)]
    pool = serving.Pool(torch_cuda, graphs)
    # small slots so that batches get cut and several are in flight
    srv = serving.Server(pool, streams=3, max_batch_n=40000, max_batch_nnz=150000, max_batch_graphs=16,
                         keep_outputs=True)
    arrivals = serving.poisson_arrivals(400.0, 1.0, 9)
    rng = np.random.default_rng(9)
    ids = rng.integers(0, len(graphs), size=arrivals.size)
    rep = srv.run(arrivals, ids)
    assert rep["requests"] == arrivals.size and rep["batches"] > 3 and rep["p99_ms"] >= rep["p50_ms"] > 0
    alone = fbcc.Solver(40000, 150000)
    exp = []
    for g in graphs:
        off = torch_cuda.from_numpy(g.offsets).cuda()
        adj = torch_cuda.from_numpy(g.adj).cuda()
        solo = alone.solve(off, adj)
        orc = oracle.solve(g.offsets, g.adj)
        for k in ("edge_bcc", "bcc_head", "is_ap", "is_bridge", "n_bcc", "n_ap", "n_bridge", "n_cc"):
            assert np.array_equal(np.asarray(solo[k]), np.asarray(orc[k]))
        exp.append(solo)
    for r in range(arrivals.size):
        got = srv.outputs[r]
        e = exp[got["graph"]]
        assert got["device_status"] == 0
        for k in ("edge_bcc", "bcc_head", "is_ap", "is_bridge", "n_bcc", "n_ap", "n_bridge", "n_cc"):
            assert np.array_equal(np.asarray(got[k]), np.asarray(e[k])), (r, k)
    alone.close()
    srv.close()


def test_serving_admission_by_footprint(torch_cuda, oracle):
    """A budget that holds one batch of the largest graph at a time: requests wait for
    memory, the in-flight footprint plus the resident graphs never exceed it, every
    result still equals the oracle, and the plain per-request loop serves the same
    requests."""
    from paper_2301_01356_gb300 import serving
    graphs = [gg.grid(150, 150, p=0.65, seed=1), gg.uniform(20000, 50000, 2), gg.cycle_chain(8000, 7, 3, 900, 3)]
    pool = serving.Pool(torch_cuda, graphs)
    big = max(serving.batch_footprint(g.n, g.nnz, 1) + (g.n + g.nnz) * 4 for g in graphs)
    budget = int(big * 1.6)
    srv = serving.Server(pool, streams=4, hbm_budget=budget, keep_outputs=True)
    arrivals = np.zeros(24)                    # all at once: admission decides
    ids = np.arange(24) % len(graphs)
    rep = srv.run(arrivals, ids)
    assert rep["peak_device_bytes"] <= budget
    assert rep["batches"] >= 3
    exp = [oracle.solve(g.offsets, g.adj) for g in graphs]
    for r in range(24):
        got = srv.outputs[r]
        for k in ("edge_bcc", "bcc_head", "is_ap", "is_bridge", "n_bcc", "n_ap", "n_bridge", "n_cc"):
            assert np.array_equal(np.asarray(got[k]), np.asarray(exp[got["graph"]][k])), (r, k)
    srv.close()
    loop = serving.per_request_loop(pool, ids)
    assert loop["requests"] == 24 and loop["graphs_per_s"] > 0
    with pytest.raises(ValueError):
        serving.Server(pool, hbm_budget=big // 4)


def test_queries_from_resident_state(torch_cuda, oracle):
    """Queries served from resident solved state (QueryServer): every answer equals the
    one derived from the oracle's labels; repeated graphs are answered without a new
    solve; a budget that holds two graphs' states evicts the least recently queried,
    and a graph solved again after eviction answers the same."""
    from paper_2301_01356_gb300 import serving
    from test_gpu_query import expected_pairs, vertex_bccs
    graphs = [gg.grid(80, 70, p=0.62, seed=4), gg.uniform(6000, 15000, 3), gg.rmat(12, 8, seed=2),
              gg.cycle_chain(5000, 10, 3, 300, 5)]
    pool = serving.Pool(torch_cuda, graphs)
    sets = []
    for g in graphs:
        e = oracle.solve(g.offsets, g.adj)
        sets.append(vertex_bccs(g.offsets, np.asarray(e["edge_bcc"])))
    budget = max(serving.QueryServer(pool).state_bytes(g) for g in range(len(graphs))) * 2 + 1
    qs = serving.QueryServer(pool, hbm_budget=budget)
    rng = np.random.default_rng(11)
    order = [0, 0, 1, 0, 2, 3, 1, 1, 0, 2, 3, 3]
    for g in order:
        n = graphs[g].n
        u = rng.integers(0, n, 500).astype(np.int32)
        v = rng.integers(0, n, 500).astype(np.int32)
        # half the pairs are the two ends of an edge, which always share a BCC
        a = rng.integers(0, graphs[g].nnz, 250)
        u[:250] = (np.searchsorted(graphs[g].offsets, a, side="right") - 1).astype(np.int32)
        v[:250] = graphs[g].adj[a]
        dev = lambda x: torch_cuda.from_numpy(x).cuda()
        got = qs.biconnected(g, dev(u), dev(v)).cpu().numpy()
        assert np.array_equal(got, expected_pairs(sets[g], u, v)), f"graph {g}"
        off, ids = qs.bccs_of(g, dev(np.arange(n, dtype=np.int32)))
        off, ids = off.cpu().numpy(), ids.cpu().numpy()
        for x in range(0, n, 97):
            assert np.array_equal(np.sort(ids[off[x]:off[x + 1]]), sets[g][x]), f"graph {g}: BCCs of {x}"
        assert qs.held <= budget
    assert qs.hits > 0 and qs.evictions > 0 and qs.solves > len(graphs)
    rep = qs.run(np.array([0, 1, 0, 1, 0], np.int64), pairs=1000, seed=3)
    assert rep["requests"] == 5 and rep["answered_from_resident_state"] >= 3
    qs.close()
