"""Biconnectivity queries (fbcc_query_*) against answers derived from the oracle.

A vertex lies in BCC k iff an edge of BCC k is incident to it, so the oracle's
per-arc labels give every vertex's set of BCCs; two vertices are biconnected iff
those sets meet (in one BCC at most, since two BCCs share at most one vertex).
"""
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


def vertex_bccs(offsets, edge_bcc):
    """Sorted BCC indices of every vertex, from the per-arc labels."""
    n = offsets.size - 1
    return [np.unique(edge_bcc[offsets[v]:offsets[v + 1]]) for v in range(n)]


def expected_pairs(sets, u, v):
    out = np.full(u.size, -1, np.int32)
    for i, (a, b) in enumerate(zip(u, v)):
        if a != b:
            c = np.intersect1d(sets[a], sets[b], assume_unique=True)
            assert c.size <= 1
            if c.size:
                out[i] = c[0]
    return out


def check_queries(torch, solver, g, sets, u, v, base=0, what=""):
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()
    got = solver.biconnected(dev(u + base), dev(v + base)).cpu().numpy()
    assert np.array_equal(got, expected_pairs(sets, u, v)), f"{what}: biconnected"
    verts = np.arange(g.n, dtype=np.int32)
    off, ids = solver.bccs_of(dev(verts + base))
    off, ids = off.cpu().numpy(), ids.cpu().numpy()
    assert off[0] == 0 and off[-1] == sum(s.size for s in sets), f"{what}: total count"
    for x in range(g.n):
        assert np.array_equal(np.sort(ids[off[x]:off[x + 1]]), sets[x]), f"{what}: BCCs of {x}"


def graphs():
    return [gg.cycle(7), gg.path(9), gg.star(6), gg.complete(6), gg.cycles_chain_exact([3, 4, 5], 2),
            gg.from_edges(5, [], []), gg.grid(40, 35, p=0.62, extra_frac=0.001, seed=3),
            gg.uniform(3000, 7000, 2), gg.rmat(13, 8, seed=5), gg.cycle_chain(4000, 12, 3, 300, 7),
            gg.knn3(5000, 5, 3)]


def test_queries_match_oracle(torch_cuda, oracle):
    from paper_2301_01356_gb300 import fbcc
    rng = np.random.default_rng(11)
    s = fbcc.Solver(1 << 16, 1 << 19)
    for g in graphs():
        off = torch_cuda.from_numpy(g.offsets).cuda()
        adj = torch_cuda.from_numpy(g.adj).cuda()
        got = s.solve(off, adj)
        exp = oracle.solve(g.offsets, g.adj)
        assert np.array_equal(got["edge_bcc"], exp["edge_bcc"])
        sets = vertex_bccs(g.offsets, exp["edge_bcc"])
        if g.n <= 12:   # every pair
            u, v = np.meshgrid(np.arange(g.n), np.arange(g.n))
            u, v = u.ravel(), v.ravel()
        else:           # both ends of random edges, random pairs, two-hop pairs
            src = np.repeat(np.arange(g.n), np.diff(g.offsets))
            a = rng.integers(0, g.nnz, 3000)
            two = g.adj[g.offsets[g.adj[a]]] if g.nnz else a
            u = np.concatenate([src[a], rng.integers(0, g.n, 3000), src[a]])
            v = np.concatenate([g.adj[a], rng.integers(0, g.n, 3000), two])
        check_queries(torch_cuda, s, g, sets, u.astype(np.int64), v.astype(np.int64), what=g.name)
    # ids outside the graph have no BCC
    bad = torch_cuda.tensor([-1, 5, 1 << 20], dtype=torch_cuda.int32, device="cuda")
    assert s.biconnected(bad, bad.flip(0)).cpu().tolist() == [-1, -1, -1]
    s.close()


def test_queries_after_batch_solve(torch_cuda, oracle):
    """After fbcc_solve_batch: global vertex ids in, each graph's own BCC numbering out."""
    from paper_2301_01356_gb300 import fbcc
    torch = torch_cuda
    gs = [gg.grid(20, 30, p=0.65, seed=1), gg.cycle_chain(800, 5, 3, 100, 2), gg.uniform(900, 2000, 3)]
    vb = np.zeros(len(gs) + 1, np.int64)
    ab = np.zeros(len(gs) + 1, np.int64)
    for i, g in enumerate(gs):
        vb[i + 1], ab[i + 1] = vb[i] + g.n, ab[i] + g.nnz
    loff = np.concatenate([g.offsets[:-1] for g in gs]).astype(np.int32)
    ladj = np.concatenate([g.adj for g in gs]).astype(np.int32)
    s = fbcc.Solver(int(vb[-1]), int(ab[-1]))
    dev = lambda a: torch.from_numpy(a).cuda()
    stats = torch.zeros(len(gs) * 5, dtype=torch.int64, device="cuda")
    fbcc.fbcc_solve_batch(dev(vb), dev(ab), vb, ab, dev(loff), dev(ladj), s.edge_bcc, s.bcc_head, s.is_ap,
                          s.is_bridge, stats, s.ws)
    rng = np.random.default_rng(2)
    for i, g in enumerate(gs):
        sets = vertex_bccs(g.offsets, oracle.solve(g.offsets, g.adj)["edge_bcc"])
        src = np.repeat(np.arange(g.n), np.diff(g.offsets))
        a = rng.integers(0, g.nnz, 500)
        u = np.concatenate([src[a], rng.integers(0, g.n, 500)])
        v = np.concatenate([g.adj[a], rng.integers(0, g.n, 500)])
        check_queries(torch, s, g, sets, u, v, base=int(vb[i]), what=f"batch graph {i}")
    s.close()


def test_query_without_solve_is_refused(torch_cuda):
    from paper_2301_01356_gb300 import fbcc
    s = fbcc.Solver(100, 100)
    x = torch_cuda.zeros(3, dtype=torch_cuda.int32, device="cuda")
    with pytest.raises(fbcc.FbccError):
        s.biconnected(x, x)
    s.close()
