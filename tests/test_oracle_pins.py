"""Pins for the Hopcroft-Tarjan oracle, independent of the oracle itself.

Each pin comes from the paper or from mathematics, not from re-running the
oracle's own steps: hand-derived examples (golden), the closed forms the paper
prints for its synthetic graphs, textbook closed forms, brute force from the
definitions on tiny graphs, block-cut-tree identities and generator ground truth.
"""
import itertools
import json
import os

import numpy as np
import pytest

import brute
from paper_2301_01356_gb300 import graphgen as gg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _arc_src(g):
    return np.repeat(np.arange(g.n), np.diff(g.offsets))


def _edge_ids(g):
    """edge id of every arc: rank of its src<dst arc in CSR order."""
    src = _arc_src(g)
    fwd = src < g.adj
    ids = np.full(g.nnz, -1, np.int64)
    ids[fwd] = np.arange(int(fwd.sum()))
    key = {(int(s), int(d)): int(i) for s, d, i in zip(src[fwd], g.adj[fwd], ids[fwd])}
    for a in np.nonzero(~fwd)[0]:
        ids[a] = key[(int(g.adj[a]), int(src[a]))]
    return ids


def test_hand_examples(oracle):
    cases = json.load(open(os.path.join(GOLDEN, "hand_examples.json")))["cases"]
    for c in cases:
        e = np.array(c["edges"], np.int64).reshape(-1, 2)
        g = gg.from_edges(c["n"], e[:, 0], e[:, 1])
        r = oracle.solve(g.offsets, g.adj)
        ids = _edge_ids(g)
        exp_blk = np.array(c["edge_block"], np.int32)
        assert np.array_equal(r["edge_bcc"], exp_blk[ids] if ids.size else exp_blk[:0]), c["name"]
        assert r["bcc_head"].tolist() == c["bcc_head"], c["name"]
        assert np.nonzero(r["is_ap"])[0].tolist() == c["ap"], c["name"]
        bset = {tuple(sorted(b)) for b in c["bridges"]}
        src = _arc_src(g)
        got = {(min(int(s), int(d)), max(int(s), int(d))) for s, d, f in zip(src, g.adj, r["is_bridge"]) if f}
        assert got == bset, c["name"]
        assert r["n_cc"] == c["n_cc"] and r["n_bcc"] == len(c["bcc_head"]), c["name"]
        assert r["n_bridge"] == len(bset) and r["n_ap"] == len(c["ap"]), c["name"]


def test_paper_synthetic_rows(oracle):
    """Chains have n-1 BCCs and circular grids one BCC (section 6, graph table)."""
    spec = json.load(open(os.path.join(GOLDEN, "paper_closed_forms.json")))
    for c in spec["cases"]:
        if c["family"] == "path":
            assert c["paper_bcc"] == c["paper_n"] - 1
            g = gg.path(c["test_n"])
            r = oracle.solve(g.offsets, g.adj)
            assert r["n_bcc"] == c["test_n"] - 1 and r["n_bridge"] == c["test_n"] - 1
            assert r["n_ap"] == c["test_n"] - 2
        else:
            assert c["paper_bcc"] == 1
            g = gg.grid(c["test_rows"], c["test_cols"], torus=True)
            r = oracle.solve(g.offsets, g.adj)
            assert r["n_bcc"] == 1 and r["n_ap"] == 0 and r["n_bridge"] == 0
            assert np.all(r["edge_bcc"] == 0) and r["bcc_head"].tolist() == [0]


@pytest.mark.parametrize("n", [3, 4, 7, 50, 1001])
def test_cycle_and_complete(oracle, n):
    for g in (gg.cycle(n), gg.complete(min(n, 60))):
        r = oracle.solve(g.offsets, g.adj)
        assert (r["n_bcc"], r["n_ap"], r["n_bridge"], r["n_cc"]) == (1, 0, 0, 1)
        assert np.all(r["edge_bcc"] == 0) and r["bcc_head"].tolist() == [0]


@pytest.mark.parametrize("seed", range(6))
def test_random_tree(oracle, seed):
    n = [2, 3, 10, 100, 1000, 20000][seed]
    g = gg.random_tree(n, seed)
    r = oracle.solve(g.offsets, g.adj)
    deg = np.diff(g.offsets)
    assert r["n_bcc"] == n - 1 and r["n_bridge"] == n - 1 and np.all(r["is_bridge"] == 1)
    assert np.array_equal(r["is_ap"], (deg >= 2).astype(np.uint8))
    # every edge is its own block: block ids are exactly the edge ids
    assert np.array_equal(np.sort(r["edge_bcc"]), np.repeat(np.arange(n - 1), 2))


def test_star_and_isolated(oracle):
    g = gg.star(9)
    r = oracle.solve(g.offsets, g.adj)
    assert r["n_bcc"] == 8 and r["is_ap"].tolist() == [1] + [0] * 8 and r["bcc_head"].tolist() == [0] * 8
    g = gg.from_edges(5, [], [])
    r = oracle.solve(g.offsets, g.adj)
    assert (r["n_bcc"], r["n_ap"], r["n_bridge"], r["n_cc"]) == (0, 0, 0, 5)
    g = gg.from_edges(0, [], [])
    r = oracle.solve(g.offsets, g.adj)
    assert (r["n_bcc"], r["n_cc"]) == (0, 0)


@pytest.mark.parametrize("shape", [(2, 2), (2, 7), (5, 5), (13, 4), (64, 64)])
def test_full_grid(oracle, shape):
    for torus in (False, True):
        if torus and min(shape) < 3:
            continue
        g = gg.grid(*shape, torus=torus)
        r = oracle.solve(g.offsets, g.adj)
        assert (r["n_bcc"], r["n_ap"], r["n_bridge"], r["n_cc"]) == (1, 0, 0, 1)


@pytest.mark.parametrize("lengths", [[3, 3], [3, 4, 5], [7] * 10, [3, 100, 4, 5, 6, 3, 3]])
def test_chain_of_cycles(oracle, lengths):
    g = gg.cycles_chain_exact(lengths, n_extra_isolated=2)
    r = oracle.solve(g.offsets, g.adj)
    k = len(lengths)
    assert r["n_bcc"] == k and r["n_ap"] == k - 1 and r["n_bridge"] == 0 and r["n_cc"] == 3


@pytest.mark.parametrize("seed", range(8))
def test_generator_chain_truth(oracle, seed):
    n = [50, 200, 1000, 5000, 20000, 3, 10, 100000][seed]
    k = [2, 5, 10, 64, 30, 1, 3, 40][seed]
    g = gg.cycle_chain(n, k, 3, 200 if n < 1000 else 5000, seed)
    r = oracle.solve(g.offsets, g.adj)
    assert r["n_bcc"] == g.truth_bcc and r["n_ap"] == g.truth_ap


def test_brute_force_exhaustive_n5(oracle):
    pairs = list(itertools.combinations(range(5), 2))
    for mask in range(1 << len(pairs)):
        e = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
        g = gg.from_edges(5, [x for x, _ in e], [y for _, y in e])
        r, b = oracle.solve(g.offsets, g.adj), brute.brute_bcc(g.offsets, g.adj)
        for k in ("edge_bcc", "bcc_head", "is_ap", "is_bridge", "n_bcc", "n_ap", "n_bridge", "n_cc"):
            assert np.array_equal(r[k], b[k]), (mask, k)


@pytest.mark.parametrize("seed", range(40))
def test_brute_force_random(oracle, seed):
    rng = np.random.default_rng(1000 + seed)
    for _ in range(5):
        n = int(rng.integers(6, 10))
        p = float(rng.uniform(0.15, 0.6))
        e = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < p]
        perm = rng.permutation(n)
        g = gg.from_edges(n, [perm[x] for x, _ in e], [perm[y] for _, y in e])
        r, b = oracle.solve(g.offsets, g.adj), brute.brute_bcc(g.offsets, g.adj)
        for k in ("edge_bcc", "bcc_head", "is_ap", "is_bridge", "n_bcc", "n_ap", "n_bridge", "n_cc"):
            assert np.array_equal(r[k], b[k]), (seed, k)


def _blocks(g, r):
    src = _arc_src(g)
    verts = [set() for _ in range(r["n_bcc"])]
    nedge = np.zeros(r["n_bcc"], np.int64)
    for s, d, k in zip(src, g.adj, r["edge_bcc"]):
        verts[k].update((int(s), int(d)))
        nedge[k] += 1
    return verts, nedge // 2


@pytest.mark.parametrize("seed", range(5))
def test_block_cut_identities(oracle, seed):
    """Sum over BCCs of (|V(C)|-1) = n - #CC; two BCCs share at most one vertex
    (section 4.2, first fact); heads are articulation points or component roots
    (section 4.2, head/AP lemma); bridges are the one-edge BCCs."""
    g = [gg.uniform(3000, 3600, seed), gg.grid(60, 60, p=0.6, seed=seed),
         gg.cycle_chain(4000, 12, 3, 300, seed), gg.uniform(500, 2500, seed), gg.knn3(3000, 3, seed)][seed]
    r = oracle.solve(g.offsets, g.adj)
    verts, nedge = _blocks(g, r)
    assert sum(len(v) - 1 for v in verts) == g.n - r["n_cc"]
    count = {}
    for v in verts:
        for x in v:
            count[x] = count.get(x, 0) + 1
    ap = {x for x, c in count.items() if c >= 2}
    assert ap == set(np.nonzero(r["is_ap"])[0].tolist())
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components
    ncc, lab = connected_components(csr_matrix((np.ones(g.nnz), g.adj, g.offsets), shape=(g.n, g.n)))
    root = np.full(ncc, g.n)
    np.minimum.at(root, lab, np.arange(g.n))
    assert ncc == r["n_cc"]
    for k, h in enumerate(r["bcc_head"]):
        # the head is in its block and is an articulation point or its component's root
        assert h in verts[k] and (r["is_ap"][h] or h == root[lab[h]])
        # and it is the block's vertex closest to that root: every other block vertex
        # lies beyond it, so removing the head cuts them off unless the head is the root
    src = _arc_src(g)
    assert np.array_equal(r["is_bridge"].astype(bool), nedge[r["edge_bcc"]] == 1)
    assert r["n_bridge"] == int((nedge == 1).sum())
    # canonical numbering: block ids appear in increasing order of their first edge id
    ids = _edge_ids(g)
    firsts = np.full(r["n_bcc"], np.iinfo(np.int64).max)
    np.minimum.at(firsts, r["edge_bcc"], ids)
    assert np.all(np.diff(firsts) > 0)
    del src


@pytest.mark.parametrize("seed", range(3))
def test_relabel_invariance(oracle, seed):
    """Renaming vertices permutes the AP set and keeps the edge partition and
    bridges (heads may change: the roots change)."""
    g = gg.uniform(2000, 2600, 77 + seed)
    rng = np.random.default_rng(seed)
    perm = rng.permutation(g.n)
    h = gg.relabel(g, perm)
    r, s = oracle.solve(g.offsets, g.adj), oracle.solve(h.offsets, h.adj)
    assert r["n_bcc"] == s["n_bcc"] and r["n_bridge"] == s["n_bridge"] and r["n_cc"] == s["n_cc"]
    assert np.array_equal(s["is_ap"][perm], r["is_ap"])
    src_g, src_h = _arc_src(g), _arc_src(h)
    lab_h = {(int(a), int(b)): int(k) for a, b, k in zip(src_h, h.adj, s["edge_bcc"])}
    pairs = {(int(k), lab_h[(int(perm[a]), int(perm[b]))]) for a, b, k in zip(src_g, g.adj, r["edge_bcc"])}
    assert len(pairs) == r["n_bcc"]        # a bijection between the two block numberings


def test_rejects_bad_input(oracle):
    g = gg.cycle(5)
    off, adj = g.offsets.copy(), g.adj.copy()
    with pytest.raises(oracle.OracleError):
        oracle.solve(off[:-1], adj)                      # offsets[n] != nnz
    bad = adj.copy(); bad[0] = 0                         # self-loop at vertex 0
    assert oracle.check_csr(off, bad) == 2
    bad = adj.copy(); bad[0], bad[1] = bad[1], bad[0]    # unsorted list
    assert oracle.check_csr(off, bad) == 2
    bad = adj.copy(); bad[0] = 2                         # 0->2 without 2->0
    assert oracle.check_csr(off, bad) == 2
    bad = adj.copy(); bad[0] = 9                         # id out of range
    assert oracle.check_csr(off, bad) == 1
    assert oracle.check_csr(off, adj) == 0


@pytest.mark.parametrize("seed", range(6))
def test_against_networkx(oracle, seed):
    """An independent library (networkx: biconnected_component_edges,
    articulation_points, bridges) on medium graphs of every family. The oracle's
    per-edge labels must induce the same partition of the edges, its canonical
    numbering must follow smallest edge id, and each block's head must be the
    block's vertex nearest to its component's smallest vertex (BFS depth), which
    is unique for a block."""
    nx = pytest.importorskip("networkx")
    g = [gg.uniform(1500, 2600, seed), gg.grid(40, 45, p=0.62, seed=seed),
         gg.cycle_chain(1800, 10, 3, 120, seed), gg.knn3(1500, 3, seed),
         gg.disjoint_union(gg.uniform(300, 500, seed), gg.grid(20, 20, p=0.7, seed=seed), gg.from_edges(4, [], [])),
         gg.uniform(800, 4000, seed)][seed]
    r = oracle.solve(g.offsets, g.adj)
    src = _arc_src(g)
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    G.add_edges_from((int(s), int(d)) for s, d in zip(src, g.adj) if s < d)
    eid = {}
    for i, (s, d) in enumerate((int(s), int(d)) for s, d in zip(src, g.adj) if s < d):
        eid[(s, d)] = i
    # partition of the edges, named by smallest edge id, ranked
    blocks = [sorted(eid[(min(a, b), max(a, b))] for a, b in comp) for comp in nx.biconnected_component_edges(G)]
    blocks.sort(key=lambda b: b[0])
    lab = {}
    for k, b in enumerate(blocks):
        for e in b:
            lab[e] = k
    ids = _edge_ids(g)
    assert r["n_bcc"] == len(blocks)
    assert all(int(r["edge_bcc"][a]) == lab[int(ids[a])] for a in range(g.nnz))
    # articulation points and bridges
    ap = np.zeros(g.n, np.uint8)
    ap[list(nx.articulation_points(G))] = 1
    assert np.array_equal(r["is_ap"], ap)
    br = {eid[(min(a, b), max(a, b))] for a, b in nx.bridges(G)}
    assert all(bool(r["is_bridge"][a]) == (int(ids[a]) in br) for a in range(g.nnz))
    assert r["n_cc"] == nx.number_connected_components(G)
    # heads: the block's vertex nearest to the component's smallest vertex
    depth = {}
    for comp in nx.connected_components(G):
        depth.update(nx.single_source_shortest_path_length(G, min(comp)))
    for k, b in enumerate(blocks):
        verts = set()
        for e in b:
            a = int(np.nonzero(ids == e)[0][0])
            verts.update((int(src[a]), int(g.adj[a])))
        dmin = min(depth[v] for v in verts)
        near = [v for v in verts if depth[v] == dmin]
        assert len(near) == 1 and int(r["bcc_head"][k]) == near[0], k
