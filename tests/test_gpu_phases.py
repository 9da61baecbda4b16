"""GPU intermediate phases, checked on the GPU's own spanning forest.

The forest (First-CC), the rooting (parent/first/last), the tags (w1/w2,
low/high), the fence and bridge flags and the Last-CC labels are each recomputed
on the CPU from their definitions (Algorithm 1 and sections 3.1-3.2), using the
forest the GPU chose, since any spanning forest is valid.
"""
import numpy as np
import pytest
from scipy.sparse import coo_matrix, csr_matrix
from scipy.sparse.csgraph import connected_components

from paper_2301_01356_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _partition_equal(a, b):
    """Same partition of indices (labels may differ)."""
    pairs = set(zip(a.tolist(), b.tolist()))
    return len(pairs) == len(set(a.tolist())) == len(set(b.tolist()))


def phase_check(torch, g, cfg=None):
    from paper_2301_01356_gb300 import fbcc
    s = fbcc.Solver(g.n, g.nnz, profile=1, **(cfg or {}))
    off = torch.from_numpy(g.offsets).cuda()
    adj = torch.from_numpy(g.adj).cuda()
    s.solve(off, adj)
    rd = lambda k: fbcc.fbcc_debug_read(s.ws, k, g.n).astype(np.int64)
    n = g.n
    src = np.repeat(np.arange(n), np.diff(g.offsets))
    dst = g.adj.astype(np.int64)
    A = csr_matrix((np.ones(g.nnz), g.adj, g.offsets), shape=(n, n))
    ncc, cc = connected_components(A, directed=False)

    # --- First-CC: the forest (as rooted by the next step) spans G ------------
    parent0 = rd("parent")
    h = np.nonzero(parent0 >= 0)[0]
    fu, fv = h, parent0[h]
    assert fu.size == n - ncc, "forest has n - #CC edges"
    assert np.all(A[fu, fv].A1 == 1), "forest edges are graph edges"
    F = coo_matrix((np.ones(fu.size), (fu, fv)), shape=(n, n))
    fcc, flab = connected_components(F, directed=False)
    assert fcc == ncc and _partition_equal(flab, cc), "forest spans every component"

    # --- Rooting ---------------------------------------------------------------
    first, last, parent = rd("first"), rd("last"), rd("parent")
    roots = np.nonzero(parent < 0)[0]
    cmin = np.full(ncc, n)
    np.minimum.at(cmin, cc, np.arange(n))
    assert set(roots.tolist()) == set(cmin.tolist()), "each component rooted at its smallest vertex"
    assert np.array_equal(np.sort(first), np.arange(n)), "first is a permutation"
    fe = {(min(a, b), max(a, b)) for a, b in zip(fu.tolist(), fv.tolist())}
    nr = np.nonzero(parent >= 0)[0]
    pe = {(min(a, b), max(a, b)) for a, b in zip(nr.tolist(), parent[nr].tolist())}
    assert pe == fe, "parent edges are the forest edges"
    p = parent[nr]
    assert np.all(first[p] < first[nr]) and np.all(last[nr] <= last[p]) and np.all(first[nr] <= last[nr])
    size = last - first + 1
    child_sum = np.zeros(n, np.int64)
    np.add.at(child_sum, p, size[nr])
    assert np.array_equal(size, 1 + child_sum), "subtree sizes add up"

    # --- Tagging: w1/w2 by definition, low/high bottom-up ------------------------
    tree_arc = (parent[dst] == src) | (parent[src] == dst)
    w1 = first.copy()
    w2 = first.copy()
    nt = ~tree_arc
    np.minimum.at(w1, src[nt], first[dst[nt]])
    np.maximum.at(w2, src[nt], first[dst[nt]])
    ord_ = np.argsort(first)
    # The GPU leaves out only the parent arc: arcs to children cannot lower w1, and
    # may raise w2 only to values inside every ancestor's subtree range, which
    # leaves low/high (checked next, from the definition) unchanged.
    w2c = first.copy()
    npar = parent[src] != dst
    np.maximum.at(w2c, src[npar], first[dst[npar]])
    assert np.array_equal(rd("w1"), w1[ord_]) and np.array_equal(rd("w2"), w2c[ord_]), "w1/w2"
    nnz = g.nnz
    dirb = np.unpackbits(fbcc.fbcc_debug_read(s.ws, "dirb", (nnz + 7) // 8), bitorder="little")[:nnz]
    assert np.array_equal(dirb.astype(bool), first[dst] > first[src]), "direction bits"
    low, high = w1.copy(), w2.copy()
    for v in ord_[::-1]:                       # children before parents
        if parent[v] >= 0:
            low[parent[v]] = min(low[parent[v]], low[v])
            high[parent[v]] = max(high[parent[v]], high[v])
    assert np.array_equal(rd("low"), low[ord_]) and np.array_equal(rd("high"), high[ord_]), "low/high"

    # --- Fence, bridge, Last-CC labels -----------------------------------------
    bridge = (parent >= 0) & (low == first) & (high <= last)
    vb = fbcc.fbcc_debug_read(s.ws, "vbits", n)
    assert np.array_equal((vb & 1).astype(bool), bridge), "bridge flags"
    fence = np.zeros(n, bool)
    fence[nr] = (first[p] <= low[nr]) & (last[p] >= high[nr])
    assert np.array_equal(rd("ord"), ord_), "vertex by preorder number"
    assert np.array_equal(rd("porig"), parent[ord_]), "parent by preorder number"
    assert np.array_equal((vb & 2).astype(bool), fence), "fence flags"
    assert int(fbcc.fbcc_debug_read(s.ws, "err", 1)[0]) == 0, "device error bits"
    back = nt & (((first[src] <= first[dst]) & (first[dst] <= last[src])) |
                 ((first[dst] <= first[src]) & (first[src] <= last[dst])))
    cross = nt & ~back
    plain = nr[~fence[nr]]
    su = np.concatenate([plain, src[cross]])
    sv = np.concatenate([parent[plain], dst[cross]])
    S = coo_matrix((np.ones(su.size), (su, sv)), shape=(n, n))
    _, slab = connected_components(S, directed=False)
    lab = rd("label")
    if not _partition_equal(lab[nr], slab[nr]):
        # diagnostics: skeleton edges whose endpoints got different labels, and
        # label classes that span several skeleton components
        miss_plain = plain[lab[plain] != lab[parent[plain]]]
        cs, cd = src[cross], dst[cross]
        miss_cross = np.nonzero(lab[cs] != lab[cd])[0]
        pairs = {}
        for a, b in zip(lab[nr].tolist(), slab[nr].tolist()):
            pairs.setdefault(a, set()).add(b)
        over = [k for k, v in pairs.items() if len(v) > 1]
        root_in = [int(r) for r in roots if (lab == r).sum() > 1]
        raise AssertionError(
            f"Last-CC labels differ: plain edges split {miss_plain.size}/{plain.size}, cross arcs split "
            f"{miss_cross.size}/{cs.size}, labels spanning several components {len(over)}, roots with members "
            f"{len(root_in)}; sample split plain {[(int(v), int(parent[v]), int(first[v]), int(low[v]), int(high[v]), int(first[parent[v]]), int(last[parent[v]])) for v in miss_plain[:3]]}; "
            f"sample over {[(k, sorted(pairs[k])[:4]) for k in over[:3]]}")
    s.close()


@pytest.mark.parametrize("family", ["grid", "uniform", "chain", "rmat", "path", "knn"])
def test_phases(torch_cuda, family):
    g = {
        "grid": lambda: gg.grid(211, 173, p=0.62, extra_frac=0.001, seed=9),
        "uniform": lambda: gg.uniform(30011, 70001, 5),
        "chain": lambda: gg.cycle_chain(20011, 30, 3, 2000, 3),
        "rmat": lambda: gg.rmat(14, 8, seed=2),
        "path": lambda: gg.path(10007),
        "knn": lambda: gg.knn3(20000, 4, 3),
    }[family]()
    phase_check(torch_cuda, g)
    phase_check(torch_cuda, g, {"ruler_stride": 8, "cc_local": 4096})
    phase_check(torch_cuda, g, {"cc_sample": 2, "lcc_sample": 2})
    phase_check(torch_cuda, g, {"cc_ldd": 4})
