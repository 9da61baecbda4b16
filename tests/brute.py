"""Brute-force biconnectivity for tiny graphs (test pins for the oracle).

Everything here follows the plain definitions, with no DFS bookkeeping:

* articulation point / bridge: removal increases the number of connected
  components (section 2, "Notation");
* two edges are in the same BCC iff they are equal or lie on a common simple cycle
  (the edge relation used by Tarjan-Vishkin, appendix A, and the cycle fact of
  section 4.2), found here by enumerating every simple cycle;
* head of a BCC: its shallowest vertex in a BFS tree rooted at the smallest vertex
  id of its connected component (section 4.2; the head does not depend on which
  spanning tree is used once the root is fixed).
"""
from __future__ import annotations

from collections import deque

import numpy as np


def edges_of(offsets, adj):
    n = len(offsets) - 1
    return [(u, int(adj[a])) for u in range(n) for a in range(offsets[u], offsets[u + 1]) if u < adj[a]]


def n_components(n, edges, removed_vertex=None, removed_edge=None):
    parent = list(range(n))

    def find(x):
        while parent[x] != x:
            x = parent[x]
        return x

    for e in edges:
        if e == removed_edge or removed_vertex in e:
            continue
        a, b = find(e[0]), find(e[1])
        if a != b:
            parent[a] = b
    return sum(1 for v in range(n) if v != removed_vertex and find(v) == v)


def simple_cycles(n, edges):
    """Every simple cycle (length >= 3) as a list of vertices, each at least once."""
    nbr = [[] for _ in range(n)]
    for u, v in edges:
        nbr[u].append(v)
        nbr[v].append(u)
    out = []
    for s in range(n):
        # cycles whose smallest vertex is s
        stack = [(s, [s])]
        while stack:
            x, pathv = stack.pop()
            for y in nbr[x]:
                if y == s and len(pathv) >= 3:
                    out.append(list(pathv))
                elif y > s and y not in pathv:
                    stack.append((y, pathv + [y]))
    return out


def brute_bcc(offsets, adj):
    """Canonical outputs in the oracle's format, from the definitions above."""
    offsets = [int(x) for x in offsets]
    n = len(offsets) - 1
    edges = edges_of(offsets, adj)          # in CSR order of the src<dst arc = edge id order
    eid = {e: i for i, e in enumerate(edges)}
    base = n_components(n, edges)
    is_ap = np.array([n_components(n, edges, removed_vertex=v) > base for v in range(n)], np.uint8)
    bridge_e = [n_components(n, edges, removed_edge=e) > base for e in edges]

    # edge blocks: union the edges of every simple cycle
    par = list(range(len(edges)))

    def f(x):
        while par[x] != x:
            x = par[x]
        return x

    for cyc in simple_cycles(n, edges):
        ids = [eid[(min(a, b), max(a, b))] for a, b in zip(cyc, cyc[1:] + cyc[:1])]
        for i in ids[1:]:
            ra, rb = f(ids[0]), f(i)
            if ra != rb:
                par[ra] = rb
    blocks = {}
    for i in range(len(edges)):
        blocks.setdefault(f(i), []).append(i)
    ordered = sorted(blocks.values(), key=min)       # by smallest edge id
    blk_of = {}
    for k, ids in enumerate(ordered):
        for i in ids:
            blk_of[i] = k

    # BFS depth from the smallest vertex of each component
    depth = [-1] * n
    nbr = [[] for _ in range(n)]
    for u, v in edges:
        nbr[u].append(v)
        nbr[v].append(u)
    for s in range(n):
        if depth[s] >= 0:
            continue
        depth[s] = 0
        q = deque([s])
        while q:
            x = q.popleft()
            for y in nbr[x]:
                if depth[y] < 0:
                    depth[y] = depth[x] + 1
                    q.append(y)
    heads = []
    for ids in ordered:
        verts = {x for i in ids for x in edges[i]}
        dmin = min(depth[x] for x in verts)
        shallow = [x for x in verts if depth[x] == dmin]
        assert len(shallow) == 1, "the shallowest vertex of a block is unique"
        heads.append(shallow[0])

    nnz = offsets[-1]
    edge_bcc = np.empty(nnz, np.int32)
    is_bridge = np.empty(nnz, np.uint8)
    for u in range(n):
        for a in range(offsets[u], offsets[u + 1]):
            e = (min(u, int(adj[a])), max(u, int(adj[a])))
            edge_bcc[a] = blk_of[eid[e]]
            is_bridge[a] = bridge_e[eid[e]]
    return {
        "edge_bcc": edge_bcc, "bcc_head": np.array(heads, np.int32), "is_ap": is_ap,
        "is_bridge": is_bridge, "n_bcc": len(ordered), "n_ap": int(is_ap.sum()),
        "n_bridge": int(sum(bridge_e)), "n_cc": base,
    }
