"""Seeded synthetic inputs: symmetric, sorted, simple CSR graphs.

This module makes inputs only; it holds none of the biconnectivity arithmetic and
is the one piece shared by the oracle-side tests and the GPU path. The large
families (uniform random, thinned grid, R-MAT, cycle chains, k-NN) come from the
OpenMP C generator ``csrc/graphgen.c`` (counter-based SplitMix64 draws, so the
output does not depend on the thread count); the tiny closed-form families used
to pin the oracle are built here with numpy.

Every function returns a :class:`Graph` with int64 ``offsets`` (n+1) and int32
``adj`` (2m), each adjacency list sorted ascending.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "graphgen.c")
_LIB = os.path.join(_HERE, "_build", "libgraphgen.so")
_lock = threading.Lock()
_lib = None


@dataclasses.dataclass
class Graph:
    offsets: np.ndarray          # int64, n+1
    adj: np.ndarray              # int32, 2m
    name: str = ""
    truth_bcc: int = -1          # ground truth where the family fixes it
    truth_ap: int = -1

    @property
    def n(self) -> int:
        return int(self.offsets.size - 1)

    @property
    def nnz(self) -> int:
        return int(self.offsets[-1])

    @property
    def m(self) -> int:
        return self.nnz // 2


@dataclasses.dataclass
class Batch:
    """Many graphs packed into one CSR with per-graph bases (local ids and offsets)."""
    vtx_base: np.ndarray         # int64, G+1
    arc_base: np.ndarray         # int64, G+1
    local_off: np.ndarray        # int32, n_total: list start relative to the graph's arc base
    local_adj: np.ndarray        # int32, nnz_total: neighbour ids local to the graph
    family: np.ndarray           # int32, G: 0 uniform, 1 grid, 2 cycle chain, 3 k-NN
    truth_bcc: np.ndarray        # int64, G (-1 where the family fixes none)
    truth_ap: np.ndarray

    FAMILIES = ("uniform", "grid", "chain", "knn")

    @property
    def G(self) -> int:
        return int(self.vtx_base.size - 1)

    @property
    def n_total(self) -> int:
        return int(self.vtx_base[-1])

    @property
    def nnz_total(self) -> int:
        return int(self.arc_base[-1])

    def sizes(self) -> np.ndarray:
        return np.diff(self.vtx_base)

    def graph(self, g: int) -> "Graph":
        v0, v1 = int(self.vtx_base[g]), int(self.vtx_base[g + 1])
        a0, a1 = int(self.arc_base[g]), int(self.arc_base[g + 1])
        off = np.empty(v1 - v0 + 1, np.int64)
        off[:-1] = self.local_off[v0:v1]
        off[-1] = a1 - a0
        return Graph(off, self.local_adj[a0:a1].copy(), f"batch[{g}]", int(self.truth_bcc[g]), int(self.truth_ap[g]))

    def subset(self, idx) -> "Batch":
        """A new packed batch of the graphs `idx` (in that order)."""
        idx = np.asarray(idx, dtype=np.int64)
        nv = np.diff(self.vtx_base)[idx]
        na = np.diff(self.arc_base)[idx]
        vb = np.zeros(idx.size + 1, np.int64)
        ab = np.zeros(idx.size + 1, np.int64)
        np.cumsum(nv, out=vb[1:])
        np.cumsum(na, out=ab[1:])
        loff = np.empty(int(vb[-1]), np.int32)
        ladj = np.empty(int(ab[-1]), np.int32)
        for i, g in enumerate(idx):
            loff[vb[i]:vb[i + 1]] = self.local_off[self.vtx_base[g]:self.vtx_base[g + 1]]
            ladj[ab[i]:ab[i + 1]] = self.local_adj[self.arc_base[g]:self.arc_base[g + 1]]
        return Batch(vb, ab, loff, ladj, self.family[idx].copy(), self.truth_bcc[idx].copy(),
                     self.truth_ap[idx].copy())


class _CSR(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("off", ctypes.POINTER(ctypes.c_int64)), ("adj", ctypes.POINTER(ctypes.c_int32)),
                ("truth_bcc", ctypes.c_int64), ("truth_ap", ctypes.c_int64)]


class _BATCH(ctypes.Structure):
    _fields_ = [("G", ctypes.c_int64), ("vtx_base", ctypes.POINTER(ctypes.c_int64)),
                ("arc_base", ctypes.POINTER(ctypes.c_int64)), ("loff", ctypes.POINTER(ctypes.c_int32)),
                ("ladj", ctypes.POINTER(ctypes.c_int32)), ("family", ctypes.POINTER(ctypes.c_int32)),
                ("truth_bcc", ctypes.POINTER(ctypes.c_int64)), ("truth_ap", ctypes.POINTER(ctypes.c_int64))]


def build() -> str:
    """Compile the generator library (gcc, OpenMP) unless it is up to date."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-shared", "-fPIC", _SRC,
                           "-o", tmp, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, u64, d, p = ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(_CSR)
            lib.gg_uniform.argtypes = [i64, i64, u64, p]
            lib.gg_grid.argtypes = [i64, i64, ctypes.c_int, d, d, i64, u64, p]
            lib.gg_rmat.argtypes = [ctypes.c_int, i64, d, d, d, u64, p]
            lib.gg_cycle_chain.argtypes = [i64, i64, i64, i64, u64, p]
            lib.gg_knn3.argtypes = [i64, i64, u64, p]
            lib.gg_build_csr.argtypes = [i64, i64, ctypes.c_void_p, ctypes.c_void_p, p]
            lib.gg_free.argtypes = [ctypes.c_void_p]
            lib.gg_batch_make.argtypes = [i64, u64, i64, i64, ctypes.c_int, ctypes.POINTER(_BATCH)]
            _lib = lib
        return _lib


def _take(lib, rc: int, out: _CSR, name: str) -> Graph:
    if rc:
        raise ValueError(f"generator {name} failed with code {rc}")
    n, nnz = out.n, out.nnz
    off = np.ctypeslib.as_array(out.off, shape=(n + 1,)).copy()
    adj = np.ctypeslib.as_array(out.adj, shape=(max(nnz, 1),))[:nnz].copy()
    lib.gg_free(ctypes.cast(out.off, ctypes.c_void_p))
    lib.gg_free(ctypes.cast(out.adj, ctypes.c_void_p))
    return Graph(off, adj, name, int(out.truth_bcc), int(out.truth_ap))


def from_edges(n: int, u, v, name: str = "edges") -> Graph:
    """Symmetric simple CSR of an undirected edge list (self-loops, repeats dropped)."""
    lib = _load()
    u = np.ascontiguousarray(u, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.int32)
    out = _CSR()
    rc = lib.gg_build_csr(n, u.size, u.ctypes.data, v.ctypes.data, ctypes.byref(out))
    return _take(lib, rc, out, name)


def uniform(n: int, m: int, seed: int) -> Graph:
    """n vertices, m distinct uniformly drawn edges without self-loops."""
    lib = _load()
    out = _CSR()
    return _take(lib, lib.gg_uniform(n, m, seed, ctypes.byref(out)), out, f"uniform(n={n},m={m},seed={seed})")


def grid(rows: int, cols: int, p: float = 1.0, extra_frac: float = 0.0, max_l1: int = 8,
         seed: int = 0, torus: bool = False) -> Graph:
    """rows x cols grid (id = r*cols + c), edges kept with probability p, plus
    round(extra_frac * kept) extra edges of Manhattan length 1..max_l1."""
    lib = _load()
    out = _CSR()
    rc = lib.gg_grid(rows, cols, int(torus), p, extra_frac, max_l1, seed, ctypes.byref(out))
    return _take(lib, rc, out, f"grid({rows}x{cols},p={p},extra={extra_frac},torus={torus},seed={seed})")


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 3) -> Graph:
    """R-MAT, 2^scale vertices, edge_factor * 2^scale draws, symmetrised and simplified."""
    lib = _load()
    out = _CSR()
    rc = lib.gg_rmat(scale, edge_factor, a, b, c, seed, ctypes.byref(out))
    return _take(lib, rc, out, f"rmat(scale={scale},ef={edge_factor},seed={seed})")


def cycle_chain(n: int, k: int, lmin: int = 3, lmax: int = 5000, seed: int = 0) -> Graph:
    """k cycles joined at distinct shared vertices, plus random pendant trees."""
    lib = _load()
    out = _CSR()
    rc = lib.gg_cycle_chain(n, k, lmin, lmax, seed, ctypes.byref(out))
    return _take(lib, rc, out, f"cycle_chain(n={n},k={k},seed={seed})")


def knn3(n: int, k: int = 5, seed: int = 0) -> Graph:
    """k nearest neighbours of n uniform points in the unit cube, symmetrised."""
    lib = _load()
    out = _CSR()
    return _take(lib, lib.gg_knn3(n, k, seed, ctypes.byref(out)), out, f"knn3(n={n},k={k},seed={seed})")


def batch(G: int, seed: int, nmin: int, nmax: int, families=("uniform", "grid", "chain")) -> Batch:
    """G graphs with vertex counts log-uniform on [nmin, nmax], families round-robin."""
    lib = _load()
    mask = sum(1 << Batch.FAMILIES.index(f) for f in families)
    out = _BATCH()
    rc = lib.gg_batch_make(G, seed, nmin, nmax, mask, ctypes.byref(out))
    if rc:
        raise ValueError(f"batch generator failed with code {rc}")
    take = lambda ptr, size: np.ctypeslib.as_array(ptr, shape=(max(size, 1),))[:size].copy()
    vb = take(out.vtx_base, G + 1)
    ab = take(out.arc_base, G + 1)
    res = Batch(vb, ab, take(out.loff, int(vb[-1])), take(out.ladj, int(ab[-1])), take(out.family, G),
                take(out.truth_bcc, G), take(out.truth_ap, G))
    for ptr in (out.vtx_base, out.arc_base, out.loff, out.ladj, out.family, out.truth_bcc, out.truth_ap):
        lib.gg_free(ctypes.cast(ptr, ctypes.c_void_p))
    return res


# ---- the benchmark workloads ------------------------------------------------------

def workload_uniform_64k() -> Graph:
    """n = 65,536, m = 196,608 distinct uniform edges, seed 1 (average degree 6)."""
    return uniform(65536, 196608, 1)


def workload_grid_4096() -> Graph:
    """4096 x 4096 open grid, each edge kept with p = 0.62, plus 0.1 % of the kept
    count as extra edges of Manhattan length 1..8, seed 2 (large diameter)."""
    return grid(4096, 4096, p=0.62, extra_frac=0.001, max_l1=8, seed=2)


def workload_grid_2896() -> Graph:
    """The same recipe as workload_grid_4096 on a 2896 x 2896 grid (half the vertices);
    used for detailed profiler captures."""
    return grid(2896, 2896, p=0.62, extra_frac=0.001, max_l1=8, seed=2)


def workload_batch_4096() -> Batch:
    """4,096 graphs, n log-uniform on [10^3, 10^6], uniform / thinned grid / cycle chain
    families round-robin, seed 4."""
    return batch(4096, 4, 1000, 1000000)


def workload_rmat_22() -> Graph:
    """The R-MAT recipe at scale 22 (a quarter of the vertices); profiler captures."""
    return rmat(22, 16, 0.57, 0.19, 0.19, 3)


def workload_rmat_24() -> Graph:
    """R-MAT scale 24, edge factor 16, (a,b,c) = (0.57, 0.19, 0.19), seed 3."""
    return rmat(24, 16, 0.57, 0.19, 0.19, 3)


# ---- tiny closed-form families (numpy) -------------------------------------------

def _edges(n: int, pairs, name: str) -> Graph:
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    return from_edges(n, pairs[:, 0], pairs[:, 1], name)


def cycle(n: int) -> Graph:
    return _edges(n, [(i, (i + 1) % n) for i in range(n)], f"cycle({n})")


def path(n: int) -> Graph:
    return _edges(n, [(i, i + 1) for i in range(n - 1)], f"path({n})")


def star(n: int) -> Graph:
    return _edges(n, [(0, i) for i in range(1, n)], f"star({n})")


def complete(n: int) -> Graph:
    return _edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)], f"complete({n})")


def random_tree(n: int, seed: int) -> Graph:
    rng = np.random.Generator(np.random.PCG64(seed))
    perm = rng.permutation(n)
    pairs = [(perm[i], perm[rng.integers(0, i)]) for i in range(1, n)]
    return _edges(n, pairs, f"random_tree({n},{seed})")


def cycles_chain_exact(lengths, n_extra_isolated: int = 0) -> Graph:
    """Cycles of the given lengths, cycle i+1 sharing one vertex with cycle i (a
    different shared vertex each time), plus isolated vertices."""
    pairs, nxt, join = [], 0, None
    for L in lengths:
        verts = ([join] if join is not None else []) + list(range(nxt, nxt + L - (join is not None)))
        nxt += L - (join is not None)
        pairs += [(verts[i], verts[(i + 1) % L]) for i in range(L)]
        join = verts[-1]
    return _edges(nxt + n_extra_isolated, pairs, f"cycles_chain({list(lengths)})")


def disjoint_union(*graphs: Graph) -> Graph:
    offs, adjs, base, abase = [np.zeros(1, np.int64)], [], 0, 0
    for g in graphs:
        offs.append(g.offsets[1:] + abase)
        adjs.append(g.adj + base)
        base += g.n
        abase += g.nnz
    return Graph(np.concatenate(offs), np.concatenate(adjs).astype(np.int32) if adjs else np.zeros(0, np.int32),
                 "union(" + ",".join(g.name for g in graphs) + ")")


def relabel(g: Graph, perm: np.ndarray) -> Graph:
    """The same graph with vertex v renamed perm[v]."""
    n = g.n
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(g.offsets))
    keep = src < g.adj
    return from_edges(n, perm[src[keep]], perm[g.adj[keep].astype(np.int64)], g.name + "+relabel")
