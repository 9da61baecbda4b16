"""Plant plausible mistakes in a copy of the oracle and check the pins catch each.

The copy is compiled into a temporary directory on the CPU; the oracle source in
the repository is never modified.
"""
import itertools
import multiprocessing
import os

import numpy as np
import pytest

import brute
from oracle import ht
from paper_2301_01356_gb300 import graphgen as gg

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "ht_oracle.c")

MUTANTS = {
    "fence test strict": ("if (low[u] >= first[p])", "if (low[u] > first[p])"),
    "root AP with one block": ("if (root_blocks >= 2) is_ap[s] = 1;", "if (root_blocks >= 1) is_ap[s] = 1;"),
    "back edge ignored in low": ("if (first[w] < low[u]) low[u] = first[w];", "if (0) low[u] = first[w];"),
    "low not propagated to parent": ("if (low[u] < low[p]) low[p] = low[u];", "if (0) low[p] = low[u];"),
    "blocks not sorted by key": ("qsort(kb, nblk, sizeof(keyed_block), cmp_keyed);", "(void)cmp_keyed;"),
    "bridge rule loose": ("is_bridge[a] = nedge[b] == 1;", "is_bridge[a] = nedge[b] <= 3;"),
    "head is the child": ("head[b] = p;", "head[b] = u;"),
    "key is the last edge": ("if (eid < kb[b].key) kb[b].key = eid;", "kb[b].key = eid;"),
    "reverse arc unlabelled": ("int64_t key_arc = x < y ? e : find_arc(off, adj, y, x);",
                               "int64_t key_arc = e;"),
}


def _pin_suite(lib):
    """A fast subset of the pins; returns True when every pin holds."""
    def solve(g):
        try:
            return ht.solve(g.offsets, g.adj, lib=lib)
        except Exception:
            return None

    try:
        for mask in range(0, 1 << 10, 3):
            pairs = list(itertools.combinations(range(5), 2))
            e = [pairs[i] for i in range(10) if mask >> i & 1]
            g = gg.from_edges(5, [x for x, _ in e], [y for _, y in e])
            r, b = solve(g), brute.brute_bcc(g.offsets, g.adj)
            if r is None:
                return False
            for k in ("edge_bcc", "bcc_head", "is_ap", "is_bridge", "n_bcc", "n_ap", "n_bridge"):
                if not np.array_equal(r[k], b[k]):
                    return False
        for g, nb in ((gg.cycle(6), 1), (gg.path(6), 5), (gg.grid(5, 5), 1), (gg.cycles_chain_exact([3, 4, 5]), 3)):
            r = solve(g)
            if r is None or r["n_bcc"] != nb:
                return False
        return True
    except Exception:
        return False


def _run_pins(path):
    """Child-process body: exit 0 when every pin holds for the library at ``path``."""
    os._exit(0 if _pin_suite(ht.load(path)) else 1)


def _pins_in_child(path):
    """True when the pins all hold. A planted mistake can corrupt memory (an edge
    stack underflow, say), so the library runs in a spawned child; a crash or a
    timeout counts as caught."""
    ctx = multiprocessing.get_context("spawn")
    proc = ctx.Process(target=_run_pins, args=(path,))
    proc.start()
    proc.join(120)
    if proc.is_alive():
        proc.kill()
        proc.join()
        return False
    return proc.exitcode == 0


def test_unmodified_oracle_passes():
    assert _pins_in_child(ht.build())


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for '{name}' not found exactly once"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    lib_path = ht.build(str(path), str(tmp_path / "libmutant.so"), extra_flags=("-w",))
    assert not _pins_in_child(lib_path), f"mutant '{name}' passed every pin"
