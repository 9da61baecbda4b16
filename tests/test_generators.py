"""The seeded input generators: valid simple symmetric CSR, deterministic,
thread-count independent, and the shapes the workloads promise."""
import os
import subprocess
import sys

import numpy as np

from paper_2301_01356_gb300 import graphgen as gg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_valid_csr(oracle):
    for g in (gg.uniform(1000, 3000, 1), gg.grid(30, 40, p=0.6, extra_frac=0.01, seed=2),
              gg.rmat(12, 8, seed=3), gg.cycle_chain(5000, 20, 3, 400, 4), gg.knn3(3000, 5, 5),
              gg.grid(9, 11, torus=True)):
        assert oracle.check_csr(g.offsets, g.adj) == 0, g.name


def test_deterministic_and_thread_independent():
    code = ("import sys; sys.path.insert(0, %r); from paper_2301_01356_gb300 import graphgen as gg; "
            "import hashlib; g = gg.rmat(14, 8, seed=9); h = gg.knn3(5000, 5, 3); "
            "print(hashlib.sha1(g.adj.tobytes() + g.offsets.tobytes() + h.adj.tobytes()).hexdigest())" % ROOT)
    outs = set()
    for threads in ("1", "3"):
        env = dict(os.environ, OMP_NUM_THREADS=threads)
        outs.add(subprocess.check_output([sys.executable, "-c", code], env=env, text=True).strip())
    assert len(outs) == 1


def test_workload_shapes():
    g = gg.workload_uniform_64k()
    assert g.n == 65536 and g.m == 196608
    g = gg.grid(64, 64, p=0.62, extra_frac=0.001, seed=2)
    kept_max = 2 * 64 * 63
    assert 0.5 * kept_max < g.m < 0.75 * kept_max
    src = np.repeat(np.arange(g.n), np.diff(g.offsets))
    dr = np.abs(src // 64 - g.adj // 64)
    dc = np.abs(src % 64 - g.adj % 64)
    assert np.all((dr + dc >= 1) & (dr + dc <= 8))
    g = gg.knn3(2000, 5, 1)
    assert np.all(np.diff(g.offsets) >= 5)      # every point keeps its own 5 neighbours


def test_chain_truth():
    g = gg.cycle_chain(1000, 10, 3, 50, 7)
    assert g.truth_bcc >= 10 and g.truth_ap >= 9
