"""The Tarjan-Vishkin foil (fbcc_solve_tv): the explicit skeleton of section 3.2 and
the appendix's three rules, connected in place of Last-CC's implicit one. Every
output must equal the oracle's (and FAST-BCC's), on the same graphs the main path is
tested on."""
import numpy as np
import pytest

from paper_2301_01356_gb300 import graphgen as gg
from test_gpu_parity import assert_same, small_graphs, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_tv_small_and_tiny_graphs(torch_cuda, oracle):
    from paper_2301_01356_gb300 import fbcc
    s = fbcc.Solver(4000, 40000)
    rng = np.random.default_rng(17)
    tiny = []
    for _ in range(80):
        n = int(rng.integers(1, 12))
        e = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < 0.5]
        tiny.append(gg.from_edges(n, [a for a, _ in e], [b for _, b in e]))
    for g in small_graphs() + tiny:
        off, adj = to_dev(torch_cuda, g)
        assert_same(s.solve_tv(off, adj), oracle.solve(g.offsets, g.adj), f"tv {g.name} n={g.n}")
    s.close()


@pytest.mark.parametrize("family", ["uniform", "grid", "rmat", "chain", "knn", "union"])
def test_tv_families(torch_cuda, oracle, family):
    """Graphs spanning many tiles, in int64 and int32 offsets; the foil and the main
    path alternate on one workspace and agree."""
    from paper_2301_01356_gb300 import fbcc
    g = {
        "uniform": lambda: gg.uniform(30011, 70001, 5),
        "grid": lambda: gg.grid(211, 173, p=0.62, extra_frac=0.001, seed=9),
        "rmat": lambda: gg.rmat(15, 8, seed=4),
        "chain": lambda: gg.cycle_chain(60013, 40, 3, 3000, 11),
        "knn": lambda: gg.knn3(25000, 5, 2),
        "union": lambda: gg.disjoint_union(gg.from_edges(5, [], []), gg.grid(50, 61, p=0.7, seed=1),
                                           gg.path(4000), gg.uniform(3000, 9000, 3), gg.star(3000)),
    }[family]()
    e = oracle.solve(g.offsets, g.adj)
    s = fbcc.Solver(g.n, g.nnz)
    for off64 in (True, False):
        off = torch_cuda.from_numpy(g.offsets.astype(np.int64 if off64 else np.int32)).cuda()
        adj = torch_cuda.from_numpy(g.adj).cuda()
        assert_same(s.solve_tv(off, adj), e, f"tv {family} off64={off64}")
        assert_same(s.solve(off, adj), e, f"fbcc after tv {family}")
    s.close()


def test_tv_sampled_forest_and_scratch_checks(torch_cuda, oracle):
    """The foil on a forest from sampled connectivity; a scratch below
    fbcc_tv_scratch_bytes or unaligned is refused before anything is enqueued."""
    from paper_2301_01356_gb300 import fbcc
    g = gg.rmat(14, 16, seed=6)
    e = oracle.solve(g.offsets, g.adj)
    s = fbcc.Solver(g.n, g.nnz, cc_sample=1, lcc_sample=2)
    off, adj = to_dev(torch_cuda, g)
    assert_same(s.solve_tv(off, adj), e, "tv sampled forest")
    need = fbcc.fbcc_tv_scratch_bytes(g.n, g.nnz)
    assert need >= 12 * g.nnz + 16 * g.n
    small = torch_cuda.empty(need - 256, dtype=torch_cuda.uint8, device="cuda")
    with pytest.raises(fbcc.FbccError) as ex:
        s.solve_tv(off, adj, small)
    assert ex.value.status == fbcc.FBCC_E_WORKSPACE
    big = torch_cuda.empty(need + 512, dtype=torch_cuda.uint8, device="cuda")
    with pytest.raises(fbcc.FbccError) as ex:
        fbcc.fbcc_solve_tv(off, adj, g.n, g.nnz // 2, s.edge_bcc, s.bcc_head, s.is_ap, s.is_bridge, big[16:],
                           s.ws)
    assert ex.value.status == fbcc.FBCC_E_INVALID
    s.close()


@pytest.mark.slow
def test_tv_rmat24_full_size_equals_fbcc(torch_cuda):
    """At full size (537M skeleton vertices, 6.5 GB of scratch) the foil's outputs
    equal the main path's, which the full-size oracle test pins."""
    from paper_2301_01356_gb300 import fbcc
    g = gg.workload_rmat_24()
    off = torch_cuda.from_numpy(g.offsets).cuda()
    adj = torch_cuda.from_numpy(g.adj).cuda()
    s = fbcc.Solver(g.n, g.nnz)
    st = s.enqueue(off, adj)
    torch_cuda.cuda.synchronize()
    ref = {k: t.clone() for k, t in (("eb", s.edge_bcc), ("ap", s.is_ap), ("br", s.is_bridge), ("bh", s.bcc_head))}
    ref_st = st.as_dict()
    got = s.solve_tv(off, adj)
    nb = ref_st["n_bcc"]
    assert got["device_status"] == 0
    assert all(got[k] == ref_st[k] for k in ("n_bcc", "n_ap", "n_bridge", "n_cc"))
    assert np.array_equal(got["edge_bcc"], ref["eb"][:g.nnz].cpu().numpy())
    assert np.array_equal(got["is_ap"], ref["ap"][:g.n].cpu().numpy())
    assert np.array_equal(got["is_bridge"], ref["br"][:g.nnz].cpu().numpy())
    assert np.array_equal(got["bcc_head"], ref["bh"][:nb].cpu().numpy())
    s.close()
