"""fbcc_solve_noalloc: the small-graph solve whose scratch is a static device array.

It exists for callers that cannot allocate device memory (a forbidding allocator
or memory pool, a plugin host that owns all device memory, a path that cannot take
an allocation's synchronisation). Its outputs must equal those of the ordinary
fbcc_solve entry point, exactly, on consecutive calls that reuse the same static
scratch, and graphs above its size limit must be refused.

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2301_01356_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu

KEYS = ("edge_bcc", "bcc_head", "is_ap", "is_bridge")


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _noalloc(torch, fbcc, g, off64):
    off = torch.from_numpy(g.offsets.astype(np.int64 if off64 else np.int32)).cuda()
    adj = torch.from_numpy(g.adj).cuda()
    eb = torch.full((max(g.nnz, 1),), -7, dtype=torch.int32, device="cuda")
    bh = torch.full((max(g.n, 1),), -7, dtype=torch.int32, device="cuda")
    ap = torch.full((max(g.n, 1),), 7, dtype=torch.uint8, device="cuda")
    br = torch.full((max(g.nnz, 1),), 7, dtype=torch.uint8, device="cuda")
    st = torch.zeros(5, dtype=torch.int64, device="cuda")   # one 40-byte fbcc_stats
    rc = fbcc.fbcc_solve_noalloc(off, adj, g.n, g.m, eb, bh, ap, br, st)
    assert rc == fbcc.FBCC_OK
    torch.cuda.synchronize()
    s = st.cpu().numpy()
    nb = int(s[0])
    return {"edge_bcc": eb[:g.nnz].cpu().numpy(), "bcc_head": bh[:nb].cpu().numpy(),
            "is_ap": ap[:g.n].cpu().numpy(), "is_bridge": br[:g.nnz].cpu().numpy(),
            "n_bcc": nb, "n_ap": int(s[1]), "n_bridge": int(s[2]), "n_cc": int(s[3]),
            "device_status": int(s[4] & 0xffffffff)}


def _existing(torch, fbcc, g, off64):
    solver = fbcc.Solver(g.n, g.nnz)
    off = torch.from_numpy(g.offsets.astype(np.int64 if off64 else np.int32)).cuda()
    adj = torch.from_numpy(g.adj).cuda()
    out = solver.solve(off, adj)
    solver.close()
    return out


def test_noalloc_matches_fbcc_solve_on_consecutive_calls(torch_cuda, oracle):
    """Both entry points run the same kernels, so each is also compared with the
    oracle directly: a fault in the shared path cannot hide behind agreement."""
    from paper_2301_01356_gb300 import fbcc
    graphs = [
        (gg.grid(100, 120, p=0.62, extra_frac=0.001, seed=5), False),   # many small BCCs and components
        (gg.uniform(30000, 100000, 4), True),                          # close to the size limit
        (gg.cycle_chain(2000, 12, 3, 300, 1), False),
    ]
    for g, off64 in graphs:                      # consecutive calls share the static scratch
        got = _noalloc(torch_cuda, fbcc, g, off64)
        exp = _existing(torch_cuda, fbcc, g, off64)
        ref = oracle.solve(g.offsets, g.adj)
        for k in KEYS:
            assert np.array_equal(got[k], exp[k]), f"{g.name}: {k}"
            assert np.array_equal(got[k], ref[k]), f"{g.name}: {k} differs from the oracle"
        for k in ("n_bcc", "n_ap", "n_bridge", "n_cc", "device_status"):
            assert got[k] == exp[k], f"{g.name}: {k}"
        for k in ("n_bcc", "n_ap", "n_bridge", "n_cc"):
            assert got[k] == ref[k], f"{g.name}: {k} differs from the oracle"
        assert got["device_status"] == 0
    # the same graph twice in a row gives the same answer again
    g, off64 = graphs[0]
    again = _noalloc(torch_cuda, fbcc, g, off64)
    exp = _existing(torch_cuda, fbcc, g, off64)
    for k in KEYS:
        assert np.array_equal(again[k], exp[k])


def test_noalloc_refuses_graphs_over_its_limit(torch_cuda):
    from paper_2301_01356_gb300 import fbcc
    g = gg.path(40000)                            # more than 32768 vertices
    off = torch_cuda.from_numpy(g.offsets).cuda()
    adj = torch_cuda.from_numpy(g.adj).cuda()
    buf = torch_cuda.empty(g.nnz + g.n, dtype=torch_cuda.int32, device="cuda")
    rc = fbcc.fbcc_solve_noalloc(off, adj, g.n, g.m, buf, buf, buf, buf, None)
    assert rc == fbcc.FBCC_E_WORKSPACE
