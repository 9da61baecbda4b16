"""GPU parity: libfbcc (through its C ABI) against the Hopcroft-Tarjan oracle.

Every output must be bit-identical after the shared canonical numbering:
edge_bcc, bcc_head[0:n_bcc], is_ap, is_bridge and the four counts.
"""
import numpy as np
import pytest

from paper_2301_01356_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu

KEYS = ("edge_bcc", "bcc_head", "is_ap", "is_bridge", "n_bcc", "n_ap", "n_bridge", "n_cc")


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def solver(torch_cuda):
    from paper_2301_01356_gb300 import fbcc
    s = fbcc.Solver(1 << 17, 1 << 21)
    yield s
    s.close()


def to_dev(torch, g, off64=True):
    off = torch.from_numpy(g.offsets.astype(np.int64 if off64 else np.int32)).cuda()
    adj = torch.from_numpy(g.adj).cuda()
    return off, adj


def assert_same(got, exp, what=""):
    for k in KEYS:
        assert np.array_equal(np.asarray(got[k]), np.asarray(exp[k])), f"{what}: {k} differs"
    assert got["device_status"] == 0, f"{what}: device status {got['device_status']}"


def check(torch, solver, oracle, g, off64=True, what=None):
    off, adj = to_dev(torch, g, off64)
    got = solver.solve(off, adj)
    exp = oracle.solve(g.offsets, g.adj)
    assert_same(got, exp, what or g.name)
    return got


def wheel_behind_bridge(k):
    """0 - 1 a bridge, 1 the hub of a wheel on the cycle 2..k+1: the hub (degree k+1)
    heads one label, whose key a search of the hub's list finds."""
    u = [0] + [1] * k + list(range(2, k + 1)) + [k + 1]
    v = [1] + list(range(2, k + 2)) + list(range(3, k + 2)) + [2]
    return gg.from_edges(k + 2, u, v)


def windmill_behind_bridge(k):
    """0 - 1 a bridge, then k triangles sharing vertex 1: the hub (degree 2k+1) heads
    k labels, whose keys one scan of its list finds."""
    u, v = [0], [1]
    for i in range(k):
        a, b = 2 + 2 * i, 3 + 2 * i
        u += [1, 1, a]
        v += [a, b, b]
    return gg.from_edges(2 * k + 2, u, v)


def small_graphs():
    out = [gg.cycle(3), gg.cycle(50), gg.path(2), gg.path(300), gg.star(40), gg.complete(12),
           gg.grid(7, 9), gg.grid(6, 6, torus=True), gg.cycles_chain_exact([3, 4, 5, 6], 3),
           gg.from_edges(6, [], []), gg.from_edges(3, [1], [2]), gg.random_tree(500, 3),
           wheel_behind_bridge(200), windmill_behind_bridge(100)]
    for seed in range(12):
        rng = np.random.default_rng(seed)
        n = int(rng.integers(5, 400))
        m = int(rng.integers(0, min(n * (n - 1) // 2, 3 * n)))
        out.append(gg.uniform(n, m, seed))
    return out


def test_small_graphs(torch_cuda, solver, oracle):
    for g in small_graphs():
        for off64 in (True, False):
            check(torch_cuda, solver, oracle, g, off64)


def test_random_tiny_graphs(torch_cuda, solver, oracle):
    rng = np.random.default_rng(7)
    for it in range(150):
        n = int(rng.integers(1, 12))
        p = float(rng.uniform(0.1, 0.9))
        e = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < p]
        g = gg.from_edges(n, [a for a, _ in e], [b for _, b in e])
        check(torch_cuda, solver, oracle, g, bool(it & 1), f"tiny#{it}")


@pytest.mark.parametrize("family", ["uniform", "grid", "rmat", "chain", "knn", "union"])
def test_families_several_tiles(torch_cuda, solver, oracle, family):
    """Graphs spanning many arc tiles, RMQ tiles and rulers, with a ragged tail."""
    g = {
        "uniform": lambda: gg.uniform(30011, 70001, 5),
        "grid": lambda: gg.grid(211, 173, p=0.62, extra_frac=0.001, seed=9),
        "rmat": lambda: gg.rmat(15, 8, seed=4),
        "chain": lambda: gg.cycle_chain(60013, 40, 3, 3000, 11),
        "knn": lambda: gg.knn3(25000, 5, 2),
        "union": lambda: gg.disjoint_union(gg.from_edges(5, [], []), gg.grid(50, 61, p=0.7, seed=1),
                                           gg.path(4000), gg.uniform(3000, 9000, 3), gg.from_edges(7, [], [])),
    }[family]()
    assert g.n <= solver.n_max and g.nnz <= solver.nnz_max
    check(torch_cuda, solver, oracle, g, True)
    check(torch_cuda, solver, oracle, g, False)


def test_uniform_64k_workload(torch_cuda, solver, oracle):
    g = gg.workload_uniform_64k()
    got = check(torch_cuda, solver, oracle, g, False)
    assert got["n_bcc"] > 1 and got["n_bridge"] > 0 and got["n_ap"] > 0


def test_repeated_solves_and_configs(torch_cuda, oracle):
    """Graph replay, re-capture on new inputs, and every tuning knob give the same result."""
    from paper_2301_01356_gb300 import fbcc
    g1, g2 = gg.grid(100, 120, p=0.6, seed=3), gg.uniform(9000, 20000, 4)
    e1, e2 = oracle.solve(g1.offsets, g1.adj), oracle.solve(g2.offsets, g2.adj)
    for cfg in ({}, {"ruler_stride": 8}, {"ruler_stride": 256}, {"cc_sample": 2}, {"use_graph": -1},
                {"grid_ctas": 3}, {"chase_chains": 4}, {"chase_chains": 2}, {"cc_local": 1024},
                {"cc_local": 16384}, {"lcc_sample": 2}, {"lcc_sample": 1, "cc_sample": 2}, {"lcc_sample": 4}, {"rank_variant": 1},
                {"grid_ctas": -4}, {"cc_order": 1}, {"cc_order": 1, "cc_local": 1024, "rank_variant": 1},
                {"hub_deg": -1}, {"hub_deg": 32}, {"hub_deg": 32, "cc_sample": 2, "cc_order": 1},
                {"cc_ldd": 1}, {"cc_ldd": 4}, {"cc_ldd": 16, "cc_order": 1}, {"cc_ldd": 2, "hub_deg": 32}):
        s = fbcc.Solver(20000, 50000, **cfg)
        for _ in range(2):
            for g, e in ((g1, e1), (g2, e2), (g1, e1)):
                off, adj = to_dev(torch_cuda, g)
                assert_same(s.solve(off, adj), e, f"{cfg} {g.name}")
        s.close()


def test_sampled_cc_long_lists_outside_the_sampled_component(torch_cuda, oracle):
    """Sampled First-CC and Last-CC: vertices outside the sampled largest component go
    through their own lists, a lane per short list, the whole warp per list above 32
    arcs (a star's centre, a clique, R-MAT hubs) and the whole grid, in chunks, per
    list above 2048 arcs (a star of 5000 leaves, the two sides of K_{2,3000}) -- every
    output still equals the oracle, for every sample size."""
    from paper_2301_01356_gb300 import fbcc
    k2 = 3000                                  # K_{2,3000}: two lists of 3000 arcs, queued as chunks
    bip = gg.from_edges(k2 + 2, np.r_[np.zeros(k2, np.int64), np.ones(k2, np.int64)],
                        np.r_[np.arange(2, k2 + 2), np.arange(2, k2 + 2)])
    g = gg.disjoint_union(gg.uniform(20000, 60000, 3), gg.star(300), gg.complete(40), gg.path(50),
                          gg.from_edges(4, [], []), gg.rmat(12, 16, 0.57, 0.19, 0.19, 5), gg.star(5000), bip)
    e = oracle.solve(g.offsets, g.adj)
    for cfg in ({"cc_sample": 1}, {"cc_sample": 2}, {"cc_sample": 2, "lcc_sample": 2}, {"lcc_sample": 1},
                {"lcc_sample": 3}, {"lcc_sample": 4}, {"cc_sample": 1, "lcc_sample": 4}, {"cc_ldd": 2},
                {"cc_ldd": 8, "lcc_sample": 2}):
        s = fbcc.Solver(g.n, g.nnz, **cfg)
        off, adj = to_dev(torch_cuda, g)
        for _ in range(2):
            assert_same(s.solve(off, adj), e, f"{cfg}")
        s.close()


def test_sampling_vote_picks_the_pass(torch_cuda, oracle):
    """After sampling, a vote of arc sources decides the rest: a connected graph's
    sample wins it and the pass goes by vertex; 200 equal components leave no
    component with half the votes, and the tiled full pass runs instead. Both
    give the oracle's outputs."""
    from paper_2301_01356_gb300 import fbcc
    one = gg.uniform(30000, 150000, 8)
    many = gg.disjoint_union(*[gg.uniform(150, 600, 100 + i) for i in range(200)])
    for g, strong in ((one, 1), (many, 0)):
        e = oracle.solve(g.offsets, g.adj)
        s = fbcc.Solver(g.n, g.nnz, cc_sample=2, lcc_sample=4, use_graph=-1)
        off, adj = to_dev(torch_cuda, g)
        assert_same(s.solve(off, adj), e, g.name)
        votes = fbcc.fbcc_debug_read(s.ws, "sampled", 4)
        assert votes[1] == strong and votes[3] == strong, (g.name, votes)
        if strong:
            assert votes[0] >= 0
        s.close()


def test_ldd_forest_and_list_overflow(torch_cuda, oracle):
    """First-CC by LDD + union-find: the clusters' reaching edges plus the hooks over
    the edges between clusters span every component with its smallest vertex as root
    (the forest is checked in the phase tests), and the outputs equal the oracle's.
    With 1/beta = 64 over a third of the vertices wake in round 0, the clusters stay
    tiny, the list of edges between clusters outgrows its space, and the full hook
    pass takes over (flag 0); a sparse graph keeps the list (flag 1)."""
    from paper_2301_01356_gb300 import fbcc
    for g, cfg, held in ((gg.uniform(30000, 150000, 8), {"cc_ldd": 2}, 1),
                         (gg.grid(300, 280, p=0.62, extra_frac=0.001, seed=4), {"cc_ldd": 8}, 1),
                         (gg.uniform(200000, 4000000, 12), {"cc_ldd": 64}, 0)):
        e = oracle.solve(g.offsets, g.adj)
        s = fbcc.Solver(g.n, g.nnz, use_graph=-1, **cfg)
        off, adj = to_dev(torch_cuda, g)
        for _ in range(2):
            assert_same(s.solve(off, adj), e, f"{g.name} {cfg}")
        assert fbcc.fbcc_debug_read(s.ws, "sampled", 2)[1] == held, (g.name, cfg)
        s.close()


def test_local_first_cross_edge_list_and_overflow(torch_cuda, oracle):
    """Local-first First-CC: edges between ranges go through a gathered list; a dense
    graph whose list outgrows the space it borrows takes the full-scan fallback."""
    from paper_2301_01356_gb300 import fbcc
    for g in (gg.grid(300, 280, p=0.62, extra_frac=0.001, seed=4),    # list: a few edges per range boundary
              gg.uniform(3000, 200000, 5),                            # ~2/3 of 200k edges cross: overflow
              gg.uniform(2500, 2600, 6)):                             # sparse, many components
        e = oracle.solve(g.offsets, g.adj)
        s = fbcc.Solver(g.n, g.nnz, cc_local=1024)
        off, adj = to_dev(torch_cuda, g)
        for _ in range(2):
            assert_same(s.solve(off, adj), e, g.name)
        s.close()


def test_host_entry_point(torch_cuda, oracle):
    from paper_2301_01356_gb300 import fbcc
    g = gg.uniform(5000, 12000, 8)
    s = fbcc.Solver(g.n, g.nnz)
    eb = np.empty(g.nnz, np.int32)
    bh = np.empty(g.n, np.int32)
    ap = np.empty(g.n, np.uint8)
    br = np.empty(g.nnz, np.uint8)
    for off in (g.offsets, g.offsets.astype(np.int32)):
        st = fbcc.fbcc_solve_host(off, g.adj, eb, bh, ap, br, s.ws).as_dict()
        got = {"edge_bcc": eb, "bcc_head": bh[:st["n_bcc"]], "is_ap": ap, "is_bridge": br, **st}
        assert_same(got, oracle.solve(g.offsets, g.adj), "host")
    s.close()


def test_host_async_three_workspaces(torch_cuda, oracle):
    """fbcc_solve_host_async on three workspaces and three streams (the pipelined
    end-to-end form of the benchmark), several rounds, equals the oracle (bcc_head
    is compared over its first n_bcc entries)."""
    from paper_2301_01356_gb300 import fbcc
    torch = torch_cuda
    graphs = [gg.uniform(6000, 15000, 3), gg.grid(90, 80, p=0.6, seed=2), gg.grid(60, 70, p=0.7, seed=5)]
    exps = [oracle.solve(g.offsets, g.adj) for g in graphs]
    nmax = max(g.n for g in graphs)
    zmax = max(g.nnz for g in graphs)
    wss = [fbcc.fbcc_workspace_create(nmax, zmax) for _ in graphs]
    streams = [torch.cuda.Stream() for _ in graphs]
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    ins = [(pin(g.offsets), pin(g.adj)) for g in graphs]
    outs = [[pin(np.full(g.nnz, -1, np.int32)), pin(np.full(g.n, -1, np.int32)), pin(np.zeros(g.n, np.uint8)),
             pin(np.zeros(g.nnz, np.uint8))] for g in graphs]
    for rnd in range(3):
        for i in range(len(graphs)):
            fbcc.fbcc_solve_host_async(*ins[i], *outs[i], wss[i], streams[i])
        for st in streams:
            st.synchronize()
        for i, (g, e) in enumerate(zip(graphs, exps)):
            eb, bh, ap, br = outs[i]
            nb = e["n_bcc"]
            assert np.array_equal(eb, e["edge_bcc"]) and np.array_equal(ap, e["is_ap"])
            assert np.array_equal(br, e["is_bridge"]) and np.array_equal(bh[:nb], e["bcc_head"])
    for w in wss:
        fbcc.fbcc_workspace_destroy(w)


def test_validate(torch_cuda):
    from paper_2301_01356_gb300 import fbcc
    s = fbcc.Solver(100, 1000)
    g = gg.cycle(6)
    off, adj = to_dev(torch_cuda, g)
    assert fbcc.fbcc_validate(off, adj, g.n, g.m, s.ws) == fbcc.FBCC_OK
    bad = g.adj.copy()
    bad[0] = 0                                       # self-loop
    assert fbcc.fbcc_validate(off, torch_cuda.from_numpy(bad).cuda(), g.n, g.m, s.ws) == fbcc.FBCC_E_NOT_SIMPLE
    bad = g.adj.copy()
    bad[0], bad[1] = bad[1], bad[0]                  # unsorted
    assert fbcc.fbcc_validate(off, torch_cuda.from_numpy(bad).cuda(), g.n, g.m, s.ws) == fbcc.FBCC_E_NOT_SIMPLE
    bad = g.adj.copy()
    bad[0] = 2                                       # asymmetric
    assert fbcc.fbcc_validate(off, torch_cuda.from_numpy(bad).cuda(), g.n, g.m, s.ws) == fbcc.FBCC_E_NOT_SIMPLE
    bad = g.adj.copy()
    bad[0] = 99                                      # out of range
    assert fbcc.fbcc_validate(off, torch_cuda.from_numpy(bad).cuda(), g.n, g.m, s.ws) == fbcc.FBCC_E_INVALID
    off_bad = off.clone()
    off_bad[-1] += 2                                 # offsets[n] != 2m
    assert fbcc.fbcc_validate(off_bad, adj, g.n, g.m, s.ws) == fbcc.FBCC_E_INVALID
    # host-side argument checks
    with pytest.raises(fbcc.FbccError):
        fbcc.fbcc_solve(off, adj, g.n, 10**6, s.edge_bcc, s.bcc_head, s.is_ap, s.is_bridge, s.ws)
    s.close()


def _pack(graphs):
    vb = np.zeros(len(graphs) + 1, np.int64)
    ab = np.zeros(len(graphs) + 1, np.int64)
    for i, g in enumerate(graphs):
        vb[i + 1] = vb[i] + g.n
        ab[i + 1] = ab[i] + g.nnz
    loff = np.concatenate([g.offsets[:-1] for g in graphs]).astype(np.int32) if vb[-1] else np.zeros(0, np.int32)
    ladj = np.concatenate([g.adj for g in graphs]).astype(np.int32)
    return vb, ab, loff, ladj


def test_batch_matches_per_graph(torch_cuda, oracle):
    """Each graph's result in a batch equals its result alone (and the oracle's)."""
    from paper_2301_01356_gb300 import fbcc
    torch = torch_cuda
    rng = np.random.default_rng(3)
    graphs = []
    for i in range(37):
        kind = i % 4
        n = int(rng.integers(3, 3000))
        graphs.append([
            lambda: gg.uniform(n, min(n * (n - 1) // 2, int(n * rng.uniform(2, 6))), i),
            lambda: gg.grid(max(2, int(np.sqrt(n))), max(2, int(np.sqrt(n))), p=float(rng.uniform(0.55, 0.75)), seed=i),
            lambda: gg.cycle_chain(max(n, 10), int(rng.integers(2, 8)), 3, 500, i),
            lambda: gg.from_edges(n, [], []),
        ][kind]())
    vb, ab, loff, ladj = _pack(graphs)
    n_tot, z_tot = int(vb[-1]), int(ab[-1])
    s = fbcc.Solver(n_tot, z_tot)
    dev = lambda a: torch.from_numpy(a).cuda()
    stats = torch.zeros(len(graphs) * 5, dtype=torch.int64, device="cuda")  # 40-byte fbcc_stats
    for _ in range(2):
        fbcc.fbcc_solve_batch(dev(vb), dev(ab), vb, ab, dev(loff), dev(ladj), s.edge_bcc, s.bcc_head, s.is_ap,
                              s.is_bridge, stats, s.ws)
        torch.cuda.synchronize()
        eb, bh = s.edge_bcc[:z_tot].cpu().numpy(), s.bcc_head[:n_tot].cpu().numpy()
        ap, br = s.is_ap[:n_tot].cpu().numpy(), s.is_bridge[:z_tot].cpu().numpy()
        st = stats.cpu().numpy().reshape(len(graphs), 5)
        for i, g in enumerate(graphs):
            e = oracle.solve(g.offsets, g.adj)
            got = {"edge_bcc": eb[ab[i]:ab[i + 1]], "bcc_head": bh[vb[i]:vb[i] + st[i, 0]],
                   "is_ap": ap[vb[i]:vb[i + 1]], "is_bridge": br[ab[i]:ab[i + 1]], "n_bcc": st[i, 0],
                   "n_ap": st[i, 1], "n_bridge": st[i, 2], "n_cc": st[i, 3], "device_status": int(st[i, 4] & 0xffffffff)}
            assert_same(got, e, f"batch graph {i}")
    s.close()


def _tuned(name):
    from paper_2301_01356_gb300 import batch as B
    return dict(B.load_tuning().get("graphs", {}).get(name, {}).get("config", {}))


def test_grid_4096_full_size(torch_cuda, oracle):
    """The benchmark's large-diameter workload at full size, in the benchmark's
    tuned configuration and in the defaults, every output."""
    from paper_2301_01356_gb300 import fbcc
    g = gg.workload_grid_4096()
    exp = oracle.solve(g.offsets, g.adj)
    off, adj = to_dev(torch_cuda, g, off64=False)
    for cfg in (_tuned("grid4096"), {}, {**_tuned("grid4096"), "cc_order": 1}):
        s = fbcc.Solver(g.n, g.nnz, **cfg)
        assert_same(s.solve(off, adj), exp, f"grid 4096 {cfg}")
        s.close()


@pytest.mark.parametrize("max_chunk_arcs", [1 << 28, 150_000])
def test_bucketed_batch_runner(torch_cuda, oracle, max_chunk_arcs):
    """The config-4 recipe at small scale: every graph's result in the bucketed
    batch equals the oracle's and its result when solved alone; also with the
    buckets split into chunks (several solves per bucket)."""
    from paper_2301_01356_gb300 import batch as B, fbcc
    bt = gg.batch(96, 7, 200, 30000, families=("uniform", "grid", "chain", "knn"))
    runner = B.BatchRunner(bt, buckets=((0, 2000), (2000, 10000), (10000, 1 << 40)), tuning={},
                           configs=[{}, {"cc_local": 4096}, {"ruler_stride": 32, "cc_sample": 2}],
                           max_chunk_arcs=max_chunk_arcs)
    if max_chunk_arcs < (1 << 28):
        assert len(runner.buckets) > 3, "the small cap splits the buckets"
    runner.run()
    torch_cuda.cuda.synchronize()
    alone = fbcc.Solver(int(bt.sizes().max()), int(np.diff(bt.arc_base).max()))
    for g in range(bt.G):
        x = bt.graph(g)
        e = oracle.solve(x.offsets, x.adj)
        got = runner.result(g)
        assert_same(got, e, f"batched graph {g}")
        off, adj = to_dev(torch_cuda, x)
        solo = alone.solve(off, adj)
        for k in KEYS:
            assert np.array_equal(np.asarray(solo[k]), np.asarray(got[k])), f"graph {g}: {k} alone vs batch"
        if bt.truth_bcc[g] >= 0:
            assert got["n_bcc"] == bt.truth_bcc[g] and got["n_ap"] == bt.truth_ap[g]
    alone.close()
    runner.close()


def test_heavy_hub_forms_both_offset_widths(torch_cuda, oracle):
    """A graph whose largest degree reaches the heavy-hub threshold (4,096 arcs), so
    that the two full arc passes and the key searches take their L2-hinted forms:
    every output equals the oracle's with int32 and int64 offsets, in the defaults
    and in the tuned R-MAT configuration, and through the Tarjan-Vishkin foil."""
    from paper_2301_01356_gb300 import fbcc
    g = gg.rmat(16, 16, seed=3)
    assert int(np.diff(g.offsets).max()) >= 4096
    e = oracle.solve(g.offsets, g.adj)
    for cfg in ({}, _tuned("rmat24")):
        s = fbcc.Solver(g.n, g.nnz, **cfg)
        for off64 in (True, False):
            off, adj = to_dev(torch_cuda, g, off64)
            assert_same(s.solve(off, adj), e, f"{cfg} off64={off64}")
            assert_same(s.solve_tv(off, adj), e, f"tv {cfg} off64={off64}")
        s.close()
