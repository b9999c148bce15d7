"""GPU parity: the CUDA path through the C ABI against the oracle.

Bar: memberships, unit statistics, dedup and graph checks bit-exact (integer
work); fitness within 1e-12 relative (Eq. 1 evaluated in binary64 on the
device against binary128 in the oracle: both are a handful of correctly
rounded operations on the same exact integers, a few ulp apart); NMI within
1e-12 absolute (a sum of the same terms in a different order).
"""
import itertools

import numpy as np
import pytest

from paper_1301_0955_gb300 import synth

pytestmark = pytest.mark.gpu

F_RTOL = 1e-12
NMI_ATOL = 1e-12


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1301_0955_gb300 import build, mscd

    build.build()
    c = mscd.Context(0)
    yield c
    c.close()


def oracle_graph(orc, g):
    G = orc.Graph(g.n, g.row_ptr, g.col, g.w)
    assert G.status == 0
    return G


def compare_units(orc, ctx, G, alphas, seeds, threads=8, check_stats=True):
    """Run both sides on the same units; assert bit-exact memberships."""
    rc, optr, onodes, of, ost = orc.run(G, alphas, seeds, threads=threads)
    assert rc == 0
    N = len(seeds)
    for s in range(len(alphas)):
        ptr, nodes, f, st = ctx.memberships(s)
        sl = slice(s * N, (s + 1) * N)
        op = optr[s * N:(s + 1) * N + 1] - optr[s * N]
        on = onodes[optr[s * N]:optr[(s + 1) * N]]
        assert np.array_equal(ptr, op), "member list lengths differ at scale %d" % s
        assert np.array_equal(nodes, on), "members differ at scale %d" % s
        np.testing.assert_allclose(f, of[sl], rtol=F_RTOL, atol=0)
        if check_stats:
            # edges, adds, removes, rounds, K, V are trajectory facts
            assert np.array_equal(st[:, :6], ost[sl, :6]), "unit statistics differ at scale %d" % s
            assert not st[:, 7].any()
    return optr, onodes


def test_hand_traces_and_small_graphs(orc, ctx):
    import json
    import os

    here = os.path.dirname(os.path.abspath(__file__))
    for case in json.load(open(os.path.join(here, "golden", "hand_traces.json")))["cases"]:
        e = np.asarray(case["edges"])
        rp, col, _ = synth.to_csr(case["n"], e[:, 0], e[:, 1])
        gid = ctx.load_csr(case["n"], rp, col)
        ctx.run(gid, np.array([case["alpha"]]), np.array([case["seed"]], np.int32))
        mem, f = ctx.membership(0, 0)
        assert mem.tolist() == case["members"]
        assert f == pytest.approx(case["f"], rel=F_RTOL)
        ctx.free_graph(gid)


@pytest.mark.parametrize("weighted", [False, True])
def test_random_small_graphs(orc, ctx, weighted):
    rng = np.random.default_rng(7 + weighted)
    alphas = np.array([1.0, 0.5, 0.75, 0.625, 0.6180339887498949, 1.3, 0.9], np.float64)
    for trial in range(25):
        n = int(rng.integers(2, 40))
        p = float(rng.uniform(0.05, 0.6))
        iu, ju = np.triu_indices(n, 1)
        keep = rng.random(iu.size) < p
        w = rng.integers(1, 5, int(keep.sum())).astype(np.float32) if weighted else None
        rp, col, ww = synth.to_csr(n, iu[keep], ju[keep], w)
        G = orc.Graph(n, rp, col, ww)
        gid = ctx.load_csr(n, rp, col, ww)
        seeds = np.arange(n, dtype=np.int32)
        assert ctx.run(gid, alphas, seeds) == 0
        compare_units(orc, ctx, G, alphas, seeds, threads=2)
        ctx.free_graph(gid)


def test_graph_checks_match_oracle(orc, ctx):
    rp, col, _ = synth.to_csr(4, np.array([0, 1, 2]), np.array([1, 2, 3]))
    cases = [(rp, col, None)]
    c2 = col.copy(); c2[0] = 7; cases.append((rp, c2, None))
    bad = rp.copy(); bad[2] = 0; cases.append((bad, col, None))
    w = np.ones(len(col), np.float32); w[3] = -1.0; cases.append((rp, col, w))
    w = np.ones(len(col), np.float32); w[3] = np.inf; cases.append((rp, col, w))
    c3 = col.copy(); c3[1] = 1; cases.append((rp, c3, None))
    c4 = col.copy(); c4[1], c4[2] = c4[2], c4[1]; cases.append((rp, c4, None))
    c5 = col.copy(); c5[2] = 0; cases.append((rp, c5, None))
    c6 = col.copy(); c6[-1] = 1; cases.append((rp, c6, None))
    w = np.ones(len(col), np.float32); w[0] = 2.0; cases.append((rp, col, w))
    c7 = c6.copy(); c7[1] = 1; cases.append((rp, c7, None))
    w = np.array([2.0 ** 100, 2.0 ** 100, 2.0 ** -100, 2.0 ** -100], np.float32)
    rr, cc, _ = synth.to_csr(3, np.array([0, 1]), np.array([1, 2]))
    cases.append((rr, cc, w))
    for r, c, ww in cases:
        n = len(r) - 1
        want = orc.Graph(n, r, c, ww).status
        got, gid = ctx.try_load_csr(n, np.ascontiguousarray(r, np.int64), np.ascontiguousarray(c, np.int32), ww)
        assert got == want, (r, c, ww)
        if gid >= 0:
            ctx.free_graph(gid)


def test_weights_and_degrees_match_oracle(orc, ctx):
    rng = np.random.default_rng(3)
    for kind in range(4):
        n = 300
        iu, ju = np.triu_indices(n, 1)
        keep = rng.random(iu.size) < 0.05
        m = int(keep.sum())
        w = [rng.uniform(0.5, 2.0, m), np.exp(rng.uniform(-8, 8, m)), rng.integers(1, 9, m) * 4.0,
             rng.uniform(1e-40, 1e-38, m)][kind].astype(np.float32)
        rp, col, ww = synth.to_csr(n, iu[keep], ju[keep], w)
        G = orc.Graph(n, rp, col, ww)
        gid = ctx.load_csr(n, rp, col, ww)
        info = ctx.graph_info(gid)
        assert info["unit_exp"] == G.info()["unit_exp"]
        assert info["volume"] == G.info()["volume"]
        assert np.array_equal(ctx.graph_degrees(gid), G.degrees())
        ctx.free_graph(gid)


def test_planted_full_parity(orc, ctx):
    """All 8,000 units of the 1,000-node planted partition at 8 scales: memberships,
    statistics, dedup and stability against the oracle."""
    g = synth.config_graph(0)
    G = oracle_graph(orc, g)
    rc, alphas = orc.scales_logspaced(0.5, 1.0, 8)
    gid = ctx.load_csr(g.n, g.row_ptr, g.col)
    assert ctx.run(gid, alphas) == 0
    seeds = np.arange(g.n, dtype=np.int32)
    optr, onodes = compare_units(orc, ctx, G, alphas, seeds)
    N = g.n
    covers = []
    for s in range(8):
        p = optr[s * N:(s + 1) * N + 1] - optr[s * N]
        nd = onodes[optr[s * N]:optr[(s + 1) * N]]
        cptr, cnodes, u2c, first = orc.unique_communities(p, nd)
        gp, gn, gf, gs2c = ctx.communities(s)
        assert np.array_equal(gp, cptr) and np.array_equal(gn, cnodes)
        assert np.array_equal(gs2c, u2c)
        covers.append((cptr, cnodes))
    nmi, w3, w5 = ctx.stability()
    want = np.array([orc.nmi(N, *covers[s], *covers[s + 1]) for s in range(7)])
    np.testing.assert_allclose(nmi, want, atol=NMI_ATOL, rtol=0)
    np.testing.assert_allclose(w3, orc.window_means(want, 8, 3), atol=NMI_ATOL)
    np.testing.assert_allclose(w5, orc.window_means(want, 8, 5), atol=NMI_ATOL)
    st = ctx.run_stats()
    assert st["units"] == 8000 and st["undecided"] == 0
    ctx.free_graph(gid)


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("schedule,hybrid", [(0, False), (1, False), (0, True)])
def test_slot_class_escalation(orc, ctx, weighted, schedule, hybrid):
    """Tiny shared-memory classes force units through every class: two
    shared-memory classes, then global arenas of growing capacity, in the
    persistent schedule and in the plain one-launch-per-scale form, and with
    the first global class keeping its hash table in shared memory.  Results
    must not change."""
    from paper_1301_0955_gb300 import mscd

    c2 = mscd.Context(0, smem_slots=32, mid_slots=64, schedule=schedule, hash_smem_slots=512 if hybrid else 0)
    g = synth.config_graph(0)
    w = None
    if weighted:
        w = np.random.default_rng(4).uniform(0.5, 2.0, g.nnz // 2).astype(np.float32)
        iu = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
        up = iu < g.col
        rp, col, w = synth.to_csr(g.n, iu[up], g.col[up], w[: int(up.sum())])
        g = synth.CSRGraph(g.n, rp, col, w, g.labels, g.name)
    G = oracle_graph(orc, g)
    alphas = np.array([1.0, 0.6, 0.5])
    seeds = np.arange(0, g.n, 3, dtype=np.int32)
    gid = c2.load_csr(g.n, g.row_ptr, g.col, g.w)
    assert c2.run(gid, alphas, seeds) == 0
    st = c2.run_stats()
    assert st["overflow_units"] > 0
    classes = {(l["cap"], l["smem"]) for l in st["launches"]}
    assert (32, 1) in classes and (64, 1) in classes and any(cap > 64 and not sm for cap, sm in classes)
    if schedule == mscd.SCHED_PER_SCALE:
        assert st["grow_launches"] >= 3 * len(alphas)
    compare_units(orc, c2, G, alphas, seeds)
    c2.close()


def test_output_buffer_growth(orc, ctx):
    """Many units with large communities exceed the first output buffer."""
    g = synth.planted_partition(n_super=2, n_comm=2, comm_size=400, p_comm=0.2, p_super=0.05, p_out=0.01, seed=9)
    G = oracle_graph(orc, g)
    alphas = np.array([0.5, 0.55])
    seeds = np.repeat(np.arange(0, g.n, 5, dtype=np.int32), 4)  # repeated seeds are allowed
    gid = ctx.load_csr(g.n, g.row_ptr, g.col)
    assert ctx.run(gid, alphas, seeds) == 0
    compare_units(orc, ctx, G, alphas, seeds)
    ctx.free_graph(gid)


def test_edge_cases(orc, ctx):
    # empty graph with no seeds, isolated nodes, single node
    gid = ctx.load_csr(0, np.zeros(1, np.int64), np.zeros(0, np.int32))
    assert ctx.run(gid, np.array([0.7])) == 0
    assert ctx.run_stats()["units"] == 0
    ctx.free_graph(gid)
    gid = ctx.load_csr(3, np.zeros(4, np.int64), np.zeros(0, np.int32))
    ctx.run(gid, np.array([0.7, 1.0]))
    for s in range(2):
        for i in range(3):
            mem, f = ctx.membership(s, i)
            assert mem.tolist() == [i] and f == 0.0
    ptr, nodes, f, s2c = ctx.communities(0)
    assert len(ptr) == 4 and s2c.tolist() == [0, 1, 2]
    ctx.free_graph(gid)
    # bad arguments
    from paper_1301_0955_gb300 import mscd

    rp, col, _ = synth.to_csr(4, np.array([0, 1, 2]), np.array([1, 2, 3]))
    gid = ctx.load_csr(4, rp, col)
    for bad_alpha in (0.0, -1.0, np.nan, np.inf):
        with pytest.raises(mscd.MscdError):
            ctx.run(gid, np.array([bad_alpha]))
    with pytest.raises(mscd.MscdError):
        ctx.run(gid, np.array([0.5]), np.array([4], np.int32))
    ctx.free_graph(gid)


def test_device_pointer_inputs(orc, ctx):
    torch = pytest.importorskip("torch")
    g = synth.config_graph(0)
    G = oracle_graph(orc, g)
    dev = torch.device("cuda:0")
    rp = torch.from_numpy(g.row_ptr).to(dev)
    col = torch.from_numpy(g.col).to(dev)
    gid = ctx.load_csr(g.n, rp, col)
    alphas = torch.tensor([0.9, 0.55], dtype=torch.float64, device=dev)
    seeds = torch.arange(0, g.n, 7, dtype=torch.int32, device=dev)
    stream = torch.cuda.Stream()
    assert ctx.run(gid, alphas, seeds, stream=stream) == 0
    compare_units(orc, ctx, G, alphas.cpu().numpy(), seeds.cpu().numpy())
    ctx.free_graph(gid)


def test_unit_order_independent(orc, ctx):
    """Shuffled seed order gives the same community per seed (units are independent)."""
    g = synth.config_graph(0)
    gid = ctx.load_csr(g.n, g.row_ptr, g.col)
    alphas = np.array([0.8, 0.52])
    seeds = np.arange(g.n, dtype=np.int32)
    ctx.run(gid, alphas, seeds)
    a = [ctx.memberships(s) for s in range(2)]
    perm = np.random.default_rng(0).permutation(g.n).astype(np.int32)
    ctx.run(gid, alphas, perm)
    for s in range(2):
        ptr, nodes, f, st = ctx.memberships(s)
        p0, n0, f0, st0 = a[s]
        for j in range(0, g.n, 37):
            i = perm[j]
            assert np.array_equal(nodes[ptr[j]:ptr[j + 1]], n0[p0[i]:p0[i + 1]])
    ctx.free_graph(gid)


@pytest.mark.parametrize("small_class", [False, True])
def test_initial_members_parity(orc, ctx, small_class):
    """Growth from seeds plus initial members (repeats, the seed itself and
    empty lists included) against the oracle; with a 32-slot first class the
    larger initial sets overflow and are grown again in the next classes."""
    from paper_1301_0955_gb300 import mscd

    c = mscd.Context(0, smem_slots=32) if small_class else ctx
    g = synth.config_graph(0)
    G = oracle_graph(orc, g)
    rng = np.random.default_rng(13 + small_class)
    seeds = np.sort(rng.choice(g.n, 200, replace=False)).astype(np.int32)
    lists = []
    for i, sd in enumerate(seeds):
        kind = i % 4
        if kind == 0:
            lists.append(np.zeros(0, np.int32))
        elif kind == 1:  # a neighbourhood around the seed, with the seed and a repeat
            nb = g.col[g.row_ptr[sd]:g.row_ptr[sd + 1]]
            lists.append(np.concatenate([nb[:5], [sd], nb[:1]]).astype(np.int32))
        else:  # random nodes anywhere
            lists.append(rng.integers(0, g.n, int(rng.integers(1, 60 if kind == 2 else 300))).astype(np.int32))
    iptr = np.concatenate([[0], np.cumsum([len(x) for x in lists])]).astype(np.int64)
    inodes = np.concatenate(lists).astype(np.int32)
    alphas = np.array([1.0, 0.7, 0.5])
    gid = c.load_csr(g.n, g.row_ptr, g.col)
    assert c.run_init(gid, alphas, seeds, iptr, inodes) == 0
    rc, optr, onodes, of, ost = orc.run(G, alphas, seeds, threads=8, init=(iptr, inodes))
    assert rc == 0
    N = len(seeds)
    for s in range(len(alphas)):
        ptr, nodes, f, st = c.memberships(s)
        op = optr[s * N:(s + 1) * N + 1] - optr[s * N]
        assert np.array_equal(ptr, op) and np.array_equal(nodes, onodes[optr[s * N]:optr[(s + 1) * N]])
        np.testing.assert_allclose(f, of[s * N:(s + 1) * N], rtol=F_RTOL, atol=0)
        assert np.array_equal(st[:, :6], ost[s * N:(s + 1) * N, :6])
    if small_class:
        assert c.run_stats()["overflow_units"] > 0
    with pytest.raises(mscd.MscdError) as e:  # a member id out of range
        bad = inodes.copy()
        bad[-1] = g.n
        c.run_init(gid, alphas, seeds, iptr, bad)
    assert e.value.rc == mscd.EINVAL
    c.free_graph(gid)
    if small_class:
        c.close()


@pytest.mark.parametrize("cap", [1, 2])
def test_round_cap_parity(orc, cap):
    """The repetition cap: both sides stop every unit after the same number of
    rounds, report the time-out, and leave the same (partial) communities."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1301_0955_gb300 import mscd

    g = synth.hierarchical_lfr(5000, 20, 200, 2.5, 1.5, (20, 1000), (0.3, 0.1), seed=17)
    G = oracle_graph(orc, g)
    alphas = np.array([1.0, 0.7, 0.5, 0.35])
    seeds = np.arange(0, g.n, 2, dtype=np.int32)
    rc_o, optr, onodes, of, ost = orc.run(G, alphas, seeds, threads=8, max_rounds=cap)
    assert rc_o == -8  # some unit needs more rounds than the cap
    c = mscd.Context(0, max_rounds=cap)
    try:
        gid = c.load_csr(g.n, g.row_ptr, g.col)
        assert c.run(gid, alphas, seeds) == mscd.ETIMEOUT
        N = len(seeds)
        for s in range(len(alphas)):
            ptr, nodes, f, st = c.memberships(s)
            assert np.array_equal(ptr, optr[s * N:(s + 1) * N + 1] - optr[s * N])
            assert np.array_equal(nodes, onodes[optr[s * N]:optr[(s + 1) * N]])
            np.testing.assert_allclose(f, of[s * N:(s + 1) * N], rtol=F_RTOL, atol=0)
            assert np.array_equal(st[:, :6], ost[s * N:(s + 1) * N, :6])
    finally:
        c.close()


def structured_graphs():
    """Symmetric graphs where ranking and fitness ties are the rule (the
    smaller-id rule and the strict tests decide most steps; the torus,
    hypercube and complete bipartite graph send thousands of decisions to the
    exact tie test), and a ring and a wheel whose units grow to every node."""
    out = {}
    n = 1000
    out["ring1000"] = (n, [(i, (i + 1) % n) for i in range(n)])
    r_, c_ = 30, 30
    out["torus30x30"] = (r_ * c_, [(r * c_ + c, r * c_ + (c + 1) % c_) for r in range(r_) for c in range(c_)]
                         + [(r * c_ + c, ((r + 1) % r_) * c_ + c) for r in range(r_) for c in range(c_)])
    out["hypercube10"] = (1024, [(i, i ^ (1 << b)) for i in range(1024) for b in range(10) if i < i ^ (1 << b)])
    out["K20,30"] = (50, [(i, 20 + j) for i in range(20) for j in range(30)])
    out["K60"] = (60, list(itertools.combinations(range(60), 2)))
    cav = [(10 * c + i, 10 * c + j) for c in range(50) for i, j in itertools.combinations(range(10), 2)]
    out["caveman50x10"] = (500, cav + [(10 * c + 9, (10 * c + 10) % 500) for c in range(50)])
    out["wheel500"] = (501, [(0, i) for i in range(1, 501)] + [(i, i % 500 + 1) for i in range(1, 501)])
    return out


@pytest.mark.parametrize("name", sorted(structured_graphs()))
def test_structured_tie_graphs(orc, ctx, name):
    n, edges = structured_graphs()[name]
    e = np.asarray(edges, np.int64)
    lo, hi = np.minimum(e[:, 0], e[:, 1]), np.maximum(e[:, 0], e[:, 1])
    key = np.unique(lo * n + hi)
    rp, col, _ = synth.to_csr(n, key // n, key % n)
    G = orc.Graph(n, rp, col)
    assert G.status == 0
    gid = ctx.load_csr(n, rp, col)
    alphas = np.array([1.0, 0.5, 0.75, 0.3, 1.5])
    seeds = np.arange(n, dtype=np.int32)
    assert ctx.run(gid, alphas, seeds) == 0
    compare_units(orc, ctx, G, alphas, seeds, threads=8)
    ctx.free_graph(gid)
    # the same graph with weights from {1/2, 1, 2}: weighted ties stay frequent
    w = np.random.default_rng(len(name)).choice(np.array([0.5, 1.0, 2.0], np.float32), len(key))
    rp, col, ww = synth.to_csr(n, key // n, key % n, w)
    G = orc.Graph(n, rp, col, ww)
    assert G.status == 0
    gid = ctx.load_csr(n, rp, col, ww)
    assert ctx.run(gid, alphas, seeds) == 0
    compare_units(orc, ctx, G, alphas, seeds, threads=8)
    ctx.free_graph(gid)


def test_hub_node_wide_slots(orc, ctx):
    """A hub of degree 70,000 (degrees beyond 16 bits: 32-bit slot values) and
    units touching more than 32,768 nodes (32-bit hash buckets), against the
    oracle."""
    rng = np.random.default_rng(17)
    n = 70_001
    leaves = np.arange(1, n, dtype=np.int64)
    # the hub (node 0) joined to every leaf, leaves joined in small rings of 5
    ring = leaves.reshape(-1, 5)
    ea = [np.zeros(n - 1, np.int64), ring.ravel()]
    eb = [leaves, np.roll(ring, -1, axis=1).ravel()]
    extra = rng.integers(1, n, (2000, 2))
    extra = extra[extra[:, 0] != extra[:, 1]]
    ea.append(extra[:, 0])
    eb.append(extra[:, 1])
    a = np.concatenate(ea)
    b = np.concatenate(eb)
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    key = np.unique(lo * n + hi)
    rp, col, _ = synth.to_csr(n, key // n, key % n)
    G = orc.Graph(n, rp, col)
    assert G.status == 0
    gid = ctx.load_csr(n, rp, col)
    assert ctx.graph_info(gid)["n"] == n
    seeds = np.array([0, 1, 2, 3, 5000, 69999], np.int32)
    alphas = np.array([1.0, 0.5, 0.3])
    assert ctx.run(gid, alphas, seeds) == 0
    compare_units(orc, ctx, G, alphas, seeds, threads=4)
    st = ctx.run_stats()
    assert any(l["cap"] > 32768 for l in st["launches"])
    ctx.free_graph(gid)
