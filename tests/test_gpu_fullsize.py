"""GPU parity at the workloads' full graph sizes, on sampled units.

* lfr-100k (100,000 nodes, 20 scales, every node a seed): the whole run, in
  the configuration bench.py times, then a seeded sample of (scale, seed)
  units grown one by one by the oracle; memberships bit-exact, fitness within
  1e-12 relative, statistics exact.  Properties that hold at any size are
  checked on everything: seed in its community, sorted unique members,
  dedup consistent with the memberships, NMI in [0, 1].
* lfr-1m-weighted (1,000,000 nodes, FP32 weights in [0.5, 2], 32 scales): a
  seeded subset of seeds on the full graph (the whole 32M-unit set is the
  batching workload), sampled against the oracle the same way.
"""
import numpy as np
import pytest

from paper_1301_0955_gb300 import synth

pytestmark = pytest.mark.gpu

F_RTOL = 1e-12


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


def check_sample(orc, ctx, G, alphas, seeds, per_scale, rng):
    import os

    threads = os.cpu_count() or 1
    N = len(seeds)
    for s, a in enumerate(alphas):
        ptr, nodes, f, st = ctx.memberships(s)
        pick = np.sort(rng.choice(N, min(per_scale, N), replace=False))
        rc, optr, onodes, of, ost = orc.run(G, [a], seeds[pick].astype(np.int32), threads=threads)
        assert rc == 0
        for t, j in enumerate(pick):
            got = nodes[ptr[j]:ptr[j + 1]]
            want = onodes[optr[t]:optr[t + 1]]
            assert np.array_equal(got, want), (s, int(seeds[j]))
            assert f[j] == pytest.approx(of[t], rel=F_RTOL, abs=0)
            assert np.array_equal(st[j, :6], ost[t, :6]), (s, int(seeds[j]))


def check_properties(ctx, seeds, n_scales, n):
    for s in range(n_scales):
        ptr, nodes, f, st = ctx.memberships(s, with_stats=False)
        lens = np.diff(ptr)
        assert (lens >= 1).all()
        # each list strictly ascending and holding its seed
        starts = ptr[:-1]
        inner = np.ones(len(nodes), bool)
        inner[starts] = False
        assert (np.diff(nodes)[inner[1:]] > 0).all()
        seg = np.repeat(np.arange(len(seeds)), lens)
        has_seed = np.zeros(len(seeds), bool)
        np.logical_or.at(has_seed, seg, nodes == seeds[seg])
        assert has_seed.all()
        cptr, cnodes, cf, s2c = ctx.communities(s)
        assert len(cptr) - 1 <= len(seeds)
        # every unit's list equals its community's list (spot check)
        for j in np.random.default_rng(s).choice(len(seeds), 200, replace=False):
            c = s2c[j]
            assert np.array_equal(nodes[ptr[j]:ptr[j + 1]], cnodes[cptr[c]:cptr[c + 1]])
    nmi, w3, w5 = ctx.stability()
    assert np.all((nmi > -1e-12) & (nmi < 1 + 1e-12))


def test_lfr100k_full_run_sampled(orc, ctx):
    from paper_1301_0955_gb300 import mscd

    g = synth.config_graph(1)
    G = orc.Graph(g.n, g.row_ptr, g.col)
    alphas = mscd.scales_logspaced(0.5, 1.0, 20)
    gid = ctx.load_csr(g.n, g.row_ptr, g.col)
    assert ctx.run(gid, alphas) == mscd.OK
    st = ctx.run_stats()
    assert st["units"] == 2_000_000 and st["undecided"] == 0
    seeds = np.arange(g.n, dtype=np.int32)
    check_properties(ctx, seeds, len(alphas), g.n)
    check_sample(orc, ctx, G, alphas, seeds, 25, np.random.default_rng(42))
    ctx.free_graph(gid)


def test_lfr1m_weighted_sampled(orc, ctx):
    from paper_1301_0955_gb300 import mscd

    g = synth.config_graph(2)
    G = orc.Graph(g.n, g.row_ptr, g.col, g.w)
    assert G.status == 0
    alphas = mscd.scales_logspaced(0.5, 1.0, 32)
    gid = ctx.load_csr(g.n, g.row_ptr, g.col, g.w)
    info = ctx.graph_info(gid)
    assert info["unit_exp"] == G.info()["unit_exp"] and info["volume"] == G.info()["volume"]
    seeds = np.sort(np.random.default_rng(2).choice(g.n, 4000, replace=False)).astype(np.int32)
    assert ctx.run(gid, alphas, seeds) == mscd.OK
    assert ctx.run_stats()["undecided"] == 0
    check_properties(ctx, seeds, len(alphas), g.n)
    check_sample(orc, ctx, G, alphas, seeds, 8, np.random.default_rng(7))
    ctx.free_graph(gid)


def test_uneven_batch_quarter_sampled(orc, ctx):
    """The uneven batch (256 two-level graphs, log-uniform sizes) at a quarter
    of its node counts (2.3M nodes, 16 scales, 37M units), batched as one
    disjoint union in the launch configuration of the benchmark: a seeded
    sample of units of a seeded sample of parts against the oracle on the
    part's own graph."""
    import multiprocessing as mp

    from paper_1301_0955_gb300 import mscd

    specs = synth.uneven_batch_specs(256, seed=4, scale_nodes=0.25)
    with mp.get_context("spawn").Pool(min(16, len(specs))) as pool:
        graphs = pool.map(synth.graph_from_spec, specs, chunksize=1)
    alphas = mscd.scales_logspaced(0.5, 1.0, 16)
    gids = [ctx.load_csr(g.n, g.row_ptr, g.col) for g in graphs]
    uid = ctx.graph_union(gids)
    for gid in gids:
        ctx.free_graph(gid)
    off = ctx.graph_parts(uid)
    assert ctx.run(uid, alphas) == mscd.OK
    assert ctx.run_stats()["undecided"] == 0
    rng = np.random.default_rng(99)
    parts = np.sort(rng.choice(len(graphs), 12, replace=False))
    for s in range(0, 16, 5):
        for p in parts:
            g = graphs[p]
            o = int(off[p])
            G = orc.Graph(g.n, g.row_ptr, g.col)
            pick = np.sort(rng.choice(g.n, min(4, g.n), replace=False)).astype(np.int32)
            rc, optr, onodes, of, ost = orc.run(G, [alphas[s]], pick, threads=8)
            assert rc == 0
            for t, j in enumerate(pick):
                mem, f = ctx.membership(s, o + int(j))  # one unit at a time: the run holds 37M
                assert np.array_equal(mem - o, onodes[optr[t]:optr[t + 1]]), (s, p, int(j))
                assert f == pytest.approx(of[t], rel=F_RTOL, abs=0)
    nmi, w3, w5 = ctx.stability(part=int(parts[0]))
    assert np.all((nmi > -1e-12) & (nmi < 1 + 1e-12))
    ctx.free_graph(uid)
