"""GPU parity at the workloads' full graph sizes, in the launch configuration
the benchmark times, on samples the oracle grows one by one.

* lfr-1m-weighted (1,000,000 nodes, FP32 weights in [0.5, 2], 32 scales,
  every node a seed: 32,000,000 units in one run): 10,016 units stratified
  over the 32 scales against the oracle (memberships bit-exact, fitness within
  1e-12 relative, statistics exact); properties that hold at any size on
  every unit (each seed inside its community, lists sorted).
* lfr-100k (100,000 nodes, 20 scales, every node a seed): 10,000 units
  stratified over the scales; the whole dedup of the two finest scales
  (every community, its list, its fitness and every seed's community)
  against the oracle's dedup of all 200,000 units, and the NMI between them
  against the oracle's.
* the uneven batch (256 two-level graphs) at a quarter of its node counts:
  10,000 units stratified over the 16 scales, drawn over the whole union,
  against the oracle on each unit's own graph.
"""
import os

import numpy as np
import pytest

from paper_1301_0955_gb300 import synth

pytestmark = pytest.mark.gpu

F_RTOL = 1e-12
THREADS = os.cpu_count() or 1


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


def oracle_cover(ptr, nodes, first):
    """The oracle's deduplicated communities as (ptr, nodes), in its order."""
    lens = ptr[first + 1] - ptr[first]
    cp = np.zeros(len(first) + 1, np.int64)
    cp[1:] = np.cumsum(lens)
    cn = np.concatenate([nodes[ptr[u]:ptr[u + 1]] for u in first]).astype(np.int32) if len(first) else \
        np.zeros(0, np.int32)
    return cp, cn


def check_scale_sample(orc, ctx, G, alpha, s, seeds, pick):
    """Units `pick` (indices into seeds) of scale s against the oracle."""
    cptr, cnodes, cf, s2c = ctx.communities(s)
    f, st = ctx.unit_stats(s)
    rc, optr, onodes, of, ost = orc.run(G, [alpha], seeds[pick].astype(np.int32), threads=THREADS)
    assert rc == 0
    for t, j in enumerate(pick):
        c = s2c[j]
        got = cnodes[cptr[c]:cptr[c + 1]]
        want = onodes[optr[t]:optr[t + 1]]
        assert np.array_equal(got, want), (s, int(seeds[j]))
        assert f[j] == pytest.approx(of[t], rel=F_RTOL, abs=0), (s, int(seeds[j]))
        assert cf[c] == pytest.approx(of[t], rel=F_RTOL, abs=0)
        assert np.array_equal(st[j, :6], ost[t, :6]), (s, int(seeds[j]))


def check_seed_in_community(ctx, s, seeds):
    """Every unit of scale s: its community holds its seed, lists are sorted
    and unique (vectorised over the whole scale)."""
    cptr, cnodes, cf, s2c = ctx.communities(s)
    lens = np.diff(cptr)
    assert (lens >= 1).all()
    seg = np.repeat(np.arange(len(lens)), lens)
    inner = np.ones(len(cnodes), bool)
    inner[cptr[:-1]] = False
    assert (np.diff(cnodes)[inner[1:]] > 0).all()
    # key (community, node) is sorted because lists are sorted: binary search
    n = int(cnodes.max()) + 1 if len(cnodes) else 1
    n = max(n, int(seeds.max()) + 1)
    keys = seg.astype(np.int64) * n + cnodes
    q = s2c.astype(np.int64) * n + seeds
    pos = np.searchsorted(keys, q)
    assert (pos < len(keys)).all() and (keys[np.minimum(pos, len(keys) - 1)] == q).all()


def test_lfr1m_weighted_full_run(orc, ctx):
    """The benchmark's call: all 1,000,000 seeds x 32 scales in one run."""
    from paper_1301_0955_gb300 import mscd

    g = synth.config_graph(2)
    G = orc.Graph(g.n, g.row_ptr, g.col, g.w)
    assert G.status == 0
    alphas = mscd.scales_logspaced(0.5, 1.0, 32)
    gid = ctx.load_csr(g.n, g.row_ptr, g.col, g.w)
    info = ctx.graph_info(gid)
    assert info["unit_exp"] == G.info()["unit_exp"] and info["volume"] == G.info()["volume"]
    assert ctx.run(gid, alphas) == mscd.OK
    st = ctx.run_stats()
    assert st["units"] == 32_000_000 and st["undecided"] == 0
    seeds = np.arange(g.n, dtype=np.int32)
    rng = np.random.default_rng(2024)
    for s, a in enumerate(alphas):
        pick = np.sort(rng.choice(g.n, 313, replace=False))  # 32 x 313 = 10,016 units
        check_scale_sample(orc, ctx, G, a, s, seeds, pick)
        if s % 8 == 0 or s == len(alphas) - 1:
            check_seed_in_community(ctx, s, seeds)
    nmi, w3, w5 = ctx.stability()
    assert len(nmi) == 31 and np.all((nmi > -1e-12) & (nmi < 1 + 1e-12))
    ctx.free_graph(gid)


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
    rng = np.random.default_rng(42)
    for s, a in enumerate(alphas):
        check_scale_sample(orc, ctx, G, a, s, seeds, np.sort(rng.choice(g.n, 500, replace=False)))
        check_seed_in_community(ctx, s, seeds)
    # the whole dedup of the two finest scales and the NMI between them
    covers = []
    for s in (0, 1):
        rc, optr, onodes, of, ost = orc.run(G, [alphas[s]], None, threads=THREADS)
        assert rc == 0
        nc, u2c, first = orc.dedup(optr, onodes)
        cptr, cnodes, cf, s2c = ctx.communities(s)
        ocp, ocn = oracle_cover(optr, onodes, first)
        assert len(cptr) - 1 == nc
        assert np.array_equal(cptr, ocp) and np.array_equal(cnodes, ocn)
        assert np.array_equal(s2c, u2c)
        np.testing.assert_allclose(cf, of[first], rtol=F_RTOL, atol=0)
        covers.append((ocp, ocn))
    nmi, w3, w5 = ctx.stability()
    want = orc.nmi_indexed(g.n, *covers[0], *covers[1], threads=THREADS)
    assert nmi[0] == pytest.approx(want, abs=1e-12)
    ctx.free_graph(gid)


def test_uneven_batch_quarter_sampled(orc, ctx):
    """The uneven batch (256 two-level graphs, log-uniform sizes) at a quarter
    of its node counts (2.3M nodes, 16 scales, 37M units), batched as one
    disjoint union in the launch configuration of the benchmark: 625 units per
    scale drawn over the whole union, each against the oracle on its part's
    own graph."""
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
    total = int(off[-1])
    assert ctx.run(uid, alphas) == mscd.OK
    assert ctx.run_stats()["undecided"] == 0
    rng = np.random.default_rng(99)
    Gs = {}
    for s in range(16):
        cptr, cnodes, cf, s2c = ctx.communities(s)
        f, st = ctx.unit_stats(s)
        units = np.sort(rng.choice(total, 625, replace=False))
        part = np.searchsorted(off, units, side="right") - 1
        for p in np.unique(part):
            g = graphs[p]
            o = int(off[p])
            if p not in Gs:
                Gs[p] = orc.Graph(g.n, g.row_ptr, g.col)
            local = (units[part == p] - o).astype(np.int32)
            rc, optr, onodes, of, ost = orc.run(Gs[p], [alphas[s]], local, threads=THREADS)
            assert rc == 0
            for t, j in enumerate(local):
                u = o + int(j)
                c = s2c[u]
                got = cnodes[cptr[c]:cptr[c + 1]] - o
                assert np.array_equal(got, onodes[optr[t]:optr[t + 1]]), (s, int(p), int(j))
                assert f[u] == pytest.approx(of[t], rel=F_RTOL, abs=0)
                assert np.array_equal(st[u, :6], ost[t, :6]), (s, int(p), int(j))
    nmi, w3, w5 = ctx.stability(part=0)
    assert np.all((nmi > -1e-12) & (nmi < 1 + 1e-12))
    ctx.free_graph(uid)
