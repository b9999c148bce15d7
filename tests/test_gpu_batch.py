"""GPU: many independent graphs batched as one disjoint union.

Per part, a run on the union must give what the part gives alone: memberships,
statistics and dedup bit-exact (after the node-id shift), fitness within
1e-12 relative, stability bit-identical (the per-community terms are the same
and their sums exact); and a sample of units per part against the oracle on
the part's own graph.
"""
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


def weighted_copy(g, lo, hi, seed):
    """The same structure with FP32 weights uniform in [lo, hi)."""
    iu = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    up = iu < g.col
    w = np.random.default_rng(seed).uniform(lo, hi, int(up.sum())).astype(np.float32)
    rp, col, ww = synth.to_csr(g.n, iu[up], g.col[up], w)
    return synth.CSRGraph(g.n, rp, col, ww, g.labels, g.name)


def per_scale(ctx, S):
    return [ctx.memberships(s) for s in range(S)], [ctx.communities(s) for s in range(S)]


def check_union_matches_alone(orc, ctx, graphs, alphas, sample_per_part=6):
    from paper_1301_0955_gb300 import mscd

    S = len(alphas)
    gids = [ctx.load_csr(g.n, g.row_ptr, g.col, g.w) for g in graphs]
    uid = ctx.graph_union(gids)
    off = ctx.graph_parts(uid)
    assert np.array_equal(off, np.concatenate([[0], np.cumsum([g.n for g in graphs])]))
    info = ctx.graph_info(uid)
    assert info["n"] == off[-1] and info["nnz"] == sum(g.nnz for g in graphs)
    assert ctx.run(uid, alphas) == mscd.OK
    assert ctx.run_stats()["undecided"] == 0
    umem, ucom = per_scale(ctx, S)
    ustab = [ctx.stability(part=p) for p in range(len(graphs))]
    rng = np.random.default_rng(11)
    for p, (g, gid) in enumerate(zip(graphs, gids)):
        o = int(off[p])
        assert ctx.run(gid, alphas) == mscd.OK
        mem, com = per_scale(ctx, S)
        for s in range(S):
            uptr, unodes, uf, ust = umem[s]
            ptr, nodes, f, st = mem[s]
            seg = unodes[uptr[o]:uptr[o + g.n]] - o
            assert np.array_equal(np.diff(uptr[o:o + g.n + 1]), np.diff(ptr)), (p, s)
            assert np.array_equal(seg, nodes), (p, s)
            np.testing.assert_allclose(uf[o:o + g.n], f, rtol=F_RTOL, atol=0)
            assert np.array_equal(ust[o:o + g.n, :4], st[:, :4])
            # communities of part p: a contiguous block of the union's, same order
            cptr, cnodes, cf, s2c = com[s]
            gp, gn, gf, gs2c = ucom[s]
            first = int(gs2c[o])
            C = len(cptr) - 1
            assert np.array_equal(gs2c[o:o + g.n] - first, s2c)
            assert np.array_equal(gp[first:first + C + 1] - gp[first], cptr)
            assert np.array_equal(gn[gp[first]:gp[first + C]] - o, cnodes)
        nmi, w3, w5 = ctx.stability()
        unmi, uw3, uw5 = ustab[p]
        assert np.array_equal(nmi, unmi) and np.array_equal(w3, uw3) and np.array_equal(w5, uw5), p
        # oracle on the part's own graph, a few units per scale
        G = orc.Graph(g.n, g.row_ptr, g.col, g.w)
        assert G.status == 0
        pick = np.sort(rng.choice(g.n, min(sample_per_part, g.n), replace=False)).astype(np.int32)
        rc, optr, onodes, of, ost = orc.run(G, alphas, pick, threads=4)
        assert rc == 0
        for s in range(S):
            ptr, nodes, f, st = mem[s]
            for t, j in enumerate(pick):
                u = s * len(pick) + t
                assert np.array_equal(nodes[ptr[j]:ptr[j + 1]], onodes[optr[u]:optr[u + 1]]), (p, s, j)
                assert f[j] == pytest.approx(of[u], rel=F_RTOL, abs=0)
        # the part's stability against the oracle's NMI of its deduplicated covers
        covers = [(c[0], c[1]) for c in com]
        want = np.array([orc.nmi(g.n, *covers[s], *covers[s + 1]) for s in range(S - 1)])
        np.testing.assert_allclose(nmi, want, atol=NMI_ATOL, rtol=0)
    for gid in gids + [uid]:
        ctx.free_graph(gid)


def test_uneven_batch_small(orc, ctx):
    """Twelve two-level graphs of log-uniform size in [100, 3000], mean degree
    10-40, mixing 0.2-0.4 (the uneven batching recipe at small sizes)."""
    from paper_1301_0955_gb300 import mscd

    graphs = synth.uneven_batch(12, seed=4, n_range=(100, 3000))
    check_union_matches_alone(orc, ctx, graphs, mscd.scales_logspaced(0.5, 1.0, 6))


def test_union_weighted_units(orc, ctx):
    """Weighted parts whose exact weight units differ (weights in [0.5, 2),
    [1/256, 1/64) and [8, 32)): the union rescales them to one unit."""
    from paper_1301_0955_gb300 import mscd

    base = synth.uneven_batch(3, seed=5, n_range=(200, 800))
    graphs = [weighted_copy(base[0], 0.5, 2.0, 1), weighted_copy(base[1], 1 / 256, 1 / 64, 2),
              weighted_copy(base[2], 8.0, 32.0, 3)]
    check_union_matches_alone(orc, ctx, graphs, mscd.scales_logspaced(0.5, 1.0, 4))


def test_union_errors(ctx):
    from paper_1301_0955_gb300 import mscd

    g = synth.uneven_batch(2, seed=6, n_range=(100, 200))
    a = ctx.load_csr(g[0].n, g[0].row_ptr, g[0].col)
    w = weighted_copy(g[1], 0.5, 2.0, 4)
    b = ctx.load_csr(w.n, w.row_ptr, w.col, w.w)
    with pytest.raises(mscd.MscdError) as e:
        ctx.graph_union([a, b])  # weighted and unweighted mixed
    assert e.value.rc == mscd.EINVAL
    u = ctx.graph_union([a, a])  # the same graph twice is two parts
    with pytest.raises(mscd.MscdError):
        ctx.graph_union([u, a])  # a union is not a part
    assert len(ctx.graph_parts(u)) == 3 and len(ctx.graph_parts(a)) == 2
    for gid in (a, b, u):
        ctx.free_graph(gid)
