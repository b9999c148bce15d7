"""GPU: the accuracy study in the shape of Table 1, at reduced size.

One (macro mu1, micro mu2) = (0.05, 0.2) setting of the table, on a
3,000-node two-level LFR-style graph (micro communities of 10-50 nodes
grouped 2-6 per macro community), 12 scales on [0.3, 1]: the independent
growth of every seed with dedup, and the full method (Alg. 2, seed rule 1).
Each scale's communities must equal the oracle's, and their NMI against
each planted level (computed on the GPU) the oracle's NMI; and the shape of
the table must show: the micro level found near alpha = 1, the macro level
at the small scales.
"""
import numpy as np
import pytest

from paper_1301_0955_gb300 import synth

pytestmark = pytest.mark.gpu


def planted_cover(labels):
    order = np.argsort(labels, kind="stable").astype(np.int32)
    counts = np.bincount(labels)
    ptr = np.concatenate([[0], np.cumsum(counts[counts > 0])]).astype(np.int64)
    return ptr, order


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1301_0955_gb300 import build, mscd

    build.build()
    g = synth.hierarchical_lfr(3000, 30, 100, 2.0, 1.0, (10, 50), (0.2, 0.05), group_range=(2, 6), seed=200,
                               name="acc-small")
    ctx = mscd.Context(0)
    gid = ctx.load_csr(g.n, g.row_ptr, g.col)
    yield mscd, ctx, gid, g
    ctx.close()


def nmi_rows(orc, ctx, g, covers):
    """[scale] -> (macro, micro) NMI, GPU and oracle side by side."""
    planted = [planted_cover(g.labels[1]), planted_cover(g.labels[0])]  # macro, micro
    rows = []
    for cp, cn in covers:
        gpu = [ctx.nmi_covers(g.n, (cp, cn), planted[l]) for l in (0, 1)]
        want = [orc.nmi(g.n, cp, cn, *planted[l]) for l in (0, 1)]
        np.testing.assert_allclose(gpu, want, atol=1e-12, rtol=0)
        rows.append(gpu)
    return np.array(rows)


def test_every_seed_with_dedup(orc, setup):
    mscd, ctx, gid, g = setup
    rc, alphas = orc.scales_logspaced(0.3, 1.0, 12)
    assert ctx.run(gid, alphas) == mscd.OK
    G = orc.Graph(g.n, g.row_ptr, g.col)
    rc, optr, onodes, of, ost = orc.run(G, alphas, None, threads=8)
    assert rc == 0
    N = g.n
    covers = []
    for s in range(len(alphas)):
        p = optr[s * N:(s + 1) * N + 1] - optr[s * N]
        nd = onodes[optr[s * N]:optr[(s + 1) * N]]
        cp, cn, u2c, first = orc.unique_communities(p, nd)
        gp, gn, gf, gs2c = ctx.communities(s)
        assert np.array_equal(gp, cp) and np.array_equal(gn, cn) and np.array_equal(gs2c, u2c), s
        covers.append((cp, cn))
    nm = nmi_rows(orc, ctx, g, covers)
    # the shape of Table 1: micro communities towards alpha = 1, macro ones
    # at the small scales
    assert nm[:3, 1].max() >= 0.9 and nm[-4:, 0].max() >= 0.9
    assert np.argmax(nm[:, 1]) < np.argmax(nm[:, 0])


def test_full_method_rule1(orc, setup):
    mscd, ctx, gid, g = setup
    rc, alphas = orc.scales_logspaced(0.3, 1.0, 12)
    prio = np.random.default_rng(300).permutation(g.n).astype(np.int32)
    assert ctx.full_run(gid, alphas, prio=prio, seed_rule=1) == mscd.OK
    G = orc.Graph(g.n, g.row_ptr, g.col)
    orc_rc, seeds, out = orc.full(G, alphas, 1, prio)
    assert orc_rc == 0
    covers = []
    for s, o in enumerate(out):
        r = ctx.full_scale(s)
        assert np.array_equal(r["ptr"], o["ptr"]) and np.array_equal(r["nodes"], o["nodes"]), s
        covers.append((o["ptr"], o["nodes"]))
    nm = nmi_rows(orc, ctx, g, covers)
    assert nm[:, 0].max() >= 0.9  # the macro level found by the merging method
    assert np.argmax(nm[:, 1]) < np.argmax(nm[:, 0])
