"""GPU: the full method of Alg. 2 against the oracle.

Seeds, every scale's communities (lists, seeds, fitness), the iteration and
merge counts and the stability between scales must equal the oracle's:
integer results bit-exact, fitness within 1e-12 relative, NMI within 1e-12.
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


def compare(orc, ctx, g, alphas, rule=1, prio=None, init=None, eta=0.5, weighted=False):
    G = orc.Graph(g.n, g.row_ptr, g.col, g.w)
    assert G.status == 0
    gid = ctx.load_csr(g.n, g.row_ptr, g.col, g.w)
    rc = ctx.full_run(gid, alphas, prio=prio, init=init, seed_rule=rule, eta=eta)
    orc_rc, seeds, out = orc.full(G, alphas, rule, prio, init=init, eta=eta)
    assert rc == orc_rc == 0
    if init is None:
        assert np.array_equal(ctx.full_seeds(), seeds)
    covers = []
    for s, o in enumerate(out):
        r = ctx.full_scale(s)
        assert np.array_equal(r["ptr"], o["ptr"]), s
        assert np.array_equal(r["nodes"], o["nodes"]), s
        assert np.array_equal(r["seeds"], o["seeds"]), s
        np.testing.assert_allclose(r["f"], o["f"], rtol=F_RTOL, atol=0)
        assert r["iterations"] == o["iterations"] and r["merges"] == o["merges"], s
        covers.append((o["ptr"], o["nodes"]))
    for s in range(len(out) - 1):
        want = orc.nmi(g.n, *covers[s], *covers[s + 1])
        assert ctx.full_scale(s)["nmi_next"] == pytest.approx(want, abs=1e-12)
    ctx.free_graph(gid)
    return out


@pytest.mark.parametrize("rule", [1, 2])
def test_full_method_planted(orc, ctx, rule):
    g = synth.config_graph(0)
    prio = np.random.default_rng(rule).permutation(g.n).astype(np.int32)
    rc, alphas = orc.scales_logspaced(0.5, 1.0, 8)
    out = compare(orc, ctx, g, alphas, rule, prio)
    assert sum(o["merges"] for o in out) > 0


def test_full_method_lfr_and_weighted(orc, ctx):
    g = synth.hierarchical_lfr(5000, 20, 200, 2.5, 1.5, (20, 1000), (0.3, 0.1), seed=17)
    prio = np.random.default_rng(4).permutation(g.n).astype(np.int32)
    compare(orc, ctx, g, [1.0, 0.8, 0.65, 0.5], 1, prio)
    gw = synth.hierarchical_lfr(3000, 20, 150, 2.5, 1.5, (20, 500), (0.3, 0.2, 0.1), weights=(0.5, 2.0), seed=18)
    compare(orc, ctx, gw, [0.9, 0.6], 2, np.random.default_rng(5).permutation(gw.n).astype(np.int32))


def test_full_method_initial_communities_and_eta(orc, ctx):
    g = synth.config_graph(0)
    rng = np.random.default_rng(8)
    lists = [np.unique(rng.integers(0, g.n, int(rng.integers(2, 40)))).astype(np.int32) for _ in range(60)]
    init = (np.concatenate([[0], np.cumsum([len(x) for x in lists])]).astype(np.int64),
            np.concatenate(lists).astype(np.int32))
    compare(orc, ctx, g, [1.0, 0.7], init=init, eta=0.3)


@pytest.mark.parametrize("name", ["hypercube10", "torus30x30", "ring1000", "K20,30"])
@pytest.mark.parametrize("rule", [1, 2])
def test_full_method_symmetric_graphs(orc, ctx, name, rule):
    """Tie-heavy graphs: many overlapping equal-fitness communities meet the
    merge check (the 10-cube merges over seven iterations at the finest
    scale, the torus and the ring collapse into one community)."""
    from types import SimpleNamespace

    from test_gpu_parity import structured_graphs

    n, edges = structured_graphs()[name]
    e = np.asarray(edges, np.int64)
    lo, hi = np.minimum(e[:, 0], e[:, 1]), np.maximum(e[:, 0], e[:, 1])
    key = np.unique(lo * n + hi)
    rp, col, _ = synth.to_csr(n, key // n, key % n)
    g = SimpleNamespace(n=n, row_ptr=rp, col=col, w=None)
    prio = np.random.default_rng(2).permutation(n).astype(np.int32)
    compare(orc, ctx, g, [1.0, 0.75, 0.5], rule, prio)


@pytest.mark.parametrize("max_iters", [1, 3, 7])
def test_full_method_iteration_cap(orc, ctx, max_iters):
    """The check-and-merge loop of a scale stopped after max_iters iterations
    (the 10-cube needs 8 at its first scale): both sides report the time-out,
    keep that scale's communities as they stand and stop there."""
    from types import SimpleNamespace

    from paper_1301_0955_gb300 import mscd
    from test_gpu_parity import structured_graphs

    n, edges = structured_graphs()["hypercube10"]
    e = np.asarray(edges, np.int64)
    lo, hi = np.minimum(e[:, 0], e[:, 1]), np.maximum(e[:, 0], e[:, 1])
    key = np.unique(lo * n + hi)
    rp, col, _ = synth.to_csr(n, key // n, key % n)
    g = SimpleNamespace(n=n, row_ptr=rp, col=col, w=None)
    prio = np.random.default_rng(2).permutation(n).astype(np.int32)
    alphas = [1.0, 0.75, 0.5]
    G = orc.Graph(n, rp, col)
    orc_rc, seeds, out = orc.full(G, alphas, 1, prio, max_iters=max_iters)
    assert orc_rc == -8 and len(out) == 1
    gid = ctx.load_csr(n, rp, col)
    assert ctx.full_run(gid, alphas, prio=prio, seed_rule=1, max_iters=max_iters) == mscd.ETIMEOUT
    assert np.array_equal(ctx.full_seeds(), seeds)
    r, o = ctx.full_scale(0), out[0]
    assert np.array_equal(r["ptr"], o["ptr"]) and np.array_equal(r["nodes"], o["nodes"])
    assert np.array_equal(r["seeds"], o["seeds"])
    np.testing.assert_allclose(r["f"], o["f"], rtol=F_RTOL, atol=0)
    assert r["iterations"] == o["iterations"] == max_iters and r["merges"] == o["merges"]
    with pytest.raises(mscd.MscdError):
        ctx.full_scale(1)
    ctx.free_graph(gid)
