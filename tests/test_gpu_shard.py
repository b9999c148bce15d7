"""GPU: one job's seeds split into shards, each grown by its own mscd_run,
then merged by mscd_merge_shards: the merge must equal one run over all the
seeds (lists, seed map and order bit-exact, fitness within 1e-12 relative),
and the NMI of the merged scales the run's stability (1e-12 absolute).  The
shards run one after another on the one GPU; only the gather differs from a
job split across GPUs."""
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


def whole_run(ctx, gid, alphas, seeds):
    from paper_1301_0955_gb300 import mscd

    assert ctx.run(gid, alphas, seeds) == mscd.OK
    return [ctx.communities(s) for s in range(len(alphas))], ctx.stability()


def assert_merged(merged, want):
    for (p, n, f, s2c), (wp, wn, wf, ws) in zip(merged, want):
        assert np.array_equal(p, wp) and np.array_equal(n, wn) and np.array_equal(s2c, ws)
        np.testing.assert_allclose(f, wf, rtol=F_RTOL, atol=0)


@pytest.mark.parametrize("world", [2, 3])
def test_shards_merge_to_the_whole_run(ctx, world):
    from paper_1301_0955_gb300 import mscd

    g = synth.hierarchical_lfr(5000, 20, 200, 2.5, 1.5, (20, 1000), (0.3, 0.1), seed=17)
    gid = ctx.load_csr(g.n, g.row_ptr, g.col)
    alphas = mscd.scales_logspaced(0.5, 1.0, 6)
    seeds = np.arange(g.n, dtype=np.int32)
    gathered = []
    for r in range(world):
        idx = mscd.shard_seeds(len(seeds), r, world)
        assert ctx.run(gid, alphas, np.ascontiguousarray(seeds[idx])) == mscd.OK
        shard = []
        for s in range(len(alphas)):
            ptr, nodes, f, s2c = ctx.communities(s)
            shard.append(dict(seed_index=idx, seed2comm=s2c, ptr=ptr, nodes=nodes, fitness=f))
        gathered.append(shard)
    merged = mscd.merge_gathered(gathered, len(seeds))
    want, (nmi, w3, w5) = whole_run(ctx, gid, alphas, seeds)
    assert_merged(merged, want)
    got = [ctx.nmi_covers(g.n, merged[s][:2], merged[s + 1][:2]) for s in range(len(alphas) - 1)]
    np.testing.assert_allclose(got, nmi, rtol=0, atol=NMI_ATOL)
    np.testing.assert_allclose(mscd.window_means(np.array(got), len(alphas), 3), w3, rtol=0, atol=NMI_ATOL)
    ctx.free_graph(gid)


def test_run_sharded_one_process(ctx):
    """The sharded run with a gather of one process is the plain run."""
    from paper_1301_0955_gb300 import mscd

    g = synth.config_graph(0)
    gid = ctx.load_csr(g.n, g.row_ptr, g.col)
    alphas = mscd.scales_logspaced(0.5, 1.0, 8)
    seeds = np.arange(0, g.n, 2, dtype=np.int32)
    res = ctx.run_sharded(gid, alphas, seeds, 0, 1, lambda obj: [obj])
    assert res["status"] == mscd.OK
    want, (nmi, w3, w5) = whole_run(ctx, gid, alphas, seeds)
    assert_merged(res["communities"], want)
    np.testing.assert_allclose(res["nmi"], nmi, rtol=0, atol=NMI_ATOL)
    np.testing.assert_allclose(res["win3"], w3, rtol=0, atol=NMI_ATOL)
    np.testing.assert_allclose(res["win5"], w5, rtol=0, atol=NMI_ATOL)
    ctx.free_graph(gid)
