"""GPU: the autotuner picks schedules only; results never change."""
import numpy as np
import pytest

from paper_1301_0955_gb300 import synth

pytestmark = pytest.mark.gpu


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


def all_memberships(ctx, S):
    return [ctx.memberships(s, with_stats=False)[:2] for s in range(S)]


def test_autotune_keeps_results(ctx):
    from paper_1301_0955_gb300 import mscd

    g = synth.hierarchical_lfr(20000, 20, 200, 2.5, 1.5, (20, 1000), (0.3, 0.1), seed=21)
    alphas = mscd.scales_logspaced(0.5, 1.0, 6)
    gid = ctx.load_csr(g.n, g.row_ptr, g.col)
    assert ctx.run(gid, alphas) == mscd.OK
    before = all_memberships(ctx, len(alphas))
    nmi0 = ctx.stability()[0]
    p, ms = ctx.autotune(gid, alphas, n_sample=3000, apply=True)
    assert ms > 0
    assert p["smem_slots"] in (0, 256, 512, 1024, 2048)
    assert p["global_slots"] in (0, 4096, 8192, 16384)
    assert p["global_warps_per_sm"] in (8, 12, 16, 24, 32)
    with pytest.raises(mscd.MscdError) as e:
        ctx.stability()  # tuning clears the last run
    assert e.value.rc == mscd.ENORESULT
    assert ctx.run(gid, alphas) == mscd.OK
    after = all_memberships(ctx, len(alphas))
    for (p0, n0), (p1, n1) in zip(before, after):
        assert np.array_equal(p0, p1) and np.array_equal(n0, n1)
    assert np.array_equal(nmi0, ctx.stability()[0])
    # a cached answer for the same graph shape, without timing
    p2, ms2 = ctx.autotune(gid, alphas, n_sample=3000, apply=False, cached=True)
    assert p2 == p and ms2 == ms
    ctx.free_graph(gid)


def test_slot_class_too_large_is_rejected(ctx):
    from paper_1301_0955_gb300 import mscd

    c2 = mscd.Context(0, smem_slots=16384)
    g = synth.config_graph(0)
    gid = c2.load_csr(g.n, g.row_ptr, g.col)
    with pytest.raises(mscd.MscdError) as e:
        c2.run(gid, np.array([1.0]))
    assert e.value.rc == mscd.EINVAL
    c2.close()
