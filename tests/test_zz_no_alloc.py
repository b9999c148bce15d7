"""The growth entry point that allocates no device memory (for callers that
cannot call cudaMalloc while they run) gives the same communities as the
regular run, on two calls in a row sharing its built-in scratch array.

Collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test.  It also passes alone in a fresh process."""
import numpy as np
import pytest

from paper_1301_0955_gb300 import synth

pytestmark = pytest.mark.gpu

F_RTOL = 1e-12


def test_noalloc_matches_run_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1301_0955_gb300 import build, mscd

    build.build()
    ctx = mscd.Context(0)
    g = synth.config_graph(0)  # 1,000-node planted partition
    gid = ctx.load_csr(g.n, g.row_ptr, g.col)
    alphas = mscd.scales_logspaced(0.5, 1.0, 4)
    seeds_h = np.arange(0, g.n, 3, dtype=np.int32)
    assert ctx.run(gid, alphas, seeds_h) == mscd.OK
    ref = [ctx.memberships(s) for s in range(len(alphas))]

    dev = torch.device("cuda:0")
    seeds = torch.from_numpy(seeds_h).to(dev)
    U = len(alphas) * len(seeds_h)
    need = sum(int(r[0][-1]) for r in ref)
    for call in range(2):
        out = dict(nodes=torch.full((need,), -1, dtype=torch.int32, device=dev),
                   offset=torch.zeros(U, dtype=torch.int64, device=dev),
                   len=torch.zeros(U, dtype=torch.int32, device=dev),
                   fitness=torch.zeros(U, dtype=torch.float64, device=dev),
                   stats=torch.zeros((U, mscd.NSTATS), dtype=torch.int64, device=dev),
                   status=torch.full((U,), 99, dtype=torch.int32, device=dev),
                   hash=torch.zeros(U, dtype=torch.int64, device=dev))
        rc, needed = ctx.grow_noalloc(gid, alphas, seeds, out)
        assert rc == mscd.OK, mscd.strerror(rc)
        assert needed == need
        torch.cuda.synchronize()
        nodes = out["nodes"].cpu().numpy()
        off = out["offset"].cpu().numpy()
        ln = out["len"].cpu().numpy()
        f = out["fitness"].cpu().numpy()
        st = out["stats"].cpu().numpy()
        assert (out["status"].cpu().numpy() == 0).all()
        N = len(seeds_h)
        for s, (ptr, rnodes, rf, rst) in enumerate(ref):
            for j in range(N):
                u = s * N + j
                assert np.array_equal(nodes[off[u]:off[u] + ln[u]], rnodes[ptr[j]:ptr[j + 1]]), (call, s, j)
            np.testing.assert_allclose(f[s * N:(s + 1) * N], rf, rtol=F_RTOL, atol=0)
            assert np.array_equal(st[s * N:(s + 1) * N, :6], rst[:, :6])
    # a buffer that is too small is reported with the size it needs
    small = dict(out)
    small["nodes"] = torch.zeros(16, dtype=torch.int32, device=dev)
    rc, needed = ctx.grow_noalloc(gid, alphas, seeds, small)
    assert rc == mscd.ESMALL and needed == need
    ctx.close()
