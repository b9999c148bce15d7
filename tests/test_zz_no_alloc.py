"""The growth entry point that allocates no device memory (for callers that
cannot call cudaMalloc while they run) gives the same communities as the
regular run and as the oracle, on calls in a row sharing its built-in scratch
array; sizes beyond its limits and bad seeds come back as errors.

Collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test.  It also passes alone in a fresh process."""
import os

import numpy as np
import pytest

from paper_1301_0955_gb300 import synth

pytestmark = pytest.mark.gpu

F_RTOL = 1e-12


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1301_0955_gb300 import build, mscd

    build.build()
    ctx = mscd.Context(0)
    yield torch, mscd, ctx
    ctx.close()


def outputs(torch, mscd, U, need):
    dev = torch.device("cuda:0")
    return dict(nodes=torch.full((max(need, 1),), -1, dtype=torch.int32, device=dev),
                offset=torch.zeros(U, dtype=torch.int64, device=dev),
                len=torch.zeros(U, dtype=torch.int32, device=dev),
                fitness=torch.zeros(U, dtype=torch.float64, device=dev),
                stats=torch.zeros((U, mscd.NSTATS), dtype=torch.int64, device=dev),
                status=torch.full((U,), 99, dtype=torch.int32, device=dev),
                hash=torch.zeros(U, dtype=torch.int64, device=dev))


def to_host(torch, out):
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_noalloc_matches_run_twice(env):
    torch, mscd, ctx = env
    g = synth.config_graph(0)  # 1,000-node planted partition
    gid = ctx.load_csr(g.n, g.row_ptr, g.col)
    alphas = mscd.scales_logspaced(0.5, 1.0, 4)
    seeds_h = np.arange(0, g.n, 3, dtype=np.int32)
    assert ctx.run(gid, alphas, seeds_h) == mscd.OK
    ref = [ctx.memberships(s) for s in range(len(alphas))]

    seeds = torch.from_numpy(seeds_h).to("cuda:0")
    U = len(alphas) * len(seeds_h)
    need = sum(int(r[0][-1]) for r in ref)
    for call in range(2):
        out = outputs(torch, mscd, U, need)
        rc, needed = ctx.grow_noalloc(gid, alphas, seeds, out)
        assert rc == mscd.OK, mscd.strerror(rc)
        assert needed == need
        h = to_host(torch, out)
        assert (h["status"] == 0).all()
        N = len(seeds_h)
        for s, (ptr, rnodes, rf, rst) in enumerate(ref):
            for j in range(N):
                u = s * N + j
                got = h["nodes"][h["offset"][u]:h["offset"][u] + h["len"][u]]
                assert np.array_equal(got, rnodes[ptr[j]:ptr[j + 1]]), (call, s, j)
            np.testing.assert_allclose(h["fitness"][s * N:(s + 1) * N], rf, rtol=F_RTOL, atol=0)
            assert np.array_equal(h["stats"][s * N:(s + 1) * N, :6], rst[:, :6])
    # a buffer that is too small is reported with the size it needs
    small = outputs(torch, mscd, U, need)
    small["nodes"] = torch.zeros(16, dtype=torch.int32, device="cuda:0")
    rc, needed = ctx.grow_noalloc(gid, alphas, seeds, small)
    assert rc == mscd.ESMALL and needed == need
    ctx.free_graph(gid)


def check_against_oracle(orc, h, G, alphas, seeds_h):
    N = len(seeds_h)
    for s, a in enumerate(alphas):
        rc, optr, onodes, of, ost = orc.run(G, [a], seeds_h, threads=os.cpu_count() or 1)
        assert rc == 0
        for j in range(N):
            u = s * N + j
            got = h["nodes"][h["offset"][u]:h["offset"][u] + h["len"][u]]
            assert np.array_equal(got, onodes[optr[j]:optr[j + 1]]), (s, int(seeds_h[j]))
        np.testing.assert_allclose(h["fitness"][s * N:(s + 1) * N], of, rtol=F_RTOL, atol=0)
        assert np.array_equal(h["stats"][s * N:(s + 1) * N, :6], ost[:, :6])


@pytest.mark.parametrize("which", ["lfr-100k", "weighted"])
def test_noalloc_against_oracle(orc, env, which):
    """Graphs above the 8,192-node slot cap (the 100,000-node workload graph:
    4,000 seeds x 4 scales) and a weighted graph (FP32 weights in [0.5, 2],
    exact fixed-point sums, all 3,000 seeds x 3 scales), two calls in a row,
    every unit against the oracle."""
    torch, mscd, ctx = env
    if which == "lfr-100k":
        g = synth.config_graph(1)
        seeds_h = np.sort(np.random.default_rng(8).choice(g.n, 4000, replace=False)).astype(np.int32)
        alphas = mscd.scales_logspaced(0.5, 1.0, 4)
    else:
        g = synth.hierarchical_lfr(3000, 20, 100, 2.5, 1.5, (20, 300), (0.3, 0.1), weights=(0.5, 2.0), seed=77)
        seeds_h = np.arange(g.n, dtype=np.int32)
        alphas = mscd.scales_logspaced(0.5, 1.0, 3)
    G = orc.Graph(g.n, g.row_ptr, g.col, g.w)
    assert G.status == 0
    gid = ctx.load_csr(g.n, g.row_ptr, g.col, g.w)
    seeds = torch.from_numpy(seeds_h).to("cuda:0")
    U = len(alphas) * len(seeds_h)
    # first call sizes the member-list buffer
    rc, need = ctx.grow_noalloc(gid, alphas, seeds, outputs(torch, mscd, U, 1))
    assert rc in (mscd.OK, mscd.ESMALL) and need > 0
    for call in range(2):
        out = outputs(torch, mscd, U, need)
        rc, needed = ctx.grow_noalloc(gid, alphas, seeds, out)
        assert rc == mscd.OK and needed == need, (call, mscd.strerror(rc))
        h = to_host(torch, out)
        assert (h["status"] == 0).all()
        check_against_oracle(orc, h, G, alphas, seeds_h)
    ctx.free_graph(gid)


def test_noalloc_limits_and_bad_seeds(env):
    """A unit that touches more nodes than the per-unit slot arena holds
    (8,192: the centre of a star of 10,000 leaves) returns MSCD_ERANGE; a
    seed outside the graph returns MSCD_EINVAL before anything runs; a call
    after either error still gives the right communities."""
    torch, mscd, ctx = env
    # a star of 10,000 leaves: the centre's unit touches every node
    n = 10_001
    u = np.zeros(n - 1, np.int64)
    v = np.arange(1, n, dtype=np.int64)
    rp, col, _ = synth.to_csr(n, u, v)
    gid = ctx.load_csr(n, rp, col)
    alphas = np.array([0.8])
    centre = torch.tensor([0], dtype=torch.int32, device="cuda:0")
    rc, _ = ctx.grow_noalloc(gid, alphas, centre, outputs(torch, mscd, 1, n))
    assert rc == mscd.ERANGE
    bad = torch.tensor([1, n], dtype=torch.int32, device="cuda:0")
    rc, _ = ctx.grow_noalloc(gid, alphas, bad, outputs(torch, mscd, 2, n))
    assert rc == mscd.EINVAL
    ctx.free_graph(gid)
    # the shared array after those errors: a regular call matches mscd_run
    g = synth.config_graph(0)
    gid = ctx.load_csr(g.n, g.row_ptr, g.col)
    seeds_h = np.arange(0, g.n, 7, dtype=np.int32)
    assert ctx.run(gid, alphas, seeds_h) == mscd.OK
    ptr, rnodes, rf, rst = ctx.memberships(0)
    out = outputs(torch, mscd, len(seeds_h), int(ptr[-1]))
    rc, need = ctx.grow_noalloc(gid, alphas, torch.from_numpy(seeds_h).to("cuda:0"), out)
    assert rc == mscd.OK and need == int(ptr[-1])
    h = to_host(torch, out)
    for j in range(len(seeds_h)):
        got = h["nodes"][h["offset"][j]:h["offset"][j] + h["len"][j]]
        assert np.array_equal(got, rnodes[ptr[j]:ptr[j + 1]]), j
    np.testing.assert_allclose(h["fitness"], rf, rtol=F_RTOL, atol=0)
    ctx.free_graph(gid)
