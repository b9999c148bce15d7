"""GPU: query serving with continuous batching.

A query's result must be the same alone and in any mix (bit-exact lists and
fitness), equal to what a run computes for the same seeds and scale, and
equal to the oracle on sampled seeds.
"""
import numpy as np
import pytest

from paper_1301_0955_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1301_0955_gb300 import build, mscd

    build.build()
    c = mscd.Context(0)
    graphs = [synth.config_graph(0), synth.hierarchical_lfr(20000, 20, 200, 2.5, 1.5, (20, 1000), (0.3, 0.2, 0.1),
                                                             seed=31)]
    gids = [c.load_csr(g.n, g.row_ptr, g.col) for g in graphs]
    yield c, graphs, gids
    c.close()


def query_lists(ptr, nodes):
    return [nodes[ptr[i]:ptr[i + 1]] for i in range(len(ptr) - 1)]


def run_reference_lists(ctx, gid, seeds, alpha):
    """The same units through mscd_run (oracle-checked elsewhere)."""
    assert ctx.run(gid, np.array([alpha]), np.ascontiguousarray(seeds, np.int32)) == 0
    ptr, nodes, f, _ = ctx.memberships(0, with_stats=False)
    return query_lists(ptr, nodes), f


def test_alone_equals_mixed_equals_run(orc, env):
    from paper_1301_0955_gb300 import mscd

    ctx, graphs, gids = env
    rng = np.random.default_rng(5)
    probe_seeds = np.sort(rng.choice(graphs[1].n, 300, replace=False)).astype(np.int32)
    probe_alpha = 0.7
    want_lists, want_f = run_reference_lists(ctx, gids[1], probe_seeds, probe_alpha)
    ctx.serve_start(workers=3, max_batch_units=4096)
    try:
        q = ctx.submit(gids[1], probe_seeds, probe_alpha)
        assert ctx.wait(q, 120) == mscd.Q_DONE
        ptr, nodes, f, t, rc = ctx.result(q, len(probe_seeds))
        assert rc == mscd.OK and t[2] >= t[1] >= 0
        alone = query_lists(ptr, nodes)
        assert all(np.array_equal(a, b) for a, b in zip(alone, want_lists))
        assert np.array_equal(f, want_f)
        # the same query inside a mix of 80 others on both graphs at several scales
        scales = mscd.scales_logspaced(0.5, 1.0, 16)
        mix = []
        for i in range(80):
            gi = int(rng.integers(0, 2))
            n_s = int(rng.integers(1, 600))
            seeds = rng.integers(0, graphs[gi].n, n_s).astype(np.int32)
            a = float(scales[int(rng.integers(0, 16))])
            mix.append((gi, seeds, a, ctx.submit(gids[gi], seeds, a)))
            if i == 40:
                q2 = ctx.submit(gids[1], probe_seeds, probe_alpha)
        for gi, seeds, a, qid in mix:
            assert ctx.wait(qid, 300) == mscd.Q_DONE
        assert ctx.wait(q2, 300) == mscd.Q_DONE
        ptr2, nodes2, f2, _, rc2 = ctx.result(q2, len(probe_seeds))
        assert rc2 == mscd.OK
        assert np.array_equal(ptr2, ptr) and np.array_equal(nodes2, nodes) and np.array_equal(f2, f)
        results = [(gi, seeds, a, ctx.result(qid, len(seeds))) for gi, seeds, a, qid in mix]
        st = ctx.serve_stats()
        assert st["queries_done"] == st["queries_submitted"] == 82 and st["queued"] == 0
        assert st["batches"] < 82  # queries were batched together
    finally:
        ctx.serve_stop()
    # every mixed query against a run of the same units; a few against the oracle
    for k, (gi, seeds, a, (ptr, nodes, f, t, rc)) in enumerate(results[:20]):
        assert rc == mscd.OK
        wl, wf = run_reference_lists(ctx, gids[gi], seeds, a)
        got = query_lists(ptr, nodes)
        assert all(np.array_equal(x, y) for x, y in zip(got, wl)), k
        assert np.array_equal(f, wf)
        if k < 4:
            g = graphs[gi]
            G = orc.Graph(g.n, g.row_ptr, g.col)
            pick = seeds[:5]
            orc_rc, optr, onodes, of, ost = orc.run(G, np.array([a]), pick, threads=4)
            assert orc_rc == 0
            for j in range(len(pick)):
                assert np.array_equal(got[j], onodes[optr[j]:optr[j + 1]])


def test_admission_by_memory_and_busy_graph(env):
    from paper_1301_0955_gb300 import mscd

    ctx, graphs, gids = env
    # a budget of one byte: every query is admitted alone
    ctx.serve_start(workers=4, max_batch_units=2048, memory_budget=1)
    try:
        rng = np.random.default_rng(9)
        qs = []
        for i in range(12):
            seeds = rng.integers(0, graphs[0].n, 200).astype(np.int32)
            qs.append((seeds, ctx.submit(gids[0], seeds, 0.8)))
        for seeds, q in qs:
            assert ctx.wait(q, 120) == mscd.Q_DONE
            ctx.result(q, len(seeds))
        st = ctx.serve_stats()
        assert st["batches"] == 12 and st["in_flight_bytes"] == 0
        # a graph with queued queries cannot be freed
        many = [ctx.submit(gids[1], rng.integers(0, graphs[1].n, 2048).astype(np.int32), 0.5) for _ in range(40)]
        with pytest.raises(mscd.MscdError) as e:
            ctx.free_graph(gids[1])
        assert e.value.rc == mscd.EBUSY
        for q in many:
            assert ctx.wait(q, 300) == mscd.Q_DONE
            ctx.result(q, 2048)
        with pytest.raises(mscd.MscdError) as e:
            ctx.submit(gids[0], np.zeros(4096, np.int32), 0.5)  # above max_batch_units
        assert e.value.rc == mscd.ERANGE
        with pytest.raises(mscd.MscdError) as e:
            ctx.submit(gids[0], np.array([graphs[0].n], np.int32), 0.5)  # seed out of range
        assert e.value.rc == mscd.EINVAL
    finally:
        ctx.serve_stop()


def _max_overlap(starts, ends):
    ev = sorted([(t, 1) for t in starts] + [(t, -1) for t in ends], key=lambda x: (x[0], x[1]))
    cur = best = 0
    for _, d in ev:
        cur += d
        best = max(best, cur)
    return best


def test_batches_overlap_on_device(env):
    """Continuous batching: under a mixed load the batches of different
    workers are on the GPU at the same time.  Each batch's device interval is
    timed by CUDA events on its worker's stream (first copy in to last copy
    out); at least two of them must overlap, and the server's own count of
    the most batches in flight at once agrees with a sweep over the
    intervals it reports."""
    from paper_1301_0955_gb300 import mscd

    ctx, graphs, gids = env
    ctx.serve_start(workers=4, max_batch_units=4096)
    try:
        rng = np.random.default_rng(17)
        scales = mscd.scales_logspaced(0.5, 1.0, 16)
        qs = []
        for i in range(48):
            gi = i % 2
            seeds = rng.integers(0, graphs[gi].n, int(rng.integers(512, 4097))).astype(np.int32)
            qs.append((seeds, ctx.submit(gids[gi], seeds, float(scales[int(rng.integers(0, 16))]))))
        for seeds, q in qs:
            assert ctx.wait(q, 300) == mscd.Q_DONE
            ctx.result(q, len(seeds))
        st = ctx.serve_stats()
        a, b = ctx.batch_intervals()
    finally:
        ctx.serve_stop()
    assert len(a) == st["batches"] >= 2
    assert (b >= a).all()
    assert st["max_concurrent_batches"] == _max_overlap(a, b)
    assert st["max_concurrent_batches"] >= 2 and st["overlap_us"] > 0


def test_serving_graph_full_size(orc):
    """One of the four 2,000,000-node serving graphs (mean degree 25, three
    levels): queries at 4 of the 16 scales, plus one of 4096 seeds, served
    concurrently; every returned list and fitness against the oracle."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import os

    from paper_1301_0955_gb300 import build, mscd

    build.build()
    ctx = mscd.Context(0)
    g = synth.config_graph(4)
    assert g.n == 2_000_000
    gid = ctx.load_csr(g.n, g.row_ptr, g.col)
    G = orc.Graph(g.n, g.row_ptr, g.col)
    scales = mscd.scales_logspaced(0.5, 1.0, 16)
    rng = np.random.default_rng(23)
    ctx.serve_start(workers=4, max_batch_units=65536)
    try:
        qs = []
        for s in (0, 5, 10, 15):
            for _ in range(2):
                seeds = np.sort(rng.choice(g.n, 160, replace=False)).astype(np.int32)
                qs.append((s, seeds, ctx.submit(gid, seeds, float(scales[s]))))
        big = rng.choice(g.n, 4096, replace=False).astype(np.int32)
        qs.append((8, big, ctx.submit(gid, big, float(scales[8]))))
        out = []
        for s, seeds, q in qs:
            assert ctx.wait(q, 600) == mscd.Q_DONE
            ptr, nodes, f, t, rc = ctx.result(q, len(seeds))
            assert rc == mscd.OK
            out.append((s, seeds, ptr, nodes, f))
    finally:
        ctx.serve_stop()
    for s, seeds, ptr, nodes, f in out:
        pick = np.arange(len(seeds)) if len(seeds) <= 160 else np.sort(rng.choice(len(seeds), 160, replace=False))
        rc, optr, onodes, of, ost = orc.run(G, [scales[s]], seeds[pick], threads=os.cpu_count() or 1)
        assert rc == 0
        for t, j in enumerate(pick):
            assert np.array_equal(nodes[ptr[j]:ptr[j + 1]], onodes[optr[t]:optr[t + 1]]), (s, int(seeds[j]))
            assert f[j] == pytest.approx(of[t], rel=1e-12, abs=0)
    ctx.free_graph(gid)
    ctx.close()
