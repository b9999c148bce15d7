"""Seeds of one job split across GPUs: the merge of the per-GPU shards of a
scale's deduplicated communities (mscd_merge_shards, host code of the CUDA
library) must give exactly the deduplication of the whole job.

The shards and the whole-job reference both come from the oracle (each
shard is the oracle's dedup of that shard's units), so these tests need no
GPU.  Two gloo ranks exercise the exchange and the sharded run's
orchestration on the CPU."""
import os
import socket

import numpy as np
import pytest

from paper_1301_0955_gb300 import synth


@pytest.fixture(scope="module")
def lib():
    from paper_1301_0955_gb300 import build, mscd

    build.build()
    return mscd.load()


def oracle_covers(orc, G, alphas, seeds):
    """Per scale: (comm_ptr, comm_nodes, fitness, seed2comm) of the oracle's
    run over `seeds`, deduplicated."""
    rc, ptr, nodes, f, _ = orc.run(G, alphas, seeds, threads=4)
    assert rc == 0
    N, out = len(seeds), []
    for s in range(len(alphas)):
        p = ptr[s * N:(s + 1) * N + 1] - ptr[s * N]
        nd = nodes[ptr[s * N]:ptr[(s + 1) * N]]
        cptr, cnodes, u2c, first = orc.unique_communities(p, nd)
        out.append((cptr, cnodes, f[s * N:(s + 1) * N][first], u2c))
    return out


def shard_of(orc, G, alphas, seeds, idx):
    return [dict(seed_index=idx, seed2comm=c[3], ptr=c[0], nodes=c[1], fitness=c[2])
            for c in oracle_covers(orc, G, alphas, seeds[idx])]


def assert_same(merged, want):
    for (p, n, f, s2c), (wp, wn, wf, ws) in zip(merged, want):
        assert np.array_equal(p, wp)
        assert np.array_equal(n, wn)
        assert np.array_equal(s2c, ws)
        assert np.array_equal(f, wf)


@pytest.fixture(scope="module")
def planted(orc):
    g = synth.config_graph(0)
    G = orc.Graph(g.n, g.row_ptr, g.col)
    rc, alphas = orc.scales_logspaced(0.5, 1.0, 4)
    seeds = np.arange(g.n, dtype=np.int32)
    return g, G, alphas, seeds, oracle_covers(orc, G, alphas, seeds)


@pytest.mark.parametrize("split", ["round-robin-2", "round-robin-3", "blocks-2", "random-4-with-empty"])
def test_merge_equals_whole_job(lib, orc, planted, split):
    from paper_1301_0955_gb300 import mscd

    g, G, alphas, seeds, want = planted
    N = len(seeds)
    if split.startswith("round-robin"):
        world = int(split[-1])
        parts = [mscd.shard_seeds(N, r, world) for r in range(world)]
    elif split == "blocks-2":
        parts = [np.arange(0, 425, dtype=np.int64), np.arange(425, N, dtype=np.int64)]  # inside a community
    else:
        perm = np.random.default_rng(3).permutation(N).astype(np.int64)
        cuts = [0, 50, 50, 620, N]  # shard 1 is empty, the others uneven and unsorted
        parts = [perm[cuts[i]:cuts[i + 1]] for i in range(4)]
    gathered = [shard_of(orc, G, alphas, seeds, idx) for idx in parts]
    merged = mscd.merge_gathered(gathered, N)
    assert_same(merged, want)
    # the shards really overlap: some list is found in more than one shard
    for s in range(len(alphas)):
        assert sum(len(sh[s]["ptr"]) - 1 for sh in gathered) > len(want[s][0]) - 1


def test_merge_with_repeated_seed_nodes(lib, orc, planted):
    """A node listed twice as a seed is two units; both ends of the split agree."""
    from paper_1301_0955_gb300 import mscd

    g, G, alphas, _, _ = planted
    seeds = np.random.default_rng(5).integers(0, g.n, 300).astype(np.int32)
    want = oracle_covers(orc, G, alphas, seeds)
    parts = [mscd.shard_seeds(len(seeds), r, 2) for r in range(2)]
    merged = mscd.merge_gathered([shard_of(orc, G, alphas, seeds, p) for p in parts], len(seeds))
    assert_same(merged, want)


def test_single_shard_is_identity(lib):
    from paper_1301_0955_gb300 import mscd

    sh = dict(seed_index=np.array([1, 0, 2]), seed2comm=np.array([1, 0, 1], np.int32),
              ptr=np.array([0, 2, 3]), nodes=np.array([4, 7, 9], np.int32), fitness=np.array([0.5, 0.25]))
    ptr, nodes, f, s2c = mscd.merge_shards([sh], 3)
    # seed index 0 (the shard's second seed) grew [4, 7], seed indices 1 and 2 grew [9]
    assert ptr.tolist() == [0, 2, 3] and nodes.tolist() == [4, 7, 9]
    assert f.tolist() == [0.5, 0.25] and s2c.tolist() == [0, 1, 1]


def test_order_by_smallest_seed_across_shards(lib):
    """Hand example: the list [3, 5] is grown by seed 4 in shard A and by seed 1
    in shard B; it must be community 1 (after seed 0's list) and carry shard
    B's fitness."""
    from paper_1301_0955_gb300 import mscd

    a = dict(seed_index=np.array([0, 4]), seed2comm=np.array([0, 1], np.int32), ptr=np.array([0, 1, 3]),
             nodes=np.array([0, 3, 5], np.int32), fitness=np.array([0.0, 2.0]))
    b = dict(seed_index=np.array([2, 1, 3]), seed2comm=np.array([0, 1, 0], np.int32), ptr=np.array([0, 2, 4]),
             nodes=np.array([2, 6, 3, 5], np.int32), fitness=np.array([1.0, 3.0]))
    ptr, nodes, f, s2c = mscd.merge_shards([a, b], 5)
    assert ptr.tolist() == [0, 1, 3, 5]
    assert nodes.tolist() == [0, 3, 5, 2, 6]
    assert f.tolist() == [0.0, 3.0, 1.0]
    assert s2c.tolist() == [0, 1, 2, 2, 1]


def test_bad_shards_are_rejected(lib):
    from paper_1301_0955_gb300 import mscd

    def shard(**kw):
        d = dict(seed_index=np.array([0, 1]), seed2comm=np.array([0, 0], np.int32), ptr=np.array([0, 2]),
                 nodes=np.array([1, 2], np.int32), fitness=np.array([1.0]))
        d.update(kw)
        return d

    ok = mscd.merge_shards([shard()], 2)
    assert ok[0].tolist() == [0, 2]
    bad = [
        ([shard(seed_index=np.array([0, 0]))], 2),                       # a seed index twice
        ([shard()], 3),                                                  # seed 2 missing
        ([shard(seed_index=np.array([0, 2]))], 2),                       # index out of range
        ([shard(seed2comm=np.array([0, 1], np.int32))], 2),              # community id out of range
        ([shard(nodes=np.array([2, 1], np.int32))], 2),                  # list not ascending
        ([shard(nodes=np.array([1, 1], np.int32))], 2),                  # repeated member
        ([shard(nodes=np.array([-1, 2], np.int32))], 2),                 # negative id
        ([shard(ptr=np.array([0, 2, 2]), fitness=np.array([1.0, 1.0]))], 2),  # empty list
        ([shard(ptr=np.array([0, 1, 2]), fitness=np.array([1.0, 1.0]))], 2),  # a list no seed grew
    ]
    for shards, n in bad:
        with pytest.raises(mscd.MscdError) as e:
            mscd.merge_shards(shards, n)
        assert e.value.rc == mscd.EINVAL


def test_sizes_query_and_small_buffers(lib):
    import ctypes as C

    from paper_1301_0955_gb300 import mscd

    si, s2c = np.array([0, 1], np.int64), np.array([0, 1], np.int32)
    ptr, nodes = np.array([0, 2, 3], np.int64), np.array([1, 2, 5], np.int32)
    arr = (mscd.mscd_cover_shard * 1)()
    arr[0] = mscd.mscd_cover_shard(2, si.ctypes.data_as(mscd.i64p), s2c.ctypes.data_as(mscd.i32p), 2,
                                   ptr.ctypes.data_as(mscd.i64p), nodes.ctypes.data_as(mscd.i32p), None)
    nc, nn = C.c_int64(), C.c_int64()
    rc = lib.mscd_merge_shards(arr, 1, 2, None, 0, None, 0, None, None, C.byref(nc), C.byref(nn))
    assert rc == mscd.ESMALL and (nc.value, nn.value) == (2, 3)
    out_p, out_n = np.zeros(3, np.int64), np.zeros(2, np.int32)  # nodes one short
    rc = lib.mscd_merge_shards(arr, 1, 2, out_p.ctypes.data_as(mscd.i64p), 3, out_n.ctypes.data_as(mscd.i32p), 2,
                               None, None, C.byref(nc), C.byref(nn))
    assert rc == mscd.ESMALL and out_p.tolist() == [0, 0, 0]  # nothing written
    # fitness asked for, but the shard has none
    f = np.zeros(2)
    out_n = np.zeros(3, np.int32)
    rc = lib.mscd_merge_shards(arr, 1, 2, out_p.ctypes.data_as(mscd.i64p), 3, out_n.ctypes.data_as(mscd.i32p), 3,
                               f.ctypes.data_as(mscd.f64p), None, C.byref(nc), C.byref(nn))
    assert rc == mscd.EINVAL
    # no shards and no seeds: an empty cover
    rc = lib.mscd_merge_shards(None, 0, 0, out_p.ctypes.data_as(mscd.i64p), 3, None, 0, None, None, C.byref(nc),
                               C.byref(nn))
    assert rc == mscd.OK and (nc.value, nn.value) == (0, 0) and out_p[0] == 0


def test_window_means_match_oracle(lib, orc):
    from paper_1301_0955_gb300 import mscd

    rng = np.random.default_rng(11)
    for S in range(1, 12):
        nmi = rng.random(S - 1)
        for p in (2, 3, 4, 5, 7):
            a = mscd.window_means(nmi, S, p)
            b = orc.window_means(nmi, S, p)
            assert np.array_equal(np.isnan(a), np.isnan(b))
            assert np.array_equal(a[~np.isnan(a)], b[~np.isnan(b)])
    # by hand: three scales, pairs (0,1) = 0.2 and (1,2) = 0.6, window of 3
    assert mscd.window_means([0.2, 0.6], 3, 3).tolist() == [0.2, pytest.approx(0.4), 0.6]
    with pytest.raises(mscd.MscdError):
        mscd.window_means([], 0, 3)
    with pytest.raises(mscd.MscdError):
        mscd.window_means([0.5], 2, 1)


# ---- two gloo ranks ---------------------------------------------------------

def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist

    import oracle as orc
    from paper_1301_0955_gb300 import mscd

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = synth.config_graph(0)
        G = orc.Graph(g.n, g.row_ptr, g.col)
        alphas = np.array([1.0, 0.75, 0.5])
        seeds = np.arange(0, g.n, 3, dtype=np.int32)

        def all_gather(obj):
            out = [None] * world
            dist.all_gather_object(out, obj)
            return out

        class OracleContext(mscd.Context):
            """The sharded run's orchestration with the oracle in place of the
            device calls (growth + dedup, NMI), so it runs on the CPU."""

            def __init__(self):
                self.h = None

            def __del__(self):
                pass

            def run(self, gid, alphas, seeds, stream=None):
                self.covers = oracle_covers(orc, G, alphas, seeds)
                return mscd.OK

            def communities(self, s):
                c = self.covers[s]
                return c[0], c[1], c[2], c[3]

            def graph_info(self, gid):
                return dict(n=g.n)

            def nmi_covers(self, n, a, b):
                return orc.nmi(n, a[0], a[1], b[0], b[1])

        res = OracleContext().run_sharded(0, alphas, seeds, rank, world, all_gather)
        want = oracle_covers(orc, G, alphas, seeds)
        assert_same(res["communities"], want)
        nmi = [orc.nmi(g.n, want[s][0], want[s][1], want[s + 1][0], want[s + 1][1]) for s in range(2)]
        assert np.array_equal(res["nmi"], np.array(nmi))
        assert np.array_equal(res["win3"], orc.window_means(np.array(nmi), 3, 3))
        q.put((rank, "ok"))
    except Exception as e:  # reported to the parent, which fails the test
        q.put((rank, repr(e)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sharded_run(lib, orc):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    assert out == [(0, "ok"), (1, "ok")]
