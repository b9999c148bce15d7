"""Pins of the oracle's full method (Alg. 2 with the growth of Alg. 3).

The seed step is pinned by the characterisation of the greedy choice in a
given order: the seeds are pairwise farther apart than the rule's distance,
and every other candidate has a seed within that distance that comes earlier
in the order (this set is unique).  The scale loop is pinned by what its
stopping condition implies: at the end of a scale no two communities overlap
by the merge ratio, and every community is a fixed point of one growth call;
and by recovery of the planted partition.
"""
import numpy as np
import pytest

from paper_1301_0955_gb300 import synth


def within(g, u, r):
    """Nodes at distance 1..r from u."""
    out = set(g.col[g.row_ptr[u]:g.row_ptr[u + 1]].tolist())
    if r == 2:
        for v in list(out):
            out |= set(g.col[g.row_ptr[v]:g.row_ptr[v + 1]].tolist())
    out.discard(u)
    return out


@pytest.mark.parametrize("rule", [1, 2])
def test_seed_rules_are_the_ordered_greedy_choice(orc, rule):
    for trial in range(6):
        g = synth.planted_partition(n_super=2, n_comm=3, comm_size=30, p_comm=0.2, p_super=0.05, p_out=0.01,
                                    seed=50 + trial)
        G = orc.Graph(g.n, g.row_ptr, g.col)
        prio = np.random.default_rng(trial).permutation(g.n).astype(np.int32)
        rc, seeds, out = orc.full(G, [1.0], rule, prio)
        assert rc == 0
        S = set(seeds.tolist())
        deg = np.diff(g.row_ptr)
        cand = {u for u in range(g.n) if deg[u] >= 2}
        assert S <= cand
        # seeds listed in the order they were chosen
        assert all(prio[a] < prio[b] for a, b in zip(seeds[:-1], seeds[1:]))
        for s in S:
            assert not (within(g, s, rule) & S)
        for u in cand - S:
            assert any(prio[s] < prio[u] for s in within(g, u, rule) & S)


def two_cliques_bridge(m=5):
    edges = [(i, j) for i in range(m) for j in range(i + 1, m)]
    edges += [(m + i, m + j) for i in range(m) for j in range(i + 1, m)]
    edges.append((m - 1, m))
    e = np.asarray(edges)
    return synth.to_csr(2 * m, e[:, 0], e[:, 1])


def test_two_cliques_hand_example(orc):
    """Two 5-cliques joined by one edge, seeds taken in id order: rule 1
    picks 0 (removing 1..4), then 5 (removing 4 and 6..9).  At alpha = 1
    each seed grows to its own clique (f = 20/21 for {0..4}); the cliques
    overlap in nothing, so nothing merges."""
    rp, col, _ = two_cliques_bridge()
    G = orc.Graph(10, rp, col)
    rc, seeds, out = orc.full(G, [1.0], 1, np.arange(10, dtype=np.int32))
    assert rc == 0 and seeds.tolist() == [0, 5]
    o = out[0]
    comms = [o["nodes"][o["ptr"][i]:o["ptr"][i + 1]].tolist() for i in range(len(o["ptr"]) - 1)]
    assert comms == [[0, 1, 2, 3, 4], [5, 6, 7, 8, 9]]
    assert o["f"][0] == pytest.approx(20 / 21, rel=1e-15)
    assert o["merges"] == 0


def test_overlapping_initial_communities_merge(orc):
    """Initial communities {0,1,2,3} and {2,3,4}: they share 2 of the
    smaller's 3 nodes (ratio 2/3 >= 0.5), so the pre-test flags both, the
    check pairs them and they merge into the first, which keeps its seed."""
    rp, col, _ = two_cliques_bridge()
    G = orc.Graph(10, rp, col)
    init = (np.array([0, 4, 7], np.int64), np.array([0, 1, 2, 3, 2, 3, 4], np.int32))
    rc, seeds, out = orc.full(G, [1.0], init=init)
    assert rc == 0
    o = out[0]
    assert o["merges"] >= 1
    assert len(o["ptr"]) - 1 == 1 and o["seeds"][0] == 0
    assert o["nodes"].tolist() == [0, 1, 2, 3, 4]


@pytest.mark.parametrize("rule", [1, 2])
def test_scale_end_invariants(orc, rule):
    g = synth.config_graph(0)
    G = orc.Graph(g.n, g.row_ptr, g.col)
    prio = np.random.default_rng(3).permutation(g.n).astype(np.int32)
    rc, alphas = orc.scales_logspaced(0.5, 1.0, 6)
    rc, seeds, out = orc.full(G, alphas, rule, prio, eta=0.5)
    assert rc == 0 and len(out) == 6
    for a, o in zip(alphas, out):
        C = [set(o["nodes"][o["ptr"][i]:o["ptr"][i + 1]].tolist()) for i in range(len(o["ptr"]) - 1)]
        for i in range(len(C)):
            assert o["seeds"][i] in C[i]
            for j in range(i + 1, len(C)):
                inter = len(C[i] & C[j])
                assert inter < 0.5 * min(len(C[i]), len(C[j]))
        # each community is a fixed point of growth from itself
        ptr = o["ptr"]
        rc2, p2, n2, f2, st2 = orc.run(G, [a], o["seeds"], init=(ptr, o["nodes"]))
        assert rc2 == 0 and np.array_equal(p2, ptr) and np.array_equal(n2, o["nodes"])
        np.testing.assert_allclose(f2, o["f"], rtol=1e-13)


def test_planted_recovery_full_method(orc):
    g = synth.config_graph(0)
    G = orc.Graph(g.n, g.row_ptr, g.col)
    prio = np.random.default_rng(1).permutation(g.n).astype(np.int32)
    rc, seeds, out = orc.full(G, [1.0, 0.5], 1, prio)
    assert rc == 0
    labels = g.labels
    for o, level in ((out[0], 0), (out[1], 1)):
        planted = [set(np.nonzero(labels[level] == c)[0].tolist()) for c in np.unique(labels[level])]
        C = [set(o["nodes"][o["ptr"][i]:o["ptr"][i + 1]].tolist()) for i in range(len(o["ptr"]) - 1)]
        best = [max(len(p & c) / len(p | c) for c in C) for p in planted]
        assert np.mean(best) >= 0.9, (level, np.mean(best), len(C))
