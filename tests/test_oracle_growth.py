"""Pins for the oracle's community growth (Alg. 1 repeated as in Alg. 2, Eq. 1-2).

What fixes the expected values here, independently of the oracle:
* hand traces of Alg. 1 on small graphs (tests/golden/hand_traces.json);
* closed forms of Eq. 1 on cliques and stars;
* brute force over every subset of <= 12-node graphs, with f compared exactly
  (big integers for dyadic alpha, 300-bit mpmath otherwise): the result is a
  local optimum for single additions and single non-seed removals, and equals
  the global optimum where the seed's component is a clique;
* closed forms on barbells (two cliques joined by one edge): the growth
  stops at the bridge where the closed-form add test of the partner fails;
* invariants: the seed is always a member; results do not depend on the
  number of threads;
* planted recovery on the 1,000-node planted partition: the micro and macro
  communities appear at different scales.
"""
import itertools
import json
import math
import os
import random

import numpy as np
import pytest

from paper_1301_0955_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def graph_from_edges(orc, n, edges, w=None):
    e = np.asarray(edges, np.int64).reshape(-1, 2)
    rp, col, ww = synth.to_csr(n, e[:, 0], e[:, 1], None if w is None else np.asarray(w, np.float32))
    g = orc.Graph(n, rp, col, ww)
    assert g.status == 0
    return g, rp, col


@pytest.mark.parametrize("case", json.load(open(os.path.join(HERE, "golden", "hand_traces.json")))["cases"],
                         ids=lambda c: c["name"])
def test_hand_traces(orc, case):
    g, _, _ = graph_from_edges(orc, case["n"], case["edges"])
    mem, f, st, rc = orc.grow(g, case["seed"], case["alpha"])
    assert rc == 0
    assert mem.tolist() == case["members"]
    assert st["K"] == case["K"] and st["V"] == case["V"]
    assert f == pytest.approx(case["f"], rel=1e-15)
    for key in ("edges_scanned", "adds", "removes", "rounds"):
        assert st[key] == case[key], key


@pytest.mark.parametrize("m", [2, 3, 5, 8, 13])
@pytest.mark.parametrize("alpha", [0.5, 0.7, 1.0, 1.3])
def test_clique_closed_form(orc, m, alpha):
    """A clique with no outside edges is grown whole: K = V = m(m-1), f = (m(m-1))^(1-alpha)."""
    edges = list(itertools.combinations(range(m), 2))
    g, _, _ = graph_from_edges(orc, m, edges)
    for seed in range(m):
        mem, f, st, rc = orc.grow(g, seed, alpha)
        assert rc == 0 and mem.tolist() == list(range(m))
        assert st["K"] == m * (m - 1) == st["V"]
        assert f == pytest.approx((m * (m - 1)) ** (1 - alpha), rel=1e-15)


@pytest.mark.parametrize("m", [1, 2, 6, 20])
@pytest.mark.parametrize("alpha", [0.5, 0.8, 1.0])
def test_star_closed_form(orc, m, alpha):
    """From the centre of a star with m leaves and alpha <= 1 every leaf joins
    ((1+1/j) > (1+1/(m+j))^alpha), f = 2m / (2m)^alpha."""
    edges = [(0, i) for i in range(1, m + 1)]
    g, _, _ = graph_from_edges(orc, m + 1, edges)
    mem, f, st, rc = orc.grow(g, 0, alpha)
    assert mem.tolist() == list(range(m + 1))
    assert f == pytest.approx((2 * m) ** (1 - alpha), rel=1e-15)


def test_isolated_seed(orc):
    g, _, _ = graph_from_edges(orc, 3, [(1, 2)])
    mem, f, st, rc = orc.grow(g, 0, 0.7)
    assert rc == 0 and mem.tolist() == [0] and f == 0.0 and st["V"] == 0


def test_weighted_closed_form(orc):
    """Weighted clique with no outside edges at alpha = 1: f = 1 in any unit."""
    edges = list(itertools.combinations(range(5), 2))
    rng = np.random.default_rng(0)
    w = rng.uniform(0.5, 2.0, len(edges)).astype(np.float32)
    g, _, _ = graph_from_edges(orc, 5, edges, w)
    mem, f, st, rc = orc.grow(g, 2, 1.0)
    assert mem.tolist() == [0, 1, 2, 3, 4] and f == pytest.approx(1.0, rel=1e-15)


# ---------------------------------------------------------------- brute force

DYADIC = {1.0: (1, 0), 0.5: (1, 1), 0.75: (3, 2), 0.625: (5, 3)}


def f_greater(K1, V1, K2, V2, alpha):
    """Exact test K1/V1^alpha > K2/V2^alpha (f = 0 when K = 0)."""
    if K1 == 0:
        return False
    if K2 == 0:
        return True
    if alpha in DYADIC:
        P, s = DYADIC[alpha]
        return K1 ** (2 ** s) * V2 ** P > K2 ** (2 ** s) * V1 ** P
    mpmath = pytest.importorskip("mpmath")
    with mpmath.workprec(300):
        d = mpmath.log(K1) - mpmath.log(K2) - mpmath.mpf(alpha) * (mpmath.log(V1) - mpmath.log(V2))
        return d > mpmath.mpf(2) ** -250


def kv(adj_w, k, members):
    K = sum(adj_w[u].get(v, 0) for u in members for v in members if u != v)
    V = sum(k[u] for u in members)
    return K, V


def random_small_graph(rng, n, p, weighted=False):
    edges = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < p]
    w = [rng.randint(1, 4) for _ in edges] if weighted else None
    return edges, w


@pytest.mark.parametrize("alpha", [1.0, 0.5, 0.75, 0.625, 0.6180339887498949])
def test_bruteforce_local_optimum(orc, alpha):
    rng = random.Random(int(alpha * 1000))
    checked = 0
    for it in range(60):
        n = rng.randint(4, 12)
        weighted = it % 3 == 2
        edges, w = random_small_graph(rng, n, rng.uniform(0.2, 0.6), weighted)
        if not edges:
            continue
        g, rp, col = graph_from_edges(orc, n, edges, w)
        adj = [dict() for _ in range(n)]
        for idx, (a, b) in enumerate(edges):
            ww = 1 if w is None else w[idx]
            adj[a][b] = ww
            adj[b][a] = ww
        k = [sum(adj[u].values()) for u in range(n)]
        for seed in range(n):
            mem, f, st, rc = orc.grow(g, seed, alpha)
            assert rc == 0
            c = set(mem.tolist())
            assert seed in c
            K, V = kv(adj, k, c)
            unit = 2.0 ** g.info()["unit_exp"]
            assert (K, V) == (st["K"] * unit, st["V"] * unit)
            if K:
                assert f == pytest.approx(K / V ** alpha, rel=1e-14)
            for u in range(n):
                if u in c:
                    if u == seed:
                        continue
                    K2, V2 = kv(adj, k, c - {u})
                else:
                    K2, V2 = kv(adj, k, c | {u})
                assert not f_greater(K2, V2, K, V, alpha), (edges, seed, alpha, sorted(c), u)
            # global optimum over subsets containing the seed bounds the result
            others = [u for u in range(n) if u != seed]
            if n <= 10:
                best = (0, 1)
                for r in range(len(others) + 1):
                    for sub in itertools.combinations(others, r):
                        K2, V2 = kv(adj, k, set(sub) | {seed})
                        if f_greater(K2, V2, *best, alpha):
                            best = (K2, V2)
                assert not f_greater(K, V, *best, alpha)
            checked += 1
    assert checked > 200


@pytest.mark.parametrize("alpha", [1.0, 0.5, 0.75, 0.6180339887498949])
def test_bruteforce_local_optimum_float_weights(orc, alpha):
    """FP32 weights drawn uniformly from [0.5, 2] (the weighted workload's
    distribution).  Every float is a dyadic rational, so scaling by the largest
    denominator, computed here from the floats with Fraction, gives exact
    integer weights; K and V must equal the oracle's statistics in its weight
    unit, the result must be a local optimum under exact comparisons and never
    above the best subset containing the seed."""
    from fractions import Fraction

    rng = random.Random(int(alpha * 7919))
    nrng = np.random.default_rng(int(alpha * 7919))
    checked = 0
    for it in range(40):
        n = rng.randint(4, 11)
        edges = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < rng.uniform(0.25, 0.6)]
        if not edges:
            continue
        w32 = nrng.uniform(0.5, 2.0, len(edges)).astype(np.float32)
        fr = [Fraction(float(x)) for x in w32]
        L = max(f.denominator for f in fr)
        wi = [int(f * L) for f in fr]  # exact integers in units of 1/L
        g, rp, col = graph_from_edges(orc, n, edges, w32)
        assert g.status == 0
        unit = Fraction(2) ** g.info()["unit_exp"]
        adj = [dict() for _ in range(n)]
        for idx, (a, b) in enumerate(edges):
            adj[a][b] = wi[idx]
            adj[b][a] = wi[idx]
        k = [sum(adj[u].values()) for u in range(n)]
        for seed in range(n):
            mem, f, st, rc = orc.grow(g, seed, alpha)
            assert rc == 0
            c = set(mem.tolist())
            assert seed in c
            K, V = kv(adj, k, c)
            assert Fraction(K, L) == st["K"] * unit and Fraction(V, L) == st["V"] * unit
            if K:
                assert f == pytest.approx(float(Fraction(K, L)) / float(Fraction(V, L)) ** alpha, rel=1e-13)
            for u in range(n):
                if u in c:
                    if u == seed:
                        continue
                    K2, V2 = kv(adj, k, c - {u})
                else:
                    K2, V2 = kv(adj, k, c | {u})
                assert not f_greater(K2, V2, K, V, alpha), (edges, seed, alpha, sorted(c), u)
            if n <= 9:
                others = [u for u in range(n) if u != seed]
                best = (0, 1)
                for r in range(len(others) + 1):
                    for sub in itertools.combinations(others, r):
                        K2, V2 = kv(adj, k, set(sub) | {seed})
                        if f_greater(K2, V2, *best, alpha):
                            best = (K2, V2)
                assert not f_greater(K, V, *best, alpha)
            checked += 1
    assert checked > 150


def structured_graphs():
    """Small graphs whose symmetry makes ranking and fitness ties common: the
    smaller-id rule and the strict tests decide most steps."""
    out = {}
    for n in (5, 8, 12):
        out["ring%d" % n] = (n, [(i, (i + 1) % n) for i in range(n)])
        out["path%d" % n] = (n, [(i, i + 1) for i in range(n - 1)])
    out["grid3x4"] = (12, [(r * 4 + c, r * 4 + c + 1) for r in range(3) for c in range(3)]
                      + [(r * 4 + c, (r + 1) * 4 + c) for r in range(2) for c in range(4)])
    out["torus3x4"] = (12, [(r * 4 + c, r * 4 + (c + 1) % 4) for r in range(3) for c in range(4)]
                       + [(r * 4 + c, ((r + 1) % 3) * 4 + c) for r in range(3) for c in range(4)])
    out["K3,4"] = (7, [(i, 3 + j) for i in range(3) for j in range(4)])
    out["K2,5"] = (7, [(i, 2 + j) for i in range(2) for j in range(5)])
    out["cube"] = (8, [(i, i ^ (1 << b)) for i in range(8) for b in range(3) if i < i ^ (1 << b)])
    out["petersen"] = (10, [(i, (i + 1) % 5) for i in range(5)] + [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
                       + [(i, 5 + i) for i in range(5)])
    out["wheel9"] = (10, [(0, i) for i in range(1, 10)] + [(i, i % 9 + 1) for i in range(1, 10)])
    out["octahedron"] = (6, [(i, j) for i, j in itertools.combinations(range(6), 2) if j != i + 3])
    out["bowtie"] = (5, [(0, 1), (1, 2), (0, 2), (2, 3), (3, 4), (2, 4)])
    out["caveman4x3"] = (12, [(3 * c + i, 3 * c + j) for c in range(4) for i, j in itertools.combinations(range(3), 2)]
                         + [(3 * c + 2, (3 * c + 3) % 12) for c in range(4)])
    return out


@pytest.mark.parametrize("alpha", [1.0, 0.5, 0.75, 0.625, 0.6180339887498949])
@pytest.mark.parametrize("name", sorted(structured_graphs()))
def test_structured_graphs_local_optimum(orc, name, alpha):
    """Symmetric small graphs (rings, paths, grids, tori, complete bipartite,
    cube, Petersen, wheel, octahedron, bowtie, caveman): from every seed the
    result is a local optimum for single moves, checked with exact f, and is
    never above the global optimum over subsets containing the seed."""
    n, edges = structured_graphs()[name]
    edges = sorted({(min(a, b), max(a, b)) for a, b in edges})
    g, _, _ = graph_from_edges(orc, n, edges)
    adj = [dict() for _ in range(n)]
    for a, b in edges:
        adj[a][b] = adj[b][a] = 1
    k = [len(adj[u]) for u in range(n)]
    for seed in range(n):
        mem, f, st, rc = orc.grow(g, seed, alpha)
        assert rc == 0
        c = set(mem.tolist())
        assert seed in c
        K, V = kv(adj, k, c)
        assert (K, V) == (st["K"], st["V"])
        for u in range(n):
            if u == seed:
                continue
            K2, V2 = kv(adj, k, c - {u} if u in c else c | {u})
            assert not f_greater(K2, V2, K, V, alpha), (name, seed, alpha, sorted(c), u)
        others = [u for u in range(n) if u != seed]
        best = (0, 1)
        for r in range(len(others) + 1):
            for sub in itertools.combinations(others, r):
                K2, V2 = kv(adj, k, set(sub) | {seed})
                if f_greater(K2, V2, *best, alpha):
                    best = (K2, V2)
        assert not f_greater(K, V, *best, alpha)


def test_ring_closed_form(orc):
    """On a ring every node has degree 2; from {s} the two neighbours tie in
    rank (d = 1, k = 2) and the smaller id is popped first.  At alpha = 1 a
    path of j nodes has f = 2(j-1)/(2j), which rises with j, so the whole ring
    is grown (f = 1); at alpha = 0.5 the same holds (2(j-1)/sqrt(2j) rises)."""
    n = 9
    g, _, _ = graph_from_edges(orc, n, [(i, (i + 1) % n) for i in range(n)])
    for alpha in (1.0, 0.5):
        for seed in range(n):
            mem, f, st, rc = orc.grow(g, seed, alpha)
            assert mem.tolist() == list(range(n))
            assert f == pytest.approx((2 * n) ** (1 - alpha), rel=1e-15)


@pytest.mark.parametrize("alpha", [0.5, 0.75, 1.0])
def test_disjoint_cliques_reach_global_optimum(orc, alpha):
    """The seed's component is a clique: growth returns exactly that clique, the
    global optimum over subsets containing the seed."""
    sizes = [3, 5, 2, 4]
    edges, base = [], 0
    for m in sizes:
        edges += [(base + i, base + j) for i, j in itertools.combinations(range(m), 2)]
        base += m
    g, _, _ = graph_from_edges(orc, base, edges)
    base = 0
    for m in sizes:
        for seed in range(base, base + m):
            mem, f, st, rc = orc.grow(g, seed, alpha)
            assert mem.tolist() == list(range(base, base + m))
        base += m


def _f(K, V, alpha):
    import mpmath as mp

    return mp.mpf(0) if K == 0 else mp.mpf(K) / mp.power(mp.mpf(V), mp.mpf(alpha))


def _barbell_conditions(m, alpha):
    """Closed forms for two K_m joined by the bridge (m-1, m), grown from a seed
    in the first clique A = {0..m-1}: (i) every addition of an A node improves
    f, whatever A nodes are already in (K = j(j-1), V = sum of their degrees,
    m-1 for a plain A node and m for the bridge end); (ii) at c = A the bridge
    partner m (d = 1, k = m) fails the add test; (iii) no A node passes the
    remove test at c = A.  A nodes always rank before node m (d >= 1 with
    k <= m against d = 1 with k = m), so (i)-(iii) make the result exactly A."""
    import mpmath as mp

    mp.mp.prec = 300
    adds_ok = True
    for plain in range(0, m):          # plain A nodes in c
        for bridge in (0, 1):          # the bridge end m-1 in c
            j = plain + bridge
            if j == 0 or j == m:
                continue
            K, V = j * (j - 1), plain * (m - 1) + bridge * m
            cands = ([m - 1] if plain < m - 1 else []) + ([m] if not bridge else [])
            adds_ok &= all(_f(K + 2 * j, V + k, alpha) > _f(K, V, alpha) for k in cands)
    K, V = m * (m - 1), m * (m - 1) + 1
    bridge_fails = not _f(K + 2, V + m, alpha) > _f(K, V, alpha)
    no_removal = all(not _f(K - 2 * (m - 1), V - k, alpha) > _f(K, V, alpha) for k in (m - 1, m))
    return adds_ok, bridge_fails, no_removal


@pytest.mark.parametrize("m", [3, 4, 5, 7])
@pytest.mark.parametrize("alpha", [0.5, 0.6, 0.75, 0.9, 1.0])
def test_barbell_closed_form(orc, m, alpha):
    """Two m-cliques joined by one edge.  Where the closed-form conditions hold
    the growth from any seed of a clique returns exactly that clique with
    f = m(m-1) / (m(m-1)+1)^alpha (not the global optimum at alpha = 1, which
    is the whole graph with f = 1: the greedy stops at the bridge); where only
    the bridge test flips, the partner across the bridge joins."""
    edges = [(i, j) for i, j in itertools.combinations(range(m), 2)]
    edges += [(m + i, m + j) for i, j in itertools.combinations(range(m), 2)]
    edges += [(m - 1, m)]
    g, _, _ = graph_from_edges(orc, 2 * m, edges)
    adds_ok, bridge_fails, no_removal = _barbell_conditions(m, alpha)
    K, V = m * (m - 1), m * (m - 1) + 1
    for seed in range(2 * m):
        mem, f, st, rc = orc.grow(g, seed, alpha)
        assert rc == 0 and seed in mem.tolist()
        own = list(range(m)) if seed < m else list(range(m, 2 * m))
        partner = m if seed < m else m - 1
        if adds_ok and bridge_fails and no_removal:
            assert mem.tolist() == own
            assert st["K"] == K and st["V"] == V
            assert f == pytest.approx(float(_f(K, V, alpha)), rel=1e-15)
        elif adds_ok and not bridge_fails:
            assert partner in mem.tolist() and set(own) <= set(mem.tolist())
    if (m, alpha) in ((5, 1.0), (7, 0.5)):
        assert adds_ok and bridge_fails and no_removal  # the exact case is exercised


def test_round_cap(orc):
    """The repetition cap of Alg. 1 (the paper leaves its value open): a unit
    that needs R rounds (the last one adds nothing) runs min(R, cap) rounds;
    with cap >= R - 1 it ends with the uncapped community, and the run reports
    the time-out whenever some R > cap; units cut before a later growth
    round end with a different community."""
    g = synth.hierarchical_lfr(5000, 20, 200, 2.5, 1.5, (20, 1000), (0.3, 0.1), seed=17)
    G = orc.Graph(g.n, g.row_ptr, g.col)
    alphas = [1.0, 0.7, 0.5, 0.35]
    seeds = np.arange(0, g.n, 2, dtype=np.int32)
    rc, ptr, nodes, f, st = orc.run(G, alphas, seeds, threads=8)
    assert rc == 0
    R = st[:, 3]
    assert R.max() >= 3  # some unit prunes and grows again
    for cap in (1, 2, int(R.max())):
        rc2, p2, n2, f2, st2 = orc.run(G, alphas, seeds, threads=8, max_rounds=cap)
        assert rc2 == (-8 if (R > cap).any() else 0)
        assert np.array_equal(st2[:, 3], np.minimum(R, cap))
        cut = 0
        for u in range(len(R)):
            same = np.array_equal(nodes[ptr[u]:ptr[u + 1]], n2[p2[u]:p2[u + 1]])
            if R[u] - 1 <= cap:
                assert same
            else:
                cut += not same
        assert cut == int((R - 1 > cap).sum())


def test_thread_count_independent(orc):
    g0 = synth.config_graph(0)
    g = orc.Graph(g0.n, g0.row_ptr, g0.col)
    alphas = [1.0, 0.7, 0.5]
    seeds = np.arange(0, 1000, 7, dtype=np.int32)
    r1 = orc.run(g, alphas, seeds, threads=1)
    r4 = orc.run(g, alphas, seeds, threads=4)
    assert r1[0] == 0 and r4[0] == 0
    for a, b in zip(r1[1:], r4[1:]):
        assert np.array_equal(a, b)


def jaccard_best(found, planted):
    out = []
    for P in planted:
        best = 0.0
        for C in found:
            inter = len(P & C)
            if inter:
                best = max(best, inter / len(P | C))
        out.append(best)
    return float(np.mean(out))


def test_planted_recovery(orc):
    """1,000-node planted partition: some scale recovers the 20 communities and a
    coarser one the 4 super-groups (the paper's Table 1 shows the same two-band
    behaviour on its hierarchical benchmark)."""
    g0 = synth.config_graph(0)
    g = orc.Graph(g0.n, g0.row_ptr, g0.col)
    rc, alphas = orc.scales_logspaced(0.5, 1.0, 8)
    rc, ptr, nodes, f, st = orc.run(g, alphas, threads=8)
    assert rc == 0
    micro = [set(np.flatnonzero(g0.labels[0] == c).tolist()) for c in range(20)]
    macro = [set(np.flatnonzero(g0.labels[1] == c).tolist()) for c in range(4)]
    best_micro = best_macro = 0.0
    for s in range(8):
        sl = slice(s * 1000, (s + 1) * 1000 + 1)
        p = ptr[sl] - ptr[s * 1000]
        cptr, cnodes, u2c, first = orc.unique_communities(p, nodes[ptr[s * 1000]:ptr[(s + 1) * 1000]])
        found = [set(cnodes[cptr[i]:cptr[i + 1]].tolist()) for i in range(len(cptr) - 1)]
        jm = min(jaccard_best(micro, found), jaccard_best(found, micro))
        jM = min(jaccard_best(macro, found), jaccard_best(found, macro))
        best_micro, best_macro = max(best_micro, jm), max(best_macro, jM)
    assert best_micro >= 0.9
    assert best_macro >= 0.9


# ------------------------------------------------- growth from initial members

def test_initial_members_empty_and_fixed_point(orc):
    """Alg. 2 may start from given communities.  An empty initial set is the
    plain growth; a grown community is a fixed point (no addition improves f,
    so the first grow pass ends at once and no prune pass runs)."""
    from paper_1301_0955_gb300 import synth

    g = synth.config_graph(0)
    G = orc.Graph(g.n, g.row_ptr, g.col)
    seeds = np.arange(0, g.n, 7, dtype=np.int32)
    alphas = [1.0, 0.6]
    rc, ptr, nodes, f, st = orc.run(G, alphas, seeds, threads=4)
    assert rc == 0
    empty = (np.zeros(len(seeds) + 1, np.int64), np.zeros(0, np.int32))
    rc, p0, n0, f0, st0 = orc.run(G, alphas, seeds, threads=4, init=empty)
    assert rc == 0 and np.array_equal(p0, ptr) and np.array_equal(n0, nodes) and np.array_equal(st0, st)
    N = len(seeds)
    for s in range(2):
        sl = ptr[s * N:(s + 1) * N + 1]
        init = (sl - sl[0], nodes[sl[0]:sl[-1]])
        rc, p1, n1, f1, st1 = orc.run(G, [alphas[s]], seeds, threads=4, init=init)
        assert rc == 0
        assert np.array_equal(p1, init[0]) and np.array_equal(n1, init[1])
        assert (st1[:, 1] == 0).all() and (st1[:, 3] == 1).all() and (st1[:, 2] == 0).all()
        np.testing.assert_array_equal(f1, f[s * N:(s + 1) * N])


@pytest.mark.parametrize("alpha", [1.0, 0.5, 0.75])
def test_initial_members_bruteforce(orc, alpha):
    """From a random initial set on <= 12-node graphs: the seed stays; if a
    node was added the result is a local optimum for single additions and
    non-seed removals; if none was, the result is the initial set with the
    seed and no single addition improves it."""
    rng = random.Random(int(alpha * 77))
    checked = 0
    for it in range(50):
        n = rng.randint(4, 12)
        edges, w = random_small_graph(rng, n, rng.uniform(0.2, 0.6), it % 3 == 2)
        if not edges:
            continue
        g, rp, col = graph_from_edges(orc, n, edges, w)
        adj = [dict() for _ in range(n)]
        for idx, (a, b) in enumerate(edges):
            ww = 1 if w is None else w[idx]
            adj[a][b] = ww
            adj[b][a] = ww
        k = [sum(adj[u].values()) for u in range(n)]
        seeds = np.arange(n, dtype=np.int32)
        inits = [rng.sample(range(n), rng.randint(0, n - 1)) for _ in range(n)]
        iptr = np.concatenate([[0], np.cumsum([len(x) for x in inits])]).astype(np.int64)
        inodes = np.array([v for x in inits for v in x], np.int32)
        rc, ptr, nodes, f, st = orc.run(g, [alpha], seeds, init=(iptr, inodes))
        assert rc == 0
        for seed in range(n):
            c = set(nodes[ptr[seed]:ptr[seed + 1]].tolist())
            assert seed in c
            K, V = kv(adj, k, c)
            start = set(inits[seed]) | {seed}
            if st[seed, 1] == 0:
                assert c == start
            for u in range(n):
                if u in c:
                    if u == seed or st[seed, 1] == 0:
                        continue
                    K2, V2 = kv(adj, k, c - {u})
                else:
                    K2, V2 = kv(adj, k, c | {u})
                assert not f_greater(K2, V2, K, V, alpha), (edges, seed, sorted(c), u)
            checked += 1
    assert checked > 150
