"""Pins for the oracle's graph checks, exact weights, dedup, NMI and scale list.

* graph checks: one malformed input per error category, and the category
  order when several are present;
* weights: the fixed-point value times 2^unit_exp reproduces every FP32
  weight exactly (Fraction arithmetic) and the unit is the largest power of
  two dividing them all;
* dedup: brute-force pairwise set equality;
* overlapping NMI (Lancichinetti, Fortunato & Kertesz, cited in Sec. 4; the
  paper does not print it): identity gives 1, covers whose every pair fails
  the admission test give 0, symmetry, invariance under node relabelling;
* scale list (Sec. 4 formula, read as V_min + (A-V_min)(1 - log k / log X)):
  endpoints, monotone order, spacing dense near V_min.
"""
import random
from fractions import Fraction

import numpy as np
import pytest

from paper_1301_0955_gb300 import synth


def csr(n, edges, w=None):
    e = np.asarray(edges, np.int64).reshape(-1, 2)
    return synth.to_csr(n, e[:, 0], e[:, 1], None if w is None else np.asarray(w, np.float32))


def test_valid_graph(orc):
    rp, col, _ = csr(4, [(0, 1), (1, 2), (2, 3)])
    g = orc.Graph(4, rp, col)
    assert g.status == 0
    assert g.degrees().tolist() == [1, 2, 2, 1]
    assert g.info()["volume"] == 6


def test_error_categories(orc):
    rp, col, _ = csr(4, [(0, 1), (1, 2), (2, 3)])  # col: 1 | 0 2 | 1 3 | 2
    # structure: bad row_ptr start, decreasing, column out of range
    assert orc.Graph(4, np.r_[1, rp[1:]], col).status == orc.EINVAL
    bad = rp.copy(); bad[2] = 0
    assert orc.Graph(4, bad, col).status == orc.EINVAL
    c2 = col.copy(); c2[0] = 7
    assert orc.Graph(4, rp, c2).status == orc.EINVAL
    # weights
    w = np.ones(len(col), np.float32); w[3] = -1.0
    assert orc.Graph(4, rp, col, w).status == orc.EWEIGHT
    w[3] = np.nan
    assert orc.Graph(4, rp, col, w).status == orc.EWEIGHT
    w[3] = 0.0
    assert orc.Graph(4, rp, col, w).status == orc.EWEIGHT
    # self loop
    c3 = col.copy(); c3[1] = 1
    assert orc.Graph(4, rp, c3).status == orc.ESELFLOOP
    # unsorted row (row 1 = [2, 0])
    c4 = col.copy(); c4[1], c4[2] = c4[2], c4[1]
    assert orc.Graph(4, rp, c4).status == orc.EUNSORTED
    # duplicate: row 1 = [0, 0] (also asymmetric, duplicate reported first)
    c5 = col.copy(); c5[2] = 0
    assert orc.Graph(4, rp, c5).status == orc.EDUP
    # asymmetric: 3 -> 1 instead of 3 -> 2
    c6 = col.copy(); c6[-1] = 1
    assert orc.Graph(4, rp, c6).status == orc.ENOTSYM
    # unequal weights in the two directions
    w = np.ones(len(col), np.float32); w[0] = 2.0
    assert orc.Graph(4, rp, col, w).status == orc.ENOTSYM
    # category order: a self loop and an asymmetry -> self loop reported
    c7 = c6.copy(); c7[1] = 1
    assert orc.Graph(4, rp, c7).status == orc.ESELFLOOP
    # empty graph and isolated nodes are fine
    assert orc.Graph(0, np.zeros(1, np.int64), np.zeros(0, np.int32)).status == 0
    assert orc.Graph(3, np.zeros(4, np.int64), np.zeros(0, np.int32)).status == 0


def test_fixed_point_weights_exact(orc):
    rng = np.random.default_rng(5)
    for trial in range(20):
        n = 40
        edges = sorted({tuple(sorted(rng.choice(n, 2, replace=False).tolist())) for _ in range(120)})
        kind = trial % 4
        if kind == 0:
            w = rng.uniform(0.5, 2.0, len(edges))
        elif kind == 1:
            w = np.exp(rng.uniform(-8, 8, len(edges)))
        elif kind == 2:
            w = rng.integers(1, 9, len(edges)) * 4.0
        else:
            w = rng.uniform(1e-40, 1e-38, len(edges))  # FP32 subnormals
        w = w.astype(np.float32)
        rp, col, ww = csr(n, edges, w)
        g = orc.Graph(n, rp, col, ww)
        assert g.status == 0
        ue = g.info()["unit_exp"]
        wf = g.weights_fixed()
        unit = Fraction(2) ** ue
        for a, b in zip(wf.tolist(), ww.tolist()):
            assert Fraction(a) * unit == Fraction(b)
        # largest power of two dividing all: some fixed-point weight is odd
        assert (wf % 2 == 1).any()
        k = g.degrees()
        assert np.array_equal(k, np.add.reduceat(wf, rp[:-1]) * (np.diff(rp) > 0))


def test_fixed_point_range_error(orc):
    w = np.array([2.0 ** 100, 2.0 ** -100], np.float32)
    rp, col, ww = csr(3, [(0, 1), (1, 2)], w)
    assert orc.Graph(3, rp, col, ww).status == orc.ERANGE


def test_dedup_bruteforce(orc):
    rng = random.Random(3)
    for trial in range(30):
        pool = [sorted(rng.sample(range(50), rng.randint(1, 8))) for _ in range(6)]
        lists = [rng.choice(pool) for _ in range(rng.randint(1, 40))]
        ptr = np.r_[0, np.cumsum([len(l) for l in lists])]
        nodes = np.concatenate([np.asarray(l, np.int32) for l in lists])
        nc, u2c, first = orc.dedup(ptr, nodes)
        for i in range(len(lists)):
            for j in range(len(lists)):
                assert (u2c[i] == u2c[j]) == (lists[i] == lists[j])
        # numbered by first occurrence
        assert first.tolist() == sorted(first.tolist())
        assert [u2c[f] for f in first] == list(range(nc))


def cover(lists):
    ptr = np.r_[0, np.cumsum([len(l) for l in lists])].astype(np.int64)
    nodes = np.concatenate([np.asarray(sorted(l), np.int32) for l in lists])
    return ptr, nodes


def test_nmi_identity_and_symmetry(orc):
    rng = random.Random(1)
    for trial in range(30):
        n = rng.randint(5, 60)
        X = [rng.sample(range(n), rng.randint(1, n - 1)) for _ in range(rng.randint(1, 6))]
        Y = [rng.sample(range(n), rng.randint(1, n - 1)) for _ in range(rng.randint(1, 6))]
        assert orc.nmi(n, *cover(X), *cover(X)) == pytest.approx(1.0, abs=1e-15)
        a = orc.nmi(n, *cover(X), *cover(Y))
        b = orc.nmi(n, *cover(Y), *cover(X))
        assert a == pytest.approx(b, abs=1e-15)
        assert -1e-12 <= a <= 1 + 1e-12
        perm = list(range(n))
        rng.shuffle(perm)
        Xp = [[perm[u] for u in c] for c in X]
        Yp = [[perm[u] for u in c] for c in Y]
        assert orc.nmi(n, *cover(Xp), *cover(Yp)) == pytest.approx(a, abs=1e-14)


def test_nmi_zero_cases(orc):
    # every pair has P11 = P10 = P01 = P00 = 1/4: admission fails, N = 0
    assert orc.nmi(4, *cover([[0, 1]]), *cover([[0, 2]])) == pytest.approx(0.0, abs=1e-15)
    # complementary halves: P11 = P00 = 0, admission fails, N = 0
    assert orc.nmi(10, *cover([[0, 1, 2, 3, 4]]), *cover([[5, 6, 7, 8, 9]])) == pytest.approx(0.0, abs=1e-15)
    # identical partitions in a different community order
    X = [[0, 1, 2], [3, 4], [5, 6, 7, 8]]
    assert orc.nmi(9, *cover(X), *cover(X[::-1])) == pytest.approx(1.0, abs=1e-15)


def test_nmi_whole_graph_community(orc):
    """A community holding all n nodes has H = 0; its normalised term is 0 by
    the stated reading, so a cover made of it alone against itself gives 1."""
    assert orc.nmi(6, *cover([list(range(6))]), *cover([list(range(6))])) == pytest.approx(1.0)


def test_scales(orc):
    rc, s = orc.scales_logspaced(0.5, 1.0, 8)
    assert rc == 0 and s[0] == 1.0 and s[-1] == 0.5
    assert np.all(np.diff(s) < 0)
    gaps = -np.diff(s)
    assert np.all(np.diff(gaps) < 0)  # spread out towards A, dense near V_min
    rc, s1 = orc.scales_logspaced(0.5, 1.0, 1)
    assert rc == 0 and s1.tolist() == [1.0]
    assert orc.scales_logspaced(0.5, 1.0, 0)[0] == orc.EINVAL
    assert orc.scales_logspaced(-1.0, 1.0, 3)[0] == orc.EINVAL


@pytest.mark.parametrize("X,points", [
    # X a power of 2: log k / log X = j / m at k = 2^j, so the interior values
    # at those k are the fractions of the way from A down to V_min below
    (4, {2: (1, 2)}),
    (8, {2: (1, 3), 4: (2, 3)}),
    (16, {2: (1, 4), 4: (2, 4), 8: (3, 4)}),
    (32, {2: (1, 5), 4: (2, 5), 8: (3, 5), 16: (4, 5)}),
    # X a power of 3
    (9, {3: (1, 2)}),
    (27, {3: (1, 3), 9: (2, 3)}),
    # X = 20 (the benchmark's count): 20 = 4 * 5 gives no rational ratio but
    # log 4 / log 20 + log 5 / log 20 = 1, i.e. the two offsets from A sum to
    # A - V_min (checked below)
])
def test_scales_interior_closed_form(orc, X, points):
    """Interior values of the Sec. 4 scale list (read as V_min + (A - V_min)
    (1 - log k / log X), k = 1..X).  Where log k / log X is the rational j/m,
    the k-th value is V_min + (A - V_min)(1 - j/m): on [0.5, 1] the k = 2 value
    of X = 4 is the midpoint 0.75, that of X = 8 is 1 - 0.5/3, and so on.  An
    off-by-one in k (k - 1, k + 1, 0-based), another logarithm base that is not
    a ratio, or the garbled (1 - log k) / log X all move these points."""
    vmin, A = 0.5, 1.0
    rc, s = orc.scales_logspaced(vmin, A, X)
    assert rc == 0 and len(s) == X
    for k, (j, m) in points.items():
        want = vmin + (A - vmin) * (m - j) / m
        assert s[k - 1] == pytest.approx(want, rel=0, abs=4e-16), (X, k)
    # another interval: the same fractions of its width
    rc, t = orc.scales_logspaced(0.25, 2.0, X)
    for k, (j, m) in points.items():
        assert t[k - 1] == pytest.approx(0.25 + 1.75 * (m - j) / m, rel=0, abs=1e-15)


def test_scales_interior_complementary_pair(orc):
    """For X = 20 the ratios at k = 4 and k = 5 sum to one (4 * 5 = 20), so the
    two values sum to A + V_min; likewise k = 2 and 10, then k = 2 and k = 10
    against k = 20 (the end, V_min)."""
    rc, s = orc.scales_logspaced(0.5, 1.0, 20)
    assert rc == 0
    assert s[3] + s[4] == pytest.approx(1.5, abs=1e-15)
    assert s[1] + s[9] == pytest.approx(1.5, abs=1e-15)
    # X = 32 (the weighted workload's count): k = 2 and k = 16 sum to one
    rc, t = orc.scales_logspaced(0.5, 1.0, 32)
    assert t[1] + t[15] == pytest.approx(1.5, abs=1e-15)
    assert t[3] + t[7] == pytest.approx(1.5, abs=1e-15)


def test_window_means(orc):
    nmi = np.array([0.1, 0.2, 0.3, 0.4])  # 5 scales
    w3 = orc.window_means(nmi, 5, 3)
    assert w3.tolist() == pytest.approx([0.1, 0.15, 0.25, 0.35, 0.4])
    w5 = orc.window_means(nmi, 5, 5)
    assert w5.tolist() == pytest.approx([0.15, 0.2, 0.25, 0.3, 0.35])
    one = orc.window_means(np.zeros(0), 1, 3)
    assert np.isnan(one[0])


def test_nmi_hand_computed_two_covers(orc):
    """A worked example of the overlapping NMI (Sec. 4): n = 4, X = {{0, 1}},
    Y = {{0, 1, 2}}.  With h(p) = -p log2 p: H(X_1) = 1; H(Y_1) = h(3/4) +
    h(1/4) = 2 - (3/4) log2 3.  The pair has P11 = 1/2, P10 = 0, P01 = 1/4,
    P00 = 1/4, so h(P11) + h(P00) = 1 > h(P01) + h(P10) = 1/2 (admitted) and
    H(X_1, Y_1) = 3/2.  Hence H(X_1|Y) = 3/2 - H(Y_1) (normalised by 1) and
    H(Y_1|X) = 3/2 - 1 = 1/2 (normalised by H(Y_1)), and
    N = 1 - [(3/2 - H(Y_1)) + 1 / (2 H(Y_1))] / 2."""
    import math

    HY = 2.0 - 0.75 * math.log2(3.0)
    want = 1.0 - 0.5 * ((1.5 - HY) + 0.5 / HY)
    a = (np.array([0, 2], np.int64), np.array([0, 1], np.int32))
    b = (np.array([0, 3], np.int64), np.array([0, 1, 2], np.int32))
    assert orc.nmi(4, *a, *b) == pytest.approx(want, abs=1e-15)
    assert orc.nmi(4, *b, *a) == pytest.approx(want, abs=1e-15)
    # adding to Y a community of the remaining node leaves X's term (its best
    # partner is unchanged) and gives Y_2 = {3} a partner that is not admitted
    # (disjoint, |X_1| + |Y_2| <= n/2), so H(Y_2|X) = H(Y_2), normalised 1
    b2 = (np.array([0, 3, 4], np.int64), np.array([0, 1, 2, 3], np.int32))
    want2 = 1.0 - 0.5 * ((1.5 - HY) + 0.5 * (0.5 / HY + 1.0))
    assert orc.nmi(4, *a, *b2) == pytest.approx(want2, abs=1e-15)


def _random_cover(rng, n, k, lo, hi):
    ptr, nodes = [0], []
    for _ in range(k):
        m = int(rng.integers(lo, min(hi, n) + 1))
        nodes.append(np.sort(rng.choice(n, m, replace=False)))
        ptr.append(ptr[-1] + m)
    return np.array(ptr, np.int64), np.concatenate(nodes).astype(np.int32)


@pytest.mark.parametrize("seed", range(12))
def test_nmi_indexed_equals_dense_definition(orc, seed):
    """The indexed variant counts intersections through a node -> communities
    index instead of intersecting every pair of lists; everything else is the
    dense definition, so the two agree bit for bit (random overlapping covers,
    small and large communities, whole-graph and disjoint ones, 1 and 4
    threads)."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 400))
    X = _random_cover(rng, n, int(rng.integers(1, 40)), 1, max(2, n // int(rng.integers(1, 8))))
    Y = _random_cover(rng, n, int(rng.integers(1, 40)), 1, max(2, n // int(rng.integers(1, 8))))
    if seed % 3 == 0:  # a community of every node
        Y = (np.append(Y[0], Y[0][-1] + n), np.concatenate([Y[1], np.arange(n, dtype=np.int32)]))
    want = orc.nmi(n, *X, *Y)
    for t in (1, 4):
        got = orc.nmi_indexed(n, *X, *Y, threads=t)
        assert got == want or (np.isnan(got) and np.isnan(want)), (seed, t, got, want)


def test_nmi_indexed_hand_example(orc):
    """The worked two-cover example (closed form above) through the indexed variant."""
    import math

    HY = 2.0 - 0.75 * math.log2(3.0)
    want = 1.0 - 0.5 * ((1.5 - HY) + 0.5 / HY)
    a = (np.array([0, 2], np.int64), np.array([0, 1], np.int32))
    b = (np.array([0, 3], np.int64), np.array([0, 1, 2], np.int32))
    assert orc.nmi_indexed(4, *a, *b) == pytest.approx(want, abs=1e-15)
