"""Pins for the oracle's decision arithmetic (the sign of Eq. 2 and of ranking-factor
comparisons), checked against exact big-integer arithmetic and 400-bit mpmath.

Every decision of the method is the sign of
    Delta = log(a1/a2) - alpha * log(b1/b2)
(add test Eq. 2: a = (K+2d)/K, b = (V+k)/V; remove test: a = (K-2d)/K,
b = (V-k)/V; ranking factor 2 d / k^alpha of the Sec. 2 priority queue:
a = d1/d2, b = k1/k2).  For alpha = P / 2^s the sign equals the sign of
a1^(2^s) b2^P - a2^(2^s) b1^P, a plain integer comparison.
"""
import random
from fractions import Fraction

import pytest

DYADIC = [(1, 0), (1, 1), (3, 2), (5, 3), (7, 4)]  # alpha = P / 2^s: 1, 1/2, 3/4, 5/8, 7/16


def exact_sign_dyadic(a1, a2, b1, b2, P, s):
    lhs = a1 ** (2 ** s) * b2 ** P
    rhs = a2 ** (2 ** s) * b1 ** P
    return (lhs > rhs) - (lhs < rhs)


def mp_sign(a1, a2, b1, b2, alpha):
    mpmath = pytest.importorskip("mpmath")
    with mpmath.workprec(400):
        d = mpmath.log(mpmath.mpf(a1) / a2) - mpmath.mpf(alpha) * mpmath.log(mpmath.mpf(b1) / b2)
        if abs(d) < mpmath.mpf(2) ** -360:
            return 0
        return 1 if d > 0 else -1


def rand_tuple(rng, bits):
    return [rng.randrange(1, 2 ** bits) for _ in range(4)]


@pytest.mark.parametrize("P,s", DYADIC)
def test_sign_random_vs_bigint(orc, P, s):
    rng = random.Random(1000 + P)
    alpha = P / 2 ** s
    for it in range(4000):
        bits = rng.choice([3, 8, 20, 40, 61])
        a1, a2, b1, b2 = rand_tuple(rng, bits)
        got, _ = orc.sign_delta(a1, a2, b1, b2, alpha)
        assert got == exact_sign_dyadic(a1, a2, b1, b2, P, s), (a1, a2, b1, b2, alpha)


@pytest.mark.parametrize("P,s", DYADIC)
def test_sign_near_one_vs_bigint(orc, P, s):
    """Ratios close to 1 (the add/remove tests on big communities)."""
    rng = random.Random(2000 + P)
    alpha = P / 2 ** s
    for it in range(3000):
        K = rng.randrange(2, 2 ** rng.choice([10, 30, 50, 61]))
        V = K + rng.randrange(0, K + 1)
        d = rng.randrange(1, max(2, K // rng.choice([2, 100, 10 ** 6])))
        k = rng.randrange(1, max(2, V // rng.choice([2, 100, 10 ** 6])))
        for a1, a2, b1, b2 in ((K + 2 * d, K, V + k, V), (max(1, K - 2 * d), K, V - k if V > k else V + k, V)):
            got, _ = orc.sign_delta(a1, a2, b1, b2, alpha)
            assert got == exact_sign_dyadic(a1, a2, b1, b2, P, s), (a1, a2, b1, b2, alpha)


def test_constructed_exact_ties(orc):
    """a = t^P, b = t^(2^s): Delta is exactly 0 and must be reported as a tie."""
    rng = random.Random(7)
    n = 0
    for P, s in DYADIC:
        alpha = P / 2 ** s
        for it in range(300):
            u, v = rng.randrange(1, 40), rng.randrange(1, 40)
            if u == v:
                continue
            bn, bd = u ** (2 ** s), v ** (2 ** s)
            an, ad = u ** P, v ** P
            if max(bn, bd, an, ad) >= 2 ** 62:
                continue
            m = rng.randrange(1, 2 ** 62 // max(an, ad, bn, bd) + 1)
            m2 = rng.randrange(1, 2 ** 62 // max(an, ad, bn, bd) + 1)
            got, path = orc.sign_delta(an * m, ad * m, bn * m2, bd * m2, alpha)
            assert got == 0 and path == 3, (an, ad, bn, bd, alpha, got, path)
            n += 1
    assert n > 500
    # the worked example of a tie at alpha = 1/2: (d, k) = (1, 4) vs (2, 16)
    assert orc.sign_delta(1, 2, 4, 16, 0.5)[0] == 0


def test_near_ties_decided_by_binary128(orc):
    """Non-ties whose |Delta| is below the binary64 certification band."""
    rng = random.Random(11)
    seen_quad = 0
    for P, s in DYADIC:
        alpha = P / 2 ** s
        for it in range(400):
            u, v = rng.randrange(2, 60), rng.randrange(2, 60)
            if u == v:
                continue
            bn, bd = u ** (2 ** s), v ** (2 ** s)
            an, ad = u ** P, v ** P
            if max(bn, bd, an, ad) > 2 ** 30:
                continue
            m = 2 ** 30
            # perturb one operand by 1 unit at scale 2^30: |Delta| ~ 2^-60
            a1 = an * m + rng.choice([-1, 1])
            got, path = orc.sign_delta(a1, ad * m, bn, bd, alpha)
            assert got == exact_sign_dyadic(a1, ad * m, bn, bd, P, s)
            seen_quad += path == 2
    assert seen_quad > 100


def test_general_alpha_vs_mpmath(orc):
    rng = random.Random(3)
    for it in range(1500):
        alpha = rng.uniform(0.3, 1.7)
        bits = rng.choice([4, 16, 40, 61])
        a1, a2, b1, b2 = rand_tuple(rng, bits)
        got, _ = orc.sign_delta(a1, a2, b1, b2, alpha)
        assert got == mp_sign(a1, a2, b1, b2, alpha), (a1, a2, b1, b2, alpha)


def test_general_alpha_near_ties_vs_mpmath(orc):
    """Construct a1/a2 ~ (b1/b2)^alpha to within one unit for a generic alpha."""
    mpmath = pytest.importorskip("mpmath")
    rng = random.Random(5)
    paths = set()
    for it in range(400):
        alpha = rng.choice([0.7, 0.6321, 0.5385, 0.9123])
        b2 = rng.randrange(2 ** 20, 2 ** 40)
        b1 = b2 + rng.randrange(1, 2 ** 10)
        a2 = rng.randrange(2 ** 40, 2 ** 61)
        with mpmath.workprec(300):
            a1 = int(mpmath.nint(a2 * (mpmath.mpf(b1) / b2) ** mpmath.mpf(alpha)))
        a1 += rng.choice([-1, 0, 1])
        got, path = orc.sign_delta(a1, a2, b1, b2, alpha)
        paths.add(path)
        assert got == mp_sign(a1, a2, b1, b2, alpha), (a1, a2, b1, b2, alpha)
    assert 1 in paths


def test_add_remove_tests_vs_fitness(orc):
    """Eq. 2 as a strict test: add iff f(c+n) > f(c), remove iff f(c\\n) > f(c),
    with f = K / V^alpha (Eq. 1) evaluated exactly (bigint for dyadic alpha)."""
    rng = random.Random(9)
    for it in range(3000):
        P, s = rng.choice(DYADIC)
        alpha = P / 2 ** s
        K = rng.randrange(0, 2 ** rng.choice([6, 20, 40]))
        V = K + rng.randrange(1, K + 3)
        d = rng.randrange(1, 50)
        k = d + rng.randrange(0, 50)
        # add: compare (K+2d)/(V+k)^alpha with K/V^alpha
        if K == 0:
            want_add = 1
        else:
            want_add = int(exact_sign_dyadic(K + 2 * d, K, V + k, V, P, s) > 0)
        assert orc.add_test(K, V, d, k, alpha) == want_add
        if K - 2 * d > 0 and V - k > 0:
            want_rm = int(exact_sign_dyadic(K - 2 * d, K, V - k, V, P, s) > 0)
            assert orc.remove_test(K, V, d, k, alpha) == want_rm
        elif K - 2 * d == 0 and V - k > 0:
            assert orc.remove_test(K, V, d, k, alpha) == 0


def test_add_test_tie_is_rejected(orc):
    """f(c+n) == f(c) exactly is not an improvement (strict test)."""
    # alpha = 1: (K+2d)/(V+k) == K/V  <=>  2d V == K k
    assert orc.add_test(6, 9, 1, 3, 1.0) == 0
    assert orc.add_test(6, 9, 2, 3, 1.0) == 1
    # alpha = 1/2: (K+2d)^2 V == K^2 (V+k) with K=2, d=1, V=1, k=3
    assert orc.add_test(2, 1, 1, 3, 0.5) == 0


def test_priority_order(orc):
    """Ranking factor 2 d / k^alpha, max first, equal values by smaller node id."""
    rng = random.Random(13)
    for it in range(3000):
        P, s = rng.choice(DYADIC)
        alpha = P / 2 ** s
        d1, d2 = rng.randrange(1, 30), rng.randrange(1, 30)
        k1, k2 = d1 + rng.randrange(0, 60), d2 + rng.randrange(0, 60)
        i1, i2 = rng.sample(range(100), 2)
        sg = exact_sign_dyadic(d1, d2, k1, k2, P, s)
        want = 1 if sg > 0 else -1 if sg < 0 else (1 if i1 < i2 else -1)
        assert orc.priority_cmp(d1, k1, i1, d2, k2, i2, alpha) == want, (d1, k1, d2, k2, alpha)
    # exact ties of the ranking factor at alpha = 1 and 1/2 go to the smaller id
    assert orc.priority_cmp(1, 4, 9, 2, 8, 3, 1.0) == -1
    assert orc.priority_cmp(1, 4, 3, 2, 16, 9, 0.5) == 1


def test_fitness_values(orc):
    mpmath = pytest.importorskip("mpmath")
    rng = random.Random(17)
    for it in range(500):
        K = rng.randrange(1, 2 ** 40)
        V = K + rng.randrange(0, 2 ** 40)
        alpha = rng.uniform(0.3, 1.5)
        ue = rng.choice([0, -24, -23, 5])
        with mpmath.workprec(200):
            want = (mpmath.mpf(K) * mpmath.mpf(2) ** ue) / (mpmath.mpf(V) * mpmath.mpf(2) ** ue) ** mpmath.mpf(alpha)
        got = orc.fitness(K, V, alpha, ue)
        assert abs(got - float(want)) <= 2e-16 * float(want)
    assert orc.fitness(0, 5, 0.7) == 0.0
