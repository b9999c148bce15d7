"""GPU: the NMI between caller covers (mscd_nmi_covers) against the oracle."""
import numpy as np
import pytest

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


def random_cover(rng, n, k, overlap):
    lists = []
    for _ in range(k):
        m = int(rng.integers(1, max(2, n // 3)))
        lists.append(np.unique(rng.choice(n, m, replace=False)))
    if not overlap:  # a partition
        lab = rng.integers(0, k, n)
        lists = [np.nonzero(lab == c)[0] for c in range(k) if (lab == c).any()]
    ptr = np.concatenate([[0], np.cumsum([len(x) for x in lists])]).astype(np.int64)
    return ptr, np.concatenate(lists).astype(np.int32)


def test_nmi_covers_matches_oracle(orc, ctx):
    from paper_1301_0955_gb300 import mscd

    rng = np.random.default_rng(21)
    for trial in range(40):
        n = int(rng.integers(5, 400))
        a = random_cover(rng, n, int(rng.integers(1, 12)), trial % 3 != 0)
        b = random_cover(rng, n, int(rng.integers(1, 12)), trial % 2 == 0)
        want = orc.nmi(n, a[0], a[1], b[0], b[1])
        got = ctx.nmi_covers(n, a, b)
        assert got == pytest.approx(want, abs=1e-12), trial
        assert ctx.nmi_covers(n, a, a) == pytest.approx(1.0, abs=1e-12)
    bad = (np.array([0, 2], np.int64), np.array([3, 1], np.int32))  # not ascending
    with pytest.raises(mscd.MscdError):
        ctx.nmi_covers(10, bad, bad)


def mixed_cover(rng, n):
    """Communities of small (< n/10), medium (n/4..n/2) and large (n/2..n)
    sizes, sometimes with a two-block partition added: disjoint pairs with
    |A| + |B| > n/2 occur with either side small, or both medium."""
    lists = []
    for _ in range(int(rng.integers(1, 8))):
        kind = int(rng.integers(0, 3))
        m = [int(rng.integers(1, max(2, n // 10))), int(rng.integers(n // 4, max(n // 4 + 1, n // 2))),
             int(rng.integers(n // 2, n))][kind]
        lists.append(np.unique(rng.choice(n, max(1, min(m, n)), replace=False)))
    if rng.random() < 0.5:
        perm = rng.permutation(n)
        cut = int(rng.integers(1, n))
        lists += [np.sort(perm[:cut]), np.sort(perm[cut:])]
    uniq = []
    for x in lists:
        if not any(len(x) == len(y) and np.array_equal(x, y) for y in uniq):
            uniq.append(x)
    ptr = np.concatenate([[0], np.cumsum([len(x) for x in uniq])]).astype(np.int64)
    return ptr, np.concatenate(uniq).astype(np.int32)


def test_nmi_covers_disjoint_pairs(orc, ctx):
    """Admitted disjoint pairs of every size combination (a pair needs only
    |A| + |B| > n/2): the device must find each, as the dense definition does."""
    rng = np.random.default_rng(1)
    for trial in range(120):
        n = int(rng.integers(10, 300))
        a, b = mixed_cover(rng, n), mixed_cover(rng, n)
        want = orc.nmi(n, a[0], a[1], b[0], b[1])
        assert ctx.nmi_covers(n, a, b) == pytest.approx(want, abs=1e-12), trial
