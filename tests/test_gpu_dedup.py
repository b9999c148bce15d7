"""GPU: dedup's exact path for lists that share a hash.

Equal member lists have equal 64-bit hashes, and lists that differ almost
never do, so on real workloads dedup's exact comparison and regrouping of
colliding lists have nothing to do.  A testing parameter keeps only a few
bits of every list hash, so that most hash groups mix different lists and
the regrouping decides almost every community; the result must still be the
oracle's dedup (map-based, no hashing) and the stability the oracle's NMI.
"""
import numpy as np
import pytest

from paper_1301_0955_gb300 import synth

pytestmark = pytest.mark.gpu

NMI_ATOL = 1e-12


@pytest.fixture(scope="module")
def mscd_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1301_0955_gb300 import build, mscd

    build.build()
    return mscd


@pytest.mark.parametrize("bits", [1, 3, 6])
def test_dedup_with_colliding_hashes(orc, mscd_mod, bits):
    mscd = mscd_mod
    g = synth.config_graph(0)  # 1,000-node planted partition, every seed, 8 scales
    G = orc.Graph(g.n, g.row_ptr, g.col)
    rc, alphas = orc.scales_logspaced(0.5, 1.0, 8)
    ctx = mscd.Context(0, list_hash_bits=bits)
    gid = ctx.load_csr(g.n, g.row_ptr, g.col)
    assert ctx.run(gid, alphas) == mscd.OK
    N = g.n
    covers = []
    for s, a in enumerate(alphas):
        rc, optr, onodes, of, ost = orc.run(G, [a], None, threads=8)
        assert rc == 0
        cptr, cnodes, u2c, first = orc.unique_communities(optr, onodes)
        gp, gn, gf, gs2c = ctx.communities(s)
        assert len(gp) - 1 == len(first)
        assert np.array_equal(gp, cptr) and np.array_equal(gn, cnodes), (bits, s)
        assert np.array_equal(gs2c, u2c), (bits, s)
        np.testing.assert_allclose(gf, of[first], rtol=1e-12, atol=0)
        covers.append((cptr, cnodes))
    nmi, w3, w5 = ctx.stability()
    want = np.array([orc.nmi(N, *covers[s], *covers[s + 1]) for s in range(len(alphas) - 1)])
    np.testing.assert_allclose(nmi, want, atol=NMI_ATOL, rtol=0)
    ctx.free_graph(gid)
    ctx.close()


def test_bad_hash_bits_rejected(mscd_mod):
    mscd = mscd_mod
    for bits in (-1, 64):
        with pytest.raises(mscd.MscdError) as e:
            mscd.Context(0, list_hash_bits=bits)
        assert e.value.rc == mscd.EINVAL
