"""The seeded input generators: valid CSR graphs with the stated shapes."""
import numpy as np
import pytest

from paper_1301_0955_gb300 import synth


def check_csr(g):
    n = g.n
    assert g.row_ptr[0] == 0 and g.row_ptr[-1] == len(g.col)
    assert np.all(np.diff(g.row_ptr) >= 0)
    rows = np.repeat(np.arange(n), np.diff(g.row_ptr))
    assert np.all(g.col >= 0) and np.all(g.col < n)
    assert not np.any(rows == g.col)  # no self-loops
    # rows strictly ascending (no repeats)
    inner = np.ones(len(g.col), bool)
    inner[g.row_ptr[:-1][np.diff(g.row_ptr) > 0]] = False
    assert np.all(np.diff(g.col)[inner[1:]] > 0)
    # symmetric (with equal weights)
    key = rows.astype(np.int64) * n + g.col
    rkey = g.col.astype(np.int64) * n + rows
    order, rorder = np.argsort(key), np.argsort(rkey)
    assert np.array_equal(key[order], rkey[rorder])
    if g.w is not None:
        assert np.array_equal(g.w[order], g.w[rorder])
        assert np.all(g.w > 0)


def test_planted_partition_shape():
    g = synth.config_graph(0)
    check_csr(g)
    assert g.n == 1000
    assert len(np.unique(g.labels[0])) == 20 and len(np.unique(g.labels[1])) == 4
    assert 18 < len(g.col) / g.n < 27  # expected mean degree about 22
    # most edges inside the planted communities
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    inside = np.mean(g.labels[0][rows] == g.labels[0][g.col])
    assert inside > 0.6


def test_lfr_style_generator():
    g = synth.hierarchical_lfr(20_000, 20, 200, 2.5, 1.5, (20, 1000), (0.3, 0.1), seed=3)
    check_csr(g)
    deg = np.diff(g.row_ptr)
    assert deg.max() <= 200 and 12 < deg.mean() < 22
    micro, macro = g.labels
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    # mixing: about 30% of the stubs leave the micro community, about 10% the macro one
    leave_micro = np.mean(micro[rows] != micro[g.col])
    leave_macro = np.mean(macro[rows] != macro[g.col])
    assert 0.2 < leave_micro < 0.4 and 0.05 < leave_macro < 0.15
    sizes = np.bincount(micro)
    assert sizes[sizes > 0].min() >= 10


def test_weighted_and_deterministic():
    a = synth.hierarchical_lfr(3000, 20, 150, 2.5, 1.5, (20, 500), (0.3, 0.2, 0.1), weights=(0.5, 2.0), seed=18)
    b = synth.hierarchical_lfr(3000, 20, 150, 2.5, 1.5, (20, 500), (0.3, 0.2, 0.1), weights=(0.5, 2.0), seed=18)
    check_csr(a)
    assert a.w.dtype == np.float32 and a.w.min() >= 0.5 and a.w.max() <= 2.0
    assert np.array_equal(a.col, b.col) and np.array_equal(a.w, b.w) and len(a.labels) == 3


def test_uneven_batch_and_queries():
    specs = synth.uneven_batch_specs(256, seed=4)
    ns = np.array([s["n"] for s in specs])
    assert ns.min() >= 1000 and ns.max() <= 200_000
    assert all(10 <= s["mean_deg"] <= 40 and 0.2 <= s["mixing"][0] <= 0.4 for s in specs)
    # log-uniform sizes: about half below the geometric mean of the range
    assert 0.35 < np.mean(ns < np.sqrt(1000 * 200_000)) < 0.65
    q = synth.serving_queries(500, [5000, 6000, 7000, 8000], n_scales=16, max_seeds=4096, seed=7)
    assert len(q) == 500
    for g, s, seeds in q:
        assert 0 <= g < 4 and 0 <= s < 16 and 1 <= len(seeds) <= 4096
        assert len(np.unique(seeds)) == len(seeds)
    assert len({g for g, _, _ in q}) == 4 and len({s for _, s, _ in q}) == 16


@pytest.mark.slow
def test_benchmark_graph_shape():
    g = synth.config_graph(1)
    check_csr(g)
    assert g.n == 100_000 and len(g.col) == 1_868_066
