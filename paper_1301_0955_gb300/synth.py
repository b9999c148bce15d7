"""Seeded synthetic graphs shaped like the paper's generated multi-scale networks.

The paper (Sec. 4) measures on hierarchical benchmark networks of
Lancichinetti et al. (micro communities nested in macro communities, mixing
mu_1 / mu_2 per level, power-law degrees and community sizes).  Those
instances are not available, so these generators stand in for them.  This
module holds only input generation: no part of the community-growth method.

Recipes (all draws from numpy's PCG64 with the stated seed):

* ``planted_partition``: every node pair is an independent Bernoulli draw
  whose probability depends on whether the two nodes share the lowest-level
  community, only the super-group, or nothing.
* ``hierarchical_lfr``: power-law degrees on [k_min, k_max] with k_min picked
  so the mean is closest to the target; micro-community sizes power-law on
  [s_min, s_max]; micro communities grouped into the next level by drawing
  2..6 children per group (repeated for every extra level); each node's stubs
  are split by the per-level mixing fractions (``mixing[l]`` = fraction of a
  node's stubs that leave its level-l community); stubs of each class are
  paired uniformly at random inside their group (configuration model);
  self-loops and repeated pairs are dropped.  Nodes are placed in
  communities level by level of internal-degree need, so that a node's
  internal stubs fit inside its micro community.
* weights, when asked for, are float32 draws uniform on [w_lo, w_hi], one per
  undirected edge (the same value in both directions).
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class CSRGraph:
    n: int
    row_ptr: np.ndarray  # int64[n+1]
    col: np.ndarray  # int32[E], rows ascending
    w: np.ndarray | None  # float32[E] or None
    labels: list  # per level (finest first): int32[n] community ids
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])


def to_csr(n: int, u: np.ndarray, v: np.ndarray, w: np.ndarray | None = None):
    """Undirected edge list (u != v, each pair once) -> symmetric sorted CSR."""
    u = np.asarray(u, np.int64)
    v = np.asarray(v, np.int64)
    src = np.concatenate([u, v])
    dst = np.concatenate([v, u])
    order = np.argsort(src * n + dst, kind="stable")
    src, dst = src[order], dst[order]
    row_ptr = np.zeros(n + 1, np.int64)
    np.add.at(row_ptr, src + 1, 1)
    np.cumsum(row_ptr, out=row_ptr)
    ww = None
    if w is not None:
        ww = np.concatenate([w, w]).astype(np.float32)[order]
    return row_ptr, dst.astype(np.int32), ww


def _unique_pairs(n, a, b):
    a = np.asarray(a, np.int64)
    b = np.asarray(b, np.int64)
    keep = a != b
    a, b = a[keep], b[keep]
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    key = np.unique(lo * n + hi)
    return key // n, key % n


def planted_partition(n_super=4, n_comm=5, comm_size=50, p_comm=0.3, p_super=0.03, p_out=0.002, seed=0,
                      name="planted") -> CSRGraph:
    """Two-level planted partition: n = n_super * n_comm * comm_size nodes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = n_super * n_comm * comm_size
    comm = np.arange(n) // comm_size
    sup = comm // n_comm
    iu, ju = np.triu_indices(n, 1)
    p = np.where(comm[iu] == comm[ju], p_comm, np.where(sup[iu] == sup[ju], p_super, p_out))
    keep = rng.random(iu.size) < p
    rp, col, _ = to_csr(n, iu[keep], ju[keep])
    return CSRGraph(n, rp, col, None, [comm.astype(np.int32), sup.astype(np.int32)], name)


def _powerlaw_ints(rng, lo, hi, tau, size):
    ks = np.arange(lo, hi + 1, dtype=np.float64)
    p = ks ** (-tau)
    cdf = np.cumsum(p / p.sum())
    return (lo + np.searchsorted(cdf, rng.random(size), side="right")).astype(np.int64).clip(lo, hi)


def _degree_kmin(mean, kmax, tau):
    best, best_err = 1, None
    for kmin in range(1, kmax + 1):
        ks = np.arange(kmin, kmax + 1, dtype=np.float64)
        p = ks ** (-tau)
        m = (ks * p).sum() / p.sum()
        err = abs(m - mean)
        if best_err is None or err < best_err:
            best, best_err = kmin, err
    return best


def _pair_within_groups(rng, stubs, group):
    """Configuration-model pairing of stubs (node ids) inside each group."""
    if stubs.size == 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    order = np.lexsort((rng.random(stubs.size), group))
    s, g = stubs[order], group[order]
    # position inside the group run
    starts = np.flatnonzero(np.r_[True, g[1:] != g[:-1]])
    run_id = np.repeat(np.arange(starts.size), np.diff(np.r_[starts, g.size]))
    pos = np.arange(g.size) - starts[run_id]
    first = (pos % 2 == 0)
    idx = np.flatnonzero(first)
    idx = idx[idx + 1 < g.size]
    idx = idx[g[idx + 1] == g[idx]]
    return s[idx], s[idx + 1]


def _split_stubs(rng, k, mixing):
    """Split each node's degree into per-level stub classes (finest first + outside)."""
    L = len(mixing)
    fr = [1.0 - mixing[0]] + [mixing[l] - mixing[l + 1] for l in range(L - 1)] + [mixing[-1]]
    x = k[:, None] * np.asarray(fr)[None, :]
    base = np.floor(x)
    rem = (k - base.sum(1)).astype(np.int64)
    # randomised rounding: hand the remaining stubs to classes by fractional part
    frac = x - base
    out = base.astype(np.int64)
    for i in range(int(rem.max()) if rem.size else 0):
        pick = np.argmax(frac + rng.random(frac.shape) * 1e-3, axis=1)
        sel = rem > i
        out[np.flatnonzero(sel), pick[sel]] += 1
        frac[np.flatnonzero(sel), pick[sel]] = -1.0
    return out


def hierarchical_lfr(n, mean_deg, max_deg, tau_deg=2.5, tau_size=1.5, size_range=(20, 1000),
                     mixing=(0.3, 0.1), group_range=(2, 6), weights=None, seed=1, name="lfr") -> CSRGraph:
    """LFR-style hierarchical graph; ``mixing`` finest level first (len = levels)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mixing = tuple(float(m) for m in mixing)
    kmin = _degree_kmin(mean_deg, max_deg, tau_deg)
    k = _powerlaw_ints(rng, kmin, max_deg, tau_deg, n)
    # micro community sizes summing to n
    smin, smax = size_range
    sizes = []
    total = 0
    while total < n:
        s = int(_powerlaw_ints(rng, smin, smax, tau_size, 1)[0])
        sizes.append(s)
        total += s
    sizes[-1] -= total - n
    if sizes[-1] < smin and len(sizes) > 1:
        sizes[-2] += sizes[-1]
        sizes.pop()
    sizes = np.array(sizes, np.int64)
    C = sizes.size
    # place nodes: highest internal need first, each into a random free slot of
    # a community big enough for it
    need = np.ceil((1.0 - mixing[0]) * k).astype(np.int64)
    order_c = np.argsort(-sizes, kind="stable")
    slot_comm = np.repeat(order_c, sizes[order_c])  # slots sorted by community size desc
    slot_size = sizes[slot_comm]
    used = np.zeros(n, bool)
    micro = np.empty(n, np.int64)
    for r in np.unique(need)[::-1]:
        nodes_r = np.flatnonzero(need == r)
        P = int(np.searchsorted(-slot_size, -(r + 1), side="right"))  # slots in comms of size >= r+1
        free = np.flatnonzero(~used[:P])
        if free.size < nodes_r.size:
            free = np.flatnonzero(~used)  # not enough room: take any slot
        pick = rng.choice(free, nodes_r.size, replace=False)
        used[pick] = True
        micro[nodes_r] = slot_comm[pick]
    labels = [micro]
    parent = np.arange(C)
    for _ in range(1, len(mixing)):
        nprev = int(parent.max()) + 1 if labels[-1].size else 0
        perm = rng.permutation(nprev)
        gid = np.empty(nprev, np.int64)
        i, g = 0, 0
        while i < nprev:
            m = int(rng.integers(group_range[0], group_range[1] + 1))
            gid[perm[i:i + m]] = g
            i += m
            g += 1
        labels.append(gid[labels[-1]])
        parent = gid
    # stubs per class and wiring
    cls = _split_stubs(rng, k, mixing)  # [n, L+1]
    us, vs = [], []
    node_ids = np.arange(n, dtype=np.int64)
    for c in range(len(mixing) + 1):
        stubs = np.repeat(node_ids, cls[:, c])
        group = np.zeros(stubs.size, np.int64) if c == len(mixing) else labels[c][stubs]
        a, b = _pair_within_groups(rng, stubs, group)
        us.append(a)
        vs.append(b)
    u, v = _unique_pairs(n, np.concatenate(us), np.concatenate(vs))
    w = None
    if weights is not None:
        w = rng.uniform(weights[0], weights[1], u.size).astype(np.float32)
    rp, col, ww = to_csr(n, u, v, w)
    return CSRGraph(n, rp, col, ww, [lab.astype(np.int32) for lab in labels], name)


def config_graph(idx: int) -> CSRGraph:
    """The five benchmark workloads' graphs (the serving one returns one of its four)."""
    if idx == 0:
        return planted_partition(seed=0, name="planted-1k")
    if idx == 1:
        return hierarchical_lfr(100_000, 20, 200, 2.5, 1.5, (20, 1000), (0.3, 0.1), seed=1, name="lfr-100k")
    if idx == 2:
        return hierarchical_lfr(1_000_000, 30, 300, 2.5, 1.5, (20, 1000), (0.3, 0.2, 0.1),
                                weights=(0.5, 2.0), seed=2, name="lfr-1m-weighted")
    if idx == 4:
        return graph_from_spec(serving_specs()[0])
    raise ValueError(idx)


def serving_specs(n_graphs=4, n=2_000_000, scale_nodes=1.0):
    """The serving graphs: n nodes (times scale_nodes), mean degree 25, max 250,
    three levels with mixing 0.3 / 0.2 / 0.1, unweighted; seeds 5, 6, ..."""
    m = max(100, int(n * scale_nodes))
    return [dict(n=m, mean_deg=25, max_deg=250, tau_deg=2.5, tau_size=1.5, size_range=(20, 1000),
                 mixing=(0.3, 0.2, 0.1), seed=5 + i, name=f"lfr-2m-serving-{i}") for i in range(n_graphs)]


def serving_queries(n_queries, graph_sizes, n_scales=16, max_seeds=4096, seed=7):
    """Query stream: graph uniform, scale index uniform in [0, n_scales), seed
    count uniform in {1..max_seeds}, seeds distinct and uniform over the graph."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n_queries):
        g = int(rng.integers(0, len(graph_sizes)))
        s = int(rng.integers(0, n_scales))
        k = int(rng.integers(1, max_seeds + 1))
        seeds = rng.choice(graph_sizes[g], min(k, graph_sizes[g]), replace=False).astype(np.int32)
        out.append((g, s, seeds))
    return out


def uneven_batch_specs(n_graphs=256, seed=4, n_range=(1_000, 200_000), scale_nodes=1.0):
    """Parameters of the graphs of the uneven batch: node counts log-uniform in
    n_range (times scale_nodes), mean degree uniform in [10, 40], micro mixing
    uniform in [0.2, 0.4] (macro a third of it), two levels."""
    rng = np.random.Generator(np.random.PCG64(seed))
    specs = []
    for i in range(n_graphs):
        n = int(np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1]))) * scale_nodes)
        n = max(n, 100)
        md = float(rng.uniform(10, 40))
        mu = float(rng.uniform(0.2, 0.4))
        specs.append(dict(n=n, mean_deg=md, max_deg=max(4 * int(md), 40), tau_deg=2.5, tau_size=1.5,
                          size_range=(20, 1000), mixing=(mu, mu / 3), seed=1000 + i, name=f"uneven-{i}"))
    return specs


def graph_from_spec(spec):
    return hierarchical_lfr(**spec)


def uneven_batch(n_graphs=256, seed=4, n_range=(1_000, 200_000), scale_nodes=1.0):
    """Many independent two-level graphs of log-uniform size (batching workload)."""
    return [graph_from_spec(sp) for sp in uneven_batch_specs(n_graphs, seed, n_range, scale_nodes)]

