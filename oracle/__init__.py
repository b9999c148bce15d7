"""ctypes front end of the CPU oracle (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never does.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

i64p = C.POINTER(C.c_int64)
i32p = C.POINTER(C.c_int32)
f64p = C.POINTER(C.c_double)
f32p = C.POINTER(C.c_float)

OK, EINVAL, ENOTSYM, ESELFLOOP, EDUP, ERANGE = 0, -1, -2, -3, -4, -5
ETIMEOUT, ESMALL, EUNDECIDED, EUNSORTED, EWEIGHT = -8, -9, -10, -11, -12

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_graph_create.argtypes = [C.c_int64, i64p, i32p, f32p, C.POINTER(C.c_void_p)]
        L.orc_graph_destroy.argtypes = [C.c_void_p]
        L.orc_graph_info.argtypes = [C.c_void_p, i64p, i64p, i32p, i64p]
        L.orc_graph_degrees.argtypes = [C.c_void_p, i64p]
        L.orc_graph_weights.argtypes = [C.c_void_p, i64p]
        L.orc_grow.argtypes = [C.c_void_p, C.c_int32, C.c_double, C.c_int64, i32p, C.c_int64, i64p, f64p, i64p]
        L.orc_run.argtypes = [C.c_void_p, f64p, C.c_int32, i32p, C.c_int64, C.c_int64, C.c_int,
                              C.POINTER(C.c_void_p)]
        L.orc_run_init.argtypes = [C.c_void_p, f64p, C.c_int32, i32p, C.c_int64, i64p, i32p, C.c_int64, C.c_int,
                                   C.POINTER(C.c_void_p)]
        L.orc_result_destroy.argtypes = [C.c_void_p]
        L.orc_full.argtypes = [C.c_void_p, f64p, C.c_int32, C.c_int, i32p, i64p, i32p, C.c_int64, C.c_double,
                               C.c_int64, C.POINTER(C.c_void_p)]
        L.orc_full_destroy.argtypes = [C.c_void_p]
        L.orc_full_sizes.argtypes = [C.c_void_p, C.c_int32, i64p, i64p, i64p, i64p]
        L.orc_full_get.argtypes = [C.c_void_p, C.c_int32, i64p, i32p, i32p, f64p]
        L.orc_full_n_seeds.argtypes = [C.c_void_p, i32p]
        L.orc_full_n_seeds.restype = C.c_int64
        L.orc_result_sizes.argtypes = [C.c_void_p, i64p]
        L.orc_result_get.argtypes = [C.c_void_p, i64p, i32p, f64p, i64p]
        L.orc_sign_delta.argtypes = [C.c_int64] * 4 + [C.c_double, C.POINTER(C.c_int)]
        L.orc_add_test.argtypes = [C.c_int64] * 4 + [C.c_double]
        L.orc_remove_test.argtypes = [C.c_int64] * 4 + [C.c_double]
        L.orc_priority_cmp.argtypes = [C.c_int64, C.c_int64, C.c_int32, C.c_int64, C.c_int64, C.c_int32, C.c_double]
        L.orc_fitness.argtypes = [C.c_int64, C.c_int64, C.c_double, C.c_int32]
        L.orc_fitness.restype = C.c_double
        L.orc_dedup.argtypes = [C.c_int64, i64p, i32p, i64p, i32p, i64p]
        L.orc_nmi.argtypes = [C.c_int64, C.c_int64, i64p, i32p, C.c_int64, i64p, i32p]
        L.orc_nmi.restype = C.c_double
        L.orc_nmi_indexed.argtypes = [C.c_int64, C.c_int64, i64p, i32p, C.c_int64, i64p, i32p, C.c_int]
        L.orc_nmi_indexed.restype = C.c_double
        L.orc_window_means.argtypes = [f64p, C.c_int32, C.c_int32, f64p]
        L.orc_scales_logspaced.argtypes = [C.c_double, C.c_double, C.c_int32, f64p]
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


MAX_ROUNDS = 1_000_000


class Graph:
    """Validated graph with exact fixed-point weights.  ``status`` is 0 or an error code."""

    def __init__(self, n, row_ptr, col, w=None):
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.w = None if w is None else np.ascontiguousarray(w, dtype=np.float32)
        h = C.c_void_p()
        self.status = lib().orc_graph_create(int(n), _p(self.row_ptr, i64p), _p(self.col, i32p),
                                             None if self.w is None else _p(self.w, f32p), C.byref(h))
        self.h = h if self.status == OK else None
        self.n = int(n)

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.orc_graph_destroy(self.h)
            self.h = None

    def info(self):
        n, nnz, vol = C.c_int64(), C.c_int64(), C.c_int64()
        ue = C.c_int32()
        lib().orc_graph_info(self.h, C.byref(n), C.byref(nnz), C.byref(ue), C.byref(vol))
        return dict(n=n.value, nnz=nnz.value, unit_exp=ue.value, volume=vol.value)

    def degrees(self):
        k = np.zeros(self.n, np.int64)
        lib().orc_graph_degrees(self.h, _p(k, i64p))
        return k

    def weights_fixed(self):
        w = np.zeros(len(self.col), np.int64)
        lib().orc_graph_weights(self.h, _p(w, i64p))
        return w


STAT_FIELDS = ("edges_scanned", "adds", "removes", "rounds", "K", "V", "slow", "undecided")


def grow(g: Graph, seed: int, alpha: float, max_rounds: int = MAX_ROUNDS):
    """One unit: returns (members sorted int32, f, stats dict, status)."""
    cap = max(g.n, 1)
    buf = np.zeros(cap, np.int32)
    ln = C.c_int64()
    f = C.c_double()
    st = np.zeros(8, np.int64)
    rc = lib().orc_grow(g.h, int(seed), float(alpha), int(max_rounds), _p(buf, i32p), cap, C.byref(ln),
                        C.byref(f), _p(st, i64p))
    return buf[: ln.value].copy(), f.value, dict(zip(STAT_FIELDS, st.tolist())), rc


def run(g: Graph, alphas, seeds=None, threads: int = 1, max_rounds: int = MAX_ROUNDS, init=None):
    """All units, scale-major.  Returns (status, ptr, nodes, f, stats[U,8]).
    init: optional (ptr int64[n_seeds+1], nodes int32) initial members per seed."""
    alphas = np.ascontiguousarray(alphas, dtype=np.float64)
    seeds = np.arange(g.n, dtype=np.int32) if seeds is None else np.ascontiguousarray(seeds, dtype=np.int32)
    h = C.c_void_p()
    if init is None:
        rc = lib().orc_run(g.h, _p(alphas, f64p), len(alphas), _p(seeds, i32p), len(seeds), int(max_rounds),
                           int(threads), C.byref(h))
    else:
        iptr = np.ascontiguousarray(init[0], np.int64)
        inodes = np.ascontiguousarray(init[1], np.int32)
        if len(inodes) == 0:
            inodes = np.zeros(1, np.int32)
        rc = lib().orc_run_init(g.h, _p(alphas, f64p), len(alphas), _p(seeds, i32p), len(seeds), _p(iptr, i64p),
                                _p(inodes, i32p), int(max_rounds), int(threads), C.byref(h))
    if not h.value:
        return rc, None, None, None, None
    U = len(alphas) * len(seeds)
    lens = np.zeros(U, np.int64)
    lib().orc_result_sizes(h, _p(lens, i64p))
    ptr = np.zeros(U + 1, np.int64)
    nodes = np.zeros(int(lens.sum()), np.int32)
    f = np.zeros(U, np.float64)
    st = np.zeros((U, 8), np.int64)
    lib().orc_result_get(h, _p(ptr, i64p), _p(nodes, i32p), _p(f, f64p), _p(st, i64p))
    lib().orc_result_destroy(h)
    return rc, ptr, nodes, f, st


def sign_delta(a1, a2, b1, b2, alpha):
    """(sign, path); sign 99 = undecided."""
    p = C.c_int()
    s = lib().orc_sign_delta(int(a1), int(a2), int(b1), int(b2), float(alpha), C.byref(p))
    return s, p.value


def add_test(K, V, d, k, alpha):
    return lib().orc_add_test(int(K), int(V), int(d), int(k), float(alpha))


def remove_test(K, V, d, k, alpha):
    return lib().orc_remove_test(int(K), int(V), int(d), int(k), float(alpha))


def priority_cmp(d1, k1, id1, d2, k2, id2, alpha):
    return lib().orc_priority_cmp(int(d1), int(k1), int(id1), int(d2), int(k2), int(id2), float(alpha))


def fitness(K, V, alpha, unit_exp=0):
    return lib().orc_fitness(int(K), int(V), float(alpha), int(unit_exp))


def dedup(ptr, nodes):
    """Returns (n_comms, unit2comm int32[U], comm_first_unit int64[n_comms])."""
    ptr = np.ascontiguousarray(ptr, dtype=np.int64)
    nodes = np.ascontiguousarray(nodes, dtype=np.int32)
    U = len(ptr) - 1
    u2c = np.zeros(max(U, 1), np.int32)
    first = np.zeros(max(U, 1), np.int64)
    nc = C.c_int64()
    lib().orc_dedup(U, _p(ptr, i64p), _p(nodes, i32p), C.byref(nc), _p(u2c, i32p), _p(first, i64p))
    return nc.value, u2c[:U].copy(), first[: nc.value].copy()


def nmi(n, xptr, xnodes, yptr, ynodes):
    xptr = np.ascontiguousarray(xptr, dtype=np.int64)
    yptr = np.ascontiguousarray(yptr, dtype=np.int64)
    xnodes = np.ascontiguousarray(xnodes, dtype=np.int32)
    ynodes = np.ascontiguousarray(ynodes, dtype=np.int32)
    return lib().orc_nmi(int(n), len(xptr) - 1, _p(xptr, i64p), _p(xnodes, i32p), len(yptr) - 1,
                         _p(yptr, i64p), _p(ynodes, i32p))


def nmi_indexed(n, xptr, xnodes, yptr, ynodes, threads=1):
    """The same overlapping NMI as nmi(), with intersection sizes counted
    through a node -> communities index (for covers of many large
    communities); equal to nmi() bit for bit."""
    xptr = np.ascontiguousarray(xptr, dtype=np.int64)
    yptr = np.ascontiguousarray(yptr, dtype=np.int64)
    xnodes = np.ascontiguousarray(xnodes, dtype=np.int32)
    ynodes = np.ascontiguousarray(ynodes, dtype=np.int32)
    if len(xnodes) == 0:
        xnodes = np.zeros(1, np.int32)
    if len(ynodes) == 0:
        ynodes = np.zeros(1, np.int32)
    return lib().orc_nmi_indexed(int(n), len(xptr) - 1, _p(xptr, i64p), _p(xnodes, i32p), len(yptr) - 1,
                                 _p(yptr, i64p), _p(ynodes, i32p), int(threads))


def window_means(nmi_succ, S, p):
    a = np.ascontiguousarray(nmi_succ, dtype=np.float64)
    if a.size == 0:
        a = np.zeros(1, np.float64)
    out = np.zeros(S, np.float64)
    rc = lib().orc_window_means(_p(a, f64p), int(S), int(p), _p(out, f64p))
    assert rc == OK
    return out


def scales_logspaced(vmin, a, x):
    out = np.zeros(max(x, 1), np.float64)
    rc = lib().orc_scales_logspaced(float(vmin), float(a), int(x), _p(out, f64p))
    return rc, out


def unique_communities(ptr, nodes):
    """Dedup helper: (comm_ptr, comm_nodes, unit2comm, first_unit) for one scale."""
    nc, u2c, first = dedup(ptr, nodes)
    cptr = np.zeros(nc + 1, np.int64)
    for c, u in enumerate(first):
        cptr[c + 1] = cptr[c] + (ptr[u + 1] - ptr[u])
    cnodes = np.zeros(int(cptr[-1]), np.int32)
    for c, u in enumerate(first):
        cnodes[cptr[c]:cptr[c + 1]] = nodes[ptr[u]:ptr[u + 1]]
    return cptr, cnodes, u2c, first


def full(g: Graph, alphas, seed_rule=1, prio=None, init=None, eta=0.5, max_iters=1000):
    """The full method of Alg. 2 (seed rules, growth with the overlap pre-test,
    check and merge, carried over from scale to scale).  prio: int32[n] order
    of the seed candidates (lower first); init: optional (ptr, nodes) initial
    communities.  Returns (status, initial seeds, [per scale dict(ptr, nodes,
    seeds, f, iterations, merges)])."""
    alphas = np.ascontiguousarray(alphas, np.float64)
    h = C.c_void_p()
    if init is None:
        prio = np.ascontiguousarray(prio if prio is not None else np.arange(g.n), np.int32)
        rc = lib().orc_full(g.h, _p(alphas, f64p), len(alphas), int(seed_rule), _p(prio, i32p), None, None, 0,
                            float(eta), int(max_iters), C.byref(h))
    else:
        iptr = np.ascontiguousarray(init[0], np.int64)
        inodes = np.ascontiguousarray(init[1], np.int32)
        dummy = np.zeros(1, np.int32)
        rc = lib().orc_full(g.h, _p(alphas, f64p), len(alphas), 0, _p(dummy, i32p), _p(iptr, i64p),
                            _p(inodes if len(inodes) else dummy, i32p), len(iptr) - 1, float(eta), int(max_iters),
                            C.byref(h))
    if not h.value:
        return rc, None, None
    ns = lib().orc_full_n_seeds(h, None)
    seeds0 = np.zeros(max(ns, 1), np.int32)
    lib().orc_full_n_seeds(h, _p(seeds0, i32p))
    out = []
    for s in range(len(alphas)):
        nc, nn, it, mg = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        if lib().orc_full_sizes(h, s, C.byref(nc), C.byref(nn), C.byref(it), C.byref(mg)) != 0:
            break
        ptr = np.zeros(nc.value + 1, np.int64)
        nodes = np.zeros(max(nn.value, 1), np.int32)
        sd = np.zeros(max(nc.value, 1), np.int32)
        f = np.zeros(max(nc.value, 1), np.float64)
        lib().orc_full_get(h, s, _p(ptr, i64p), _p(nodes, i32p), _p(sd, i32p), _p(f, f64p))
        out.append(dict(ptr=ptr, nodes=nodes[:nn.value], seeds=sd[:nc.value], f=f[:nc.value],
                        iterations=it.value, merges=mg.value))
    lib().orc_full_destroy(h)
    return rc, seeds0[:ns], out
