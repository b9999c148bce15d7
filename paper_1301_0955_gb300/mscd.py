"""Thin Python binding of libmscd.so (include/mscd.h): argument marshalling only.

Every function of the C ABI is exposed under its C name; ``Context`` wraps a
context with numpy / torch friendly helpers.  Arrays may be numpy arrays
(host) or CUDA torch tensors (device, passed with MSCD_DEVICE_PTRS).  There
is no fallback: if the library cannot be loaded, import fails.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libmscd.so")

OK = 0
EINVAL, ENOTSYM, ESELFLOOP, EDUP, ERANGE, ENOMEM, EDEVICE = -1, -2, -3, -4, -5, -6, -7
ETIMEOUT, ESMALL, EUNDECIDED, EUNSORTED, EWEIGHT, ENORESULT, EBUSY = -8, -9, -10, -11, -12, -13, -14
Q_QUEUED, Q_RUNNING, Q_DONE = 0, 1, 2
DEVICE_PTRS = 1
SCHED_PERSISTENT = 0
SCHED_PER_SCALE = 1
TUNE_APPLY = 1
TUNE_CACHED = 2
NSTATS = 8
STAT_FIELDS = ("edges_scanned", "adds", "removes", "rounds", "K", "V", "slow", "undecided")

i64p = C.POINTER(C.c_int64)
i32p = C.POINTER(C.c_int32)
f64p = C.POINTER(C.c_double)
f32p = C.POINTER(C.c_float)
vp = C.c_void_p


class mscd_params(C.Structure):
    _fields_ = [("struct_size", C.c_int32), ("warps_per_block", C.c_int32), ("smem_slots", C.c_int32),
                ("blocks_per_sm", C.c_int32), ("mid_slots", C.c_int32), ("global_warps_per_sm", C.c_int32),
                ("global_slots", C.c_int32), ("max_rounds", C.c_int64), ("schedule", C.c_int32),
                ("hash_smem_slots", C.c_int32), ("list_hash_bits", C.c_int32)]


class mscd_serve_params(C.Structure):
    _fields_ = [("struct_size", C.c_int32), ("workers", C.c_int32), ("max_batch_units", C.c_int64),
                ("memory_budget", C.c_int64)]


class mscd_serve_stats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("queries_submitted", "queries_done", "units_done", "batches", "queued",
                                         "in_flight_bytes", "max_in_flight_bytes", "budget_bytes",
                                         "max_concurrent_batches", "overlap_us")]


class mscd_full_params(C.Structure):
    _fields_ = [("struct_size", C.c_int32), ("seed_rule", C.c_int32), ("eta", C.c_double), ("max_iters", C.c_int64)]


class mscd_run_stats(C.Structure):
    _fields_ = [("units", C.c_int64), ("edges_scanned", C.c_int64), ("adds", C.c_int64), ("removes", C.c_int64),
                ("slow_decisions", C.c_int64), ("undecided", C.c_int64), ("overflow_units", C.c_int64),
                ("grow_launches", C.c_int64), ("member_entries", C.c_int64), ("ms_grow", C.c_double),
                ("ms_dedup", C.c_double), ("ms_stability", C.c_double), ("ms_total", C.c_double),
                ("launch_cap", C.c_int32 * 8), ("launch_smem", C.c_int32 * 8), ("launch_units", C.c_int64 * 8),
                ("launch_ms", C.c_double * 8)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if not f.startswith("launch_")}
        n = min(8, self.grow_launches)
        d["launches"] = [dict(cap=self.launch_cap[i], smem=self.launch_smem[i], units=self.launch_units[i],
                              ms=self.launch_ms[i]) for i in range(n)]
        return d


class mscd_cover_shard(C.Structure):
    _fields_ = [("n_seeds", C.c_int64), ("seed_index", i64p), ("seed2comm", i32p), ("n_comms", C.c_int64),
                ("ptr", i64p), ("nodes", i32p), ("fitness", f64p)]


# name -> (restype, argtypes)
SIGNATURES = {
    "mscd_strerror": (C.c_char_p, [C.c_int]),
    "mscd_version": (C.c_int, []),
    "mscd_launch_count": (C.c_int64, []),
    "mscd_create": (C.c_int, [C.POINTER(vp), C.c_int, C.POINTER(mscd_params)]),
    "mscd_destroy": (C.c_int, [vp]),
    "mscd_graph_load_csr": (C.c_int, [vp, C.c_int64, vp, vp, vp, C.c_uint32, i32p]),
    "mscd_graph_free": (C.c_int, [vp, C.c_int32]),
    "mscd_graph_info": (C.c_int, [vp, C.c_int32, i64p, i64p, i32p, i64p]),
    "mscd_graph_degrees": (C.c_int, [vp, C.c_int32, i64p]),
    "mscd_scales_logspaced": (C.c_int, [C.c_double, C.c_double, C.c_int32, f64p]),
    "mscd_run": (C.c_int, [vp, C.c_int32, vp, C.c_int32, vp, C.c_int64, C.c_uint32, vp]),
    "mscd_run_init": (C.c_int, [vp, C.c_int32, vp, C.c_int32, vp, C.c_int64, vp, vp, C.c_uint32, vp]),
    "mscd_get_membership": (C.c_int, [vp, C.c_int32, C.c_int64, i32p, C.c_int64, i64p, f64p]),
    "mscd_get_memberships": (C.c_int, [vp, C.c_int32, i64p, i32p, C.c_int64, f64p, i64p, i64p]),
    "mscd_get_communities": (C.c_int, [vp, C.c_int32, i64p, C.c_int64, i32p, C.c_int64, f64p, i32p, i64p, i64p]),
    "mscd_get_stability": (C.c_int, [vp, f64p, f64p, f64p]),
    "mscd_get_stability_part": (C.c_int, [vp, C.c_int32, f64p, f64p, f64p]),
    "mscd_autotune": (C.c_int, [vp, C.c_int32, f64p, C.c_int32, C.c_int64, C.c_uint32, C.POINTER(mscd_params), f64p]),
    "mscd_full_run": (C.c_int, [vp, C.c_int32, f64p, C.c_int32, i32p, i64p, i32p, C.c_int64,
                                C.POINTER(mscd_full_params), vp]),
    "mscd_full_get_seeds": (C.c_int, [vp, i32p, C.c_int64, i64p]),
    "mscd_full_get_scale": (C.c_int, [vp, C.c_int32, i64p, C.c_int64, i32p, C.c_int64, i32p, f64p, i64p, i64p]),
    "mscd_full_get_info": (C.c_int, [vp, C.c_int32, i64p, i64p, i64p, f64p]),
    "mscd_serve_start": (C.c_int, [vp, C.POINTER(mscd_serve_params)]),
    "mscd_serve_stop": (C.c_int, [vp]),
    "mscd_query_submit": (C.c_int, [vp, C.c_int32, i32p, C.c_int32, C.c_double, C.POINTER(C.c_uint64)]),
    "mscd_query_poll": (C.c_int, [vp, C.c_uint64, i32p]),
    "mscd_query_wait": (C.c_int, [vp, C.c_uint64, C.c_int64, i32p]),
    "mscd_query_result": (C.c_int, [vp, C.c_uint64, i64p, i32p, C.c_int64, f64p, i64p, f64p]),
    "mscd_serve_get_stats": (C.c_int, [vp, C.POINTER(mscd_serve_stats)]),
    "mscd_serve_batch_intervals": (C.c_int, [vp, f64p, f64p, C.c_int64, i64p]),
    "mscd_graph_union": (C.c_int, [vp, i32p, C.c_int32, i32p]),
    "mscd_graph_parts": (C.c_int, [vp, C.c_int32, i64p, C.c_int32, i32p]),
    "mscd_get_run_stats": (C.c_int, [vp, C.POINTER(mscd_run_stats)]),
    "mscd_last_error": (C.c_char_p, [vp]),
    "mscd_nmi_covers": (C.c_int, [vp, C.c_int64, i64p, i32p, C.c_int64, i64p, i32p, C.c_int64, f64p]),
    "mscd_window_means": (C.c_int, [f64p, C.c_int32, C.c_int32, f64p]),
    "mscd_merge_shards": (C.c_int, [C.POINTER(mscd_cover_shard), C.c_int32, C.c_int64, i64p, C.c_int64, i32p,
                                    C.c_int64, f64p, i32p, i64p, i64p]),
    "mscd_grow_noalloc": (C.c_int, [vp, C.c_int32, f64p, C.c_int32, vp, C.c_int64, vp, C.c_int64, vp, vp, vp, vp,
                                    vp, vp, i64p, vp]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the library (built by ``build.py``); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError("libmscd.so not built: run paper_1301_0955_gb300/build.py (%s)" % path)
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def strerror(rc: int) -> str:
    return load().mscd_strerror(rc).decode()


class MscdError(RuntimeError):
    def __init__(self, rc, what=""):
        super().__init__("%s: %s (%d)" % (what, strerror(rc), rc))
        self.rc = rc


def _check(rc, what):
    if rc != OK:
        raise MscdError(rc, what)
    return rc


def _ptr(a):
    """(address, is_device) of a numpy array or torch tensor; None -> (None, False)."""
    if a is None:
        return None, False
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays passed to libmscd must be C-contiguous")
        return a.ctypes.data, False
    # torch tensor
    if not a.is_contiguous():
        raise ValueError("tensors passed to libmscd must be contiguous")
    return a.data_ptr(), bool(a.is_cuda)


def scales_logspaced(vmin: float, a: float, x: int) -> np.ndarray:
    out = np.zeros(max(x, 1), np.float64)
    _check(load().mscd_scales_logspaced(vmin, a, x, out.ctypes.data_as(f64p)), "mscd_scales_logspaced")
    return out


def window_means(nmi_succ, n_scales: int, p: int) -> np.ndarray:
    """mscd_window_means: means of successive-scale NMI over windows of p scales."""
    a = np.ascontiguousarray(nmi_succ, np.float64)
    out = np.zeros(max(n_scales, 1), np.float64)
    _check(load().mscd_window_means(a.ctypes.data_as(f64p) if len(a) else None, n_scales, p,
                                    out.ctypes.data_as(f64p)), "mscd_window_means")
    return out


def merge_shards(shards, n_seeds_total: int):
    """mscd_merge_shards on host arrays.  shards: a list of dicts with
    seed_index (int64), seed2comm (int32), ptr (int64), nodes (int32) and
    optionally fitness (float64), e.g. ``Context.communities`` of each GPU's
    share of the seeds.  Returns (ptr, nodes, fitness or None, seed2comm)."""
    keep = []
    arr = (mscd_cover_shard * max(len(shards), 1))()
    with_f = all(s.get("fitness") is not None for s in shards)
    for i, s in enumerate(shards):
        si = np.ascontiguousarray(s["seed_index"], np.int64)
        s2c = np.ascontiguousarray(s["seed2comm"], np.int32)
        ptr = np.ascontiguousarray(s["ptr"], np.int64)
        nodes = np.ascontiguousarray(s["nodes"], np.int32)
        f = np.ascontiguousarray(s["fitness"], np.float64) if with_f else None
        keep += [si, s2c, ptr, nodes, f]
        arr[i] = mscd_cover_shard(len(si), si.ctypes.data_as(i64p), s2c.ctypes.data_as(i32p), len(ptr) - 1,
                                  ptr.ctypes.data_as(i64p), nodes.ctypes.data_as(i32p),
                                  f.ctypes.data_as(f64p) if f is not None else None)
    nc, nn = C.c_int64(), C.c_int64()
    rc = load().mscd_merge_shards(arr, len(shards), n_seeds_total, None, 0, None, 0, None, None, C.byref(nc),
                                  C.byref(nn))
    if rc not in (OK, ESMALL):
        raise MscdError(rc, "mscd_merge_shards")
    ptr = np.zeros(nc.value + 1, np.int64)
    nodes = np.zeros(max(nn.value, 1), np.int32)
    f = np.zeros(max(nc.value, 1), np.float64) if with_f else None
    s2c = np.zeros(max(n_seeds_total, 1), np.int32)
    _check(load().mscd_merge_shards(arr, len(shards), n_seeds_total, ptr.ctypes.data_as(i64p), nc.value + 1,
                                    nodes.ctypes.data_as(i32p), nn.value,
                                    f.ctypes.data_as(f64p) if with_f else None, s2c.ctypes.data_as(i32p),
                                    C.byref(nc), C.byref(nn)), "mscd_merge_shards")
    return ptr, nodes[: nn.value], (f[: nc.value] if with_f else None), s2c[:n_seeds_total]


def shard_seeds(n_seeds: int, rank: int, world: int) -> np.ndarray:
    """Indices into a job's seed list of one process's share when the seeds are
    split across `world` GPUs: every world-th seed from `rank` (neighbouring
    seeds, often of one community and of similar cost, go to different GPUs)."""
    return np.arange(rank, n_seeds, world, dtype=np.int64)


def merge_gathered(gathered, n_seeds_total: int):
    """gathered[r][s]: rank r's shard of scale s (a dict for merge_shards).
    Returns per scale the merged (ptr, nodes, fitness, seed2comm)."""
    n_scales = len(gathered[0]) if gathered else 0
    return [merge_shards([g[s] for g in gathered], n_seeds_total) for s in range(n_scales)]


class Context:
    """One mscd context on one device."""

    def __init__(self, device: int = 0, smem_slots: int = 0, blocks_per_sm: int = 0, max_rounds: int = 0,
                 warps_per_block: int = 0, mid_slots: int = 0, global_warps_per_sm: int = 0,
                 global_slots: int = 0, schedule: int = 0, hash_smem_slots: int = 0, list_hash_bits: int = 0):
        L = load()
        p = mscd_params(C.sizeof(mscd_params), warps_per_block, smem_slots, blocks_per_sm, mid_slots,
                        global_warps_per_sm, global_slots, max_rounds, schedule, hash_smem_slots, list_hash_bits)
        h = vp()
        _check(L.mscd_create(C.byref(h), device, C.byref(p)), "mscd_create")
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            load().mscd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- graphs
    def load_csr(self, n, row_ptr, col, w=None) -> int:
        """Returns the graph id; raises MscdError with the check's status code."""
        rp, dev = _ptr(row_ptr)
        cp, dev2 = _ptr(col)
        wp, dev3 = _ptr(w)
        if dev != dev2 or (w is not None and dev3 != dev):
            raise ValueError("row_ptr, col and w must all be host or all be device arrays")
        gid = C.c_int32(-1)
        rc = load().mscd_graph_load_csr(self.h, int(n), rp, cp, wp, DEVICE_PTRS if dev else 0, C.byref(gid))
        _check(rc, "mscd_graph_load_csr")
        return gid.value

    def try_load_csr(self, n, row_ptr, col, w=None):
        """(status, graph id or -1) without raising."""
        try:
            return OK, self.load_csr(n, row_ptr, col, w)
        except MscdError as e:
            return e.rc, -1

    def free_graph(self, gid: int):
        _check(load().mscd_graph_free(self.h, gid), "mscd_graph_free")

    def autotune(self, gid: int, alphas, n_sample: int = 0, apply: bool = True, cached: bool = False):
        """Pick the fastest slot classes and residency on a seeded sample (see
        mscd_autotune); returns (params dict, growth ms on the sample)."""
        alphas = np.ascontiguousarray(alphas, np.float64)
        p = mscd_params()
        ms = C.c_double()
        flags = (TUNE_APPLY if apply else 0) | (TUNE_CACHED if cached else 0)
        _check(load().mscd_autotune(self.h, gid, alphas.ctypes.data_as(f64p), len(alphas), n_sample, flags,
                                    C.byref(p), C.byref(ms)), "mscd_autotune")
        return {k: getattr(p, k) for k, _ in mscd_params._fields_}, ms.value

    def nmi_covers(self, n: int, a, b) -> float:
        """Overlapping NMI between covers a, b = (ptr, nodes) of n nodes."""
        pa, na = np.ascontiguousarray(a[0], np.int64), np.ascontiguousarray(a[1], np.int32)
        pb, nb = np.ascontiguousarray(b[0], np.int64), np.ascontiguousarray(b[1], np.int32)
        out = C.c_double()
        _check(load().mscd_nmi_covers(self.h, n, pa.ctypes.data_as(i64p), na.ctypes.data_as(i32p), len(pa) - 1,
                                      pb.ctypes.data_as(i64p), nb.ctypes.data_as(i32p), len(pb) - 1, C.byref(out)),
               "mscd_nmi_covers")
        return out.value

    # ---- the full method (Alg. 2)
    def full_run(self, gid: int, alphas, prio=None, init=None, seed_rule: int = 1, eta: float = 0.5,
                 max_iters: int = 0) -> int:
        alphas = np.ascontiguousarray(alphas, np.float64)
        p = mscd_full_params(C.sizeof(mscd_full_params), seed_rule, eta, max_iters)
        if init is None:
            n = self.graph_info(gid)["n"]
            prio = np.ascontiguousarray(prio if prio is not None else np.arange(n), np.int32)
            rc = load().mscd_full_run(self.h, gid, alphas.ctypes.data_as(f64p), len(alphas),
                                      prio.ctypes.data_as(i32p), None, None, 0, C.byref(p), None)
        else:
            iptr = np.ascontiguousarray(init[0], np.int64)
            inodes = np.ascontiguousarray(init[1], np.int32)
            rc = load().mscd_full_run(self.h, gid, alphas.ctypes.data_as(f64p), len(alphas), None,
                                      iptr.ctypes.data_as(i64p), inodes.ctypes.data_as(i32p), len(iptr) - 1,
                                      C.byref(p), None)
        if rc not in (OK, ETIMEOUT, EUNDECIDED):
            raise MscdError(rc, "mscd_full_run")
        self.full_scales = len(alphas)
        return rc

    def full_seeds(self) -> np.ndarray:
        n = C.c_int64()
        rc = load().mscd_full_get_seeds(self.h, None, 0, C.byref(n))
        if rc not in (OK, ESMALL):
            _check(rc, "mscd_full_get_seeds")
        out = np.zeros(max(n.value, 1), np.int32)
        _check(load().mscd_full_get_seeds(self.h, out.ctypes.data_as(i32p), len(out), C.byref(n)),
               "mscd_full_get_seeds")
        return out[: n.value]

    def full_scale(self, s: int) -> dict:
        L = load()
        nc, nn = C.c_int64(), C.c_int64()
        rc = L.mscd_full_get_scale(self.h, s, None, 0, None, 0, None, None, C.byref(nc), C.byref(nn))
        if rc not in (OK, ESMALL):
            _check(rc, "mscd_full_get_scale")
        ptr = np.zeros(nc.value + 1, np.int64)
        nodes = np.zeros(max(nn.value, 1), np.int32)
        seeds = np.zeros(max(nc.value, 1), np.int32)
        f = np.zeros(max(nc.value, 1), np.float64)
        _check(L.mscd_full_get_scale(self.h, s, ptr.ctypes.data_as(i64p), len(ptr), nodes.ctypes.data_as(i32p),
                                     len(nodes), seeds.ctypes.data_as(i32p), f.ctypes.data_as(f64p), C.byref(nc),
                                     C.byref(nn)), "mscd_full_get_scale")
        it, mg, gr = C.c_int64(), C.c_int64(), C.c_int64()
        nmi = C.c_double()
        _check(L.mscd_full_get_info(self.h, s, C.byref(it), C.byref(mg), C.byref(gr), C.byref(nmi)),
               "mscd_full_get_info")
        return dict(ptr=ptr, nodes=nodes[: nn.value], seeds=seeds[: nc.value], f=f[: nc.value],
                    iterations=it.value, merges=mg.value, grown=gr.value, nmi_next=nmi.value)

    # ---- serving
    def serve_start(self, workers: int = 0, max_batch_units: int = 0, memory_budget: int = 0):
        p = mscd_serve_params(C.sizeof(mscd_serve_params), workers, max_batch_units, memory_budget)
        _check(load().mscd_serve_start(self.h, C.byref(p)), "mscd_serve_start")

    def serve_stop(self):
        _check(load().mscd_serve_stop(self.h), "mscd_serve_stop")

    def submit(self, gid: int, seeds, alpha: float) -> int:
        seeds = np.ascontiguousarray(seeds, np.int32)
        q = C.c_uint64()
        _check(load().mscd_query_submit(self.h, gid, seeds.ctypes.data_as(i32p), len(seeds), float(alpha),
                                        C.byref(q)), "mscd_query_submit")
        return q.value

    def poll(self, qid: int) -> int:
        st = C.c_int32()
        _check(load().mscd_query_poll(self.h, qid, C.byref(st)), "mscd_query_poll")
        return st.value

    def wait(self, qid: int, timeout_s: float = 60.0) -> int:
        st = C.c_int32()
        _check(load().mscd_query_wait(self.h, qid, int(timeout_s * 1e6), C.byref(st)), "mscd_query_wait")
        return st.value

    def result(self, qid: int, n_seeds: int):
        """(ptr, nodes, fitness, times_ms, status) of a done query; releases it."""
        L = load()
        nn = C.c_int64()
        times = np.zeros(3, np.float64)
        rc = L.mscd_query_result(self.h, qid, None, None, 0, None, C.byref(nn), None)
        if rc != ESMALL:
            _check(rc, "mscd_query_result")
        ptr = np.zeros(n_seeds + 1, np.int64)
        nodes = np.zeros(max(nn.value, 1), np.int32)
        f = np.zeros(n_seeds, np.float64)
        rc = L.mscd_query_result(self.h, qid, ptr.ctypes.data_as(i64p), nodes.ctypes.data_as(i32p), len(nodes),
                                 f.ctypes.data_as(f64p), C.byref(nn), times.ctypes.data_as(f64p))
        if rc not in (OK, ETIMEOUT, EUNDECIDED):
            raise MscdError(rc, "mscd_query_result")
        return ptr, nodes[: nn.value], f, times, rc

    def serve_stats(self) -> dict:
        st = mscd_serve_stats()
        _check(load().mscd_serve_get_stats(self.h, C.byref(st)), "mscd_serve_get_stats")
        return {k: getattr(st, k) for k, _ in mscd_serve_stats._fields_}

    def batch_intervals(self):
        """(start_ms, end_ms) device intervals of the completed serving batches."""
        n = C.c_int64()
        rc = load().mscd_serve_batch_intervals(self.h, None, None, 0, C.byref(n))
        if rc not in (OK, ESMALL):
            _check(rc, "mscd_serve_batch_intervals")
        a = np.zeros(max(n.value, 1), np.float64)
        b = np.zeros(max(n.value, 1), np.float64)
        rc = load().mscd_serve_batch_intervals(self.h, a.ctypes.data_as(f64p), b.ctypes.data_as(f64p), len(a),
                                               C.byref(n))
        if rc not in (OK, ESMALL):  # batches may have completed in between
            _check(rc, "mscd_serve_batch_intervals")
        m = min(n.value, len(a))
        return a[:m], b[:m]

    def graph_union(self, gids) -> int:
        """Disjoint union of resident graphs as one resident graph (batching)."""
        ids = np.ascontiguousarray(gids, np.int32)
        out = C.c_int32(-1)
        _check(load().mscd_graph_union(self.h, ids.ctypes.data_as(i32p), len(ids), C.byref(out)),
               "mscd_graph_union")
        return out.value

    def graph_parts(self, gid: int) -> np.ndarray:
        """Node offsets of the parts (int64[n_parts+1])."""
        P = C.c_int32()
        rc = load().mscd_graph_parts(self.h, gid, None, 0, C.byref(P))
        if rc not in (OK, ESMALL):
            _check(rc, "mscd_graph_parts")
        off = np.zeros(P.value + 1, np.int64)
        _check(load().mscd_graph_parts(self.h, gid, off.ctypes.data_as(i64p), len(off), C.byref(P)),
               "mscd_graph_parts")
        return off

    def graph_info(self, gid: int) -> dict:
        n, nnz, vol = C.c_int64(), C.c_int64(), C.c_int64()
        ue = C.c_int32()
        _check(load().mscd_graph_info(self.h, gid, C.byref(n), C.byref(nnz), C.byref(ue), C.byref(vol)),
               "mscd_graph_info")
        return dict(n=n.value, nnz=nnz.value, unit_exp=ue.value, volume=vol.value)

    def graph_degrees(self, gid: int) -> np.ndarray:
        n = self.graph_info(gid)["n"]
        k = np.zeros(max(n, 1), np.int64)
        _check(load().mscd_graph_degrees(self.h, gid, k.ctypes.data_as(i64p)), "mscd_graph_degrees")
        return k[:n]

    # ---- run
    def run(self, gid: int, alphas, seeds=None, stream=None) -> int:
        """Returns the status (OK, ETIMEOUT or EUNDECIDED); raises on other errors."""
        if isinstance(alphas, (list, tuple)):
            alphas = np.asarray(alphas, np.float64)
        ap, dev = _ptr(alphas)
        n_scales = int(alphas.shape[0])
        sp, sdev = _ptr(seeds)
        n_seeds = 0 if seeds is None else int(seeds.shape[0])
        if seeds is not None:
            if sdev != dev:
                raise ValueError("alphas and seeds must both be host or both be device arrays")
        st = None
        if stream is not None:
            st = stream if isinstance(stream, int) else stream.cuda_stream
        rc = load().mscd_run(self.h, gid, ap, n_scales, sp, n_seeds, DEVICE_PTRS if dev else 0, st)
        if rc not in (OK, ETIMEOUT, EUNDECIDED):
            raise MscdError(rc, load().mscd_last_error(self.h).decode() or "mscd_run")
        self.n_scales = n_scales
        self.n_seeds = n_seeds if seeds is not None else self.graph_info(gid)["n"]
        return rc

    def run_init(self, gid: int, alphas, seeds, init_ptr, init_nodes) -> int:
        """mscd_run from seeds plus initial members (host arrays)."""
        alphas = np.ascontiguousarray(alphas, np.float64)
        seeds = np.ascontiguousarray(seeds, np.int32)
        init_ptr = np.ascontiguousarray(init_ptr, np.int64)
        init_nodes = np.ascontiguousarray(init_nodes, np.int32)
        if len(init_nodes) == 0:
            init_nodes = np.zeros(1, np.int32)
        rc = load().mscd_run_init(self.h, gid, alphas.ctypes.data, len(alphas), seeds.ctypes.data, len(seeds),
                                  init_ptr.ctypes.data, init_nodes.ctypes.data, 0, None)
        if rc not in (OK, ETIMEOUT, EUNDECIDED):
            raise MscdError(rc, load().mscd_last_error(self.h).decode() or "mscd_run_init")
        self.n_scales = len(alphas)
        self.n_seeds = len(seeds)
        return rc

    def membership(self, scale: int, seed_idx: int):
        ln = C.c_int64()
        f = C.c_double()
        rc = load().mscd_get_membership(self.h, scale, seed_idx, None, 0, C.byref(ln), C.byref(f))
        if rc not in (OK, ESMALL):
            raise MscdError(rc, "mscd_get_membership")
        buf = np.zeros(max(ln.value, 1), np.int32)
        _check(load().mscd_get_membership(self.h, scale, seed_idx, buf.ctypes.data_as(i32p), ln.value, C.byref(ln),
                                          C.byref(f)), "mscd_get_membership")
        return buf[: ln.value], f.value

    def memberships(self, scale: int, with_stats: bool = True):
        """(ptr[n_seeds+1], nodes, fitness[n_seeds], stats[n_seeds, 8])."""
        N = self.n_seeds
        ptr = np.zeros(N + 1, np.int64)
        f = np.zeros(max(N, 1), np.float64)
        stt = np.zeros((max(N, 1), NSTATS), np.int64)
        tot = C.c_int64()
        rc = load().mscd_get_memberships(self.h, scale, ptr.ctypes.data_as(i64p), None, 0, None, None, C.byref(tot))
        if rc not in (OK, ESMALL):
            raise MscdError(rc, "mscd_get_memberships")
        nodes = np.zeros(max(tot.value, 1), np.int32)
        _check(load().mscd_get_memberships(self.h, scale, ptr.ctypes.data_as(i64p), nodes.ctypes.data_as(i32p),
                                           tot.value, f.ctypes.data_as(f64p),
                                           stt.ctypes.data_as(i64p) if with_stats else None, C.byref(tot)),
               "mscd_get_memberships")
        return ptr, nodes[: tot.value], f[:N], stt[:N]

    def unit_stats(self, scale: int):
        """(fitness[n_seeds], stats[n_seeds, 8]) of every unit of a scale,
        without copying the member lists (mscd_get_memberships with no node
        buffer)."""
        N = self.n_seeds
        f = np.zeros(max(N, 1), np.float64)
        stt = np.zeros((max(N, 1), NSTATS), np.int64)
        tot = C.c_int64()
        rc = load().mscd_get_memberships(self.h, scale, None, None, 0, f.ctypes.data_as(f64p),
                                         stt.ctypes.data_as(i64p), C.byref(tot))
        if rc not in (OK, ESMALL):
            raise MscdError(rc, "mscd_get_memberships")
        return f[:N], stt[:N]

    def communities(self, scale: int):
        """(comm_ptr, comm_nodes, fitness, seed2comm)."""
        nc, nn = C.c_int64(), C.c_int64()
        rc = load().mscd_get_communities(self.h, scale, None, 0, None, 0, None, None, C.byref(nc), C.byref(nn))
        if rc not in (OK, ESMALL):
            raise MscdError(rc, "mscd_get_communities")
        ptr = np.zeros(nc.value + 1, np.int64)
        nodes = np.zeros(max(nn.value, 1), np.int32)
        f = np.zeros(max(nc.value, 1), np.float64)
        s2c = np.zeros(max(self.n_seeds, 1), np.int32)
        _check(load().mscd_get_communities(self.h, scale, ptr.ctypes.data_as(i64p), nc.value + 1,
                                           nodes.ctypes.data_as(i32p), nn.value, f.ctypes.data_as(f64p),
                                           s2c.ctypes.data_as(i32p), C.byref(nc), C.byref(nn)),
               "mscd_get_communities")
        return ptr, nodes[: nn.value], f[: nc.value], s2c[: self.n_seeds]

    def run_sharded(self, gid: int, alphas, seeds, rank: int, world: int, all_gather):
        """One job whose seeds are split across `world` processes, one GPU each.
        This process grows its share (shard_seeds) with mscd_run; the shards of
        every scale are exchanged with all_gather(obj) -> [obj of rank 0, ...]
        (e.g. around torch.distributed.all_gather_object) and merged with
        mscd_merge_shards, giving what one run over all the seeds gives; the
        stability between successive merged scales is computed by
        mscd_nmi_covers and mscd_window_means (on a graph that is not a union,
        the values of mscd_get_stability).  Returns dict(status, communities =
        [(ptr, nodes, fitness, seed2comm)] per scale, nmi, win3, win5)."""
        alphas = np.ascontiguousarray(alphas, np.float64)
        seeds = np.ascontiguousarray(seeds, np.int32)
        idx = shard_seeds(len(seeds), rank, world)
        rc, local = OK, []
        if len(idx) == 0:  # more processes than seeds: an empty share
            none = dict(seed_index=idx, seed2comm=np.zeros(0, np.int32), ptr=np.zeros(1, np.int64),
                        nodes=np.zeros(0, np.int32), fitness=np.zeros(0, np.float64))
            local = [none] * len(alphas)
        else:
            rc = self.run(gid, alphas, np.ascontiguousarray(seeds[idx]))
            for s in range(len(alphas)):
                ptr, nodes, f, s2c = self.communities(s)
                local.append(dict(seed_index=idx, seed2comm=s2c, ptr=ptr, nodes=nodes, fitness=f))
        merged = merge_gathered(all_gather(local), len(seeds))
        n = self.graph_info(gid)["n"]
        nmi = np.array([self.nmi_covers(n, merged[s][:2], merged[s + 1][:2]) for s in range(len(alphas) - 1)],
                       np.float64)
        return dict(status=rc, communities=merged, nmi=nmi, win3=window_means(nmi, len(alphas), 3),
                    win5=window_means(nmi, len(alphas), 5))

    def stability(self, part=None):
        """(nmi_succ, window-3 means, window-5 means) of the last run, or of one
        part of a union graph."""
        S = self.n_scales
        a = np.zeros(max(S - 1, 1), np.float64)
        b = np.zeros(S, np.float64)
        c = np.zeros(S, np.float64)
        if part is None:
            _check(load().mscd_get_stability(self.h, a.ctypes.data_as(f64p), b.ctypes.data_as(f64p),
                                             c.ctypes.data_as(f64p)), "mscd_get_stability")
        else:
            _check(load().mscd_get_stability_part(self.h, part, a.ctypes.data_as(f64p), b.ctypes.data_as(f64p),
                                                  c.ctypes.data_as(f64p)), "mscd_get_stability_part")
        return a[: S - 1], b, c

    def grow_noalloc(self, gid: int, alphas, seeds, out: dict, stream=None):
        """Growth without device allocation (see mscd_grow_noalloc).  ``seeds`` is
        a CUDA int32 tensor or None; ``out`` holds CUDA tensors: nodes (int32),
        offset (int64), len (int32), fitness (float64), stats (int64, U x 8),
        status (int32), hash (int64).  Returns (status, n_nodes_needed)."""
        alphas = np.ascontiguousarray(alphas, np.float64)
        sp = None if seeds is None else seeds.data_ptr()
        n_seeds = 0 if seeds is None else int(seeds.shape[0])
        need = C.c_int64()
        st = None
        if stream is not None:
            st = stream if isinstance(stream, int) else stream.cuda_stream
        rc = load().mscd_grow_noalloc(self.h, gid, alphas.ctypes.data_as(f64p), len(alphas), sp, n_seeds,
                                      out["nodes"].data_ptr(), int(out["nodes"].numel()), out["offset"].data_ptr(),
                                      out["len"].data_ptr(), out["fitness"].data_ptr(), out["stats"].data_ptr(),
                                      out["status"].data_ptr(), out["hash"].data_ptr(), C.byref(need), st)
        return rc, need.value

    def run_stats(self) -> dict:
        s = mscd_run_stats()
        _check(load().mscd_get_run_stats(self.h, C.byref(s)), "mscd_get_run_stats")
        return s.as_dict()
