// C ABI of the library (declared in include/mscd.h).
//
// A context owns its resident graphs, the results of its last run and a
// reusable growth arena.  mscd_run grows every (scale, seed) unit with the
// growth kernel (first in the shared-memory slot class, then units that
// outgrew it in larger global-memory classes, until the class holds every
// node), deduplicates each scale and measures the stability between
// successive scales.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <map>
#include <vector>

#include "common.cuh"
#include "dedup.cuh"
#include "grow.cuh"
#include "ladder.cuh"

namespace {

struct GraphRec {
    bool live = false;
    i64 *rp = nullptr;
    i32 *col = nullptr;
    float *w = nullptr;
    i64 *wfx = nullptr, *k = nullptr;
    float *logk = nullptr;
    DevGraph g;
    // a disjoint union of parts (mscd_graph_union): node offsets, host and device
    std::vector<i64> parts;
    i64 *part_off = nullptr;  // null for a graph loaded from one CSR
    i64 max_part_n = 0;       // largest part (= n for one CSR): bounds a community's size
};

__global__ void check_seeds(const i32 *seeds, i64 N, i64 n, u32 *bad) {
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (i64)gridDim.x * blockDim.x)
        if (seeds[i] < 0 || (i64)seeds[i] >= n) atomicOr(bad, 1u);
}

// Initial member lists: offsets from 0, non-decreasing; node ids in range.
__global__ void check_init(const i64 *ptr, i64 N, const i32 *nodes, i64 n, u32 *bad) {
    const i64 stride = (i64)gridDim.x * blockDim.x;
    const i64 t0 = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (t0 == 0 && ptr[0] != 0) atomicOr(bad, 1u);
    for (i64 i = t0; i < N; i += stride)
        if (ptr[i + 1] < ptr[i]) atomicOr(bad, 1u);
    const i64 m = ptr[N];
    for (i64 j = t0; j < m; j += stride)
        if (nodes[j] < 0 || (i64)nodes[j] >= n) atomicOr(bad, 1u);
}

// Column sums of the per-unit statistics and status counts.
__global__ void sum_unit_stats(const i64 *ustat, const i32 *ulen, const i32 *ustatus, i64 U,
                               unsigned long long *tot) {
    unsigned long long s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    unsigned long long ntime = 0, nund = 0, len = 0;
    for (i64 u = (i64)blockIdx.x * blockDim.x + threadIdx.x; u < U; u += (i64)gridDim.x * blockDim.x) {
        const i64 *r = ustat + u * MSCD_NSTATS;
        s[0] += r[MSCD_STAT_EDGES];
        s[1] += r[MSCD_STAT_ADDS];
        s[2] += r[MSCD_STAT_REMOVES];
        s[3] += r[MSCD_STAT_SLOW];
        s[4] += r[MSCD_STAT_UNDECIDED];
        len += ulen[u];
        ntime += ustatus[u] == MSCD_ETIMEOUT;
        nund += ustatus[u] == MSCD_EUNDECIDED;
    }
    s[5] = ntime;
    s[6] = nund;
    s[7] = len;
    for (int j = 0; j < 8; ++j) {
        unsigned long long v = s[j];
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&tot[j], v);
    }
}

// After a scale's dedup: unit j's list is its community's list.
__global__ void point_units(const i32 *seed2comm, const i64 *comm_ptr, i64 N, i64 *uoff) {
    for (i64 j = (i64)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (i64)gridDim.x * blockDim.x)
        uoff[j] = comm_ptr[seed2comm[j]];
}

__global__ void gather_lists(const i64 *uoff, const i32 *ulen, const i64 *dst_ptr, const i32 *nodes, i64 N,
                             i32 *dst) {
    const int lane = threadIdx.x & 31;
    const i64 warps = (i64)gridDim.x * (blockDim.x >> 5);
    for (i64 u = (i64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < N; u += warps) {
        const i32 *src = nodes + uoff[u];
        i32 *d = dst + dst_ptr[u];
        for (int i = lane; i < ulen[u]; i += 32) d[i] = src[i];
    }
}

__global__ void widen_len(const i32 *ulen, i64 N, i64 *out) {
    for (i64 u = (i64)blockIdx.x * blockDim.x + threadIdx.x; u < N; u += (i64)gridDim.x * blockDim.x) out[u] = ulen[u];
}

std::atomic<long long> g_launches{0};

}  // namespace

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

struct Server;
void serve_destroy(Server *s);
struct FullState;
void full_state_free(FullState *f);
int full_run(const DevGraph &G, i64 max_part_n, const double *alphas, int32_t n_scales, int seed_rule,
             const i32 *prio_host, const i64 *init_ptr, const i32 *init_nodes, i64 n_init, double eta,
             i64 max_iters, GrowPipe &pipe, FullState *out, cudaStream_t st);
bool serve_graph_busy(Server *s, int32_t graph_id);

struct mscd_ctx {
    int device = 0;
    int sm_count = 1;
    mscd_params p{};
    cudaStream_t own = nullptr;
    std::vector<GraphRec> graphs;
    // last run
    bool have = false;
    int32_t S = 0;
    i64 N = 0, U = 0, n_nodes_graph = 0;
    double *alphas = nullptr;
    i32 *seeds = nullptr;
    i64 *init_ptr = nullptr;  // initial members per seed (mscd_run_init)
    i32 *init_nodes = nullptr;
    i64 *uoff = nullptr;
    i32 *ulen = nullptr;
    u64 *uhash = nullptr;
    double *uf = nullptr;
    i64 *ustat = nullptr;
    i32 *ustatus = nullptr;
    std::vector<ScaleResult> scales;
    int32_t n_parts = 1;
    std::vector<double> nmi_succ, win3, win5;  // per part: S-1, S and S values
    mscd_run_stats stats{};
    // autotuner results by graph shape class: parameters and growth ms of the sample
    std::map<u64, std::pair<mscd_params, double>> tune_cache;
    // the growth pipeline of runs: its arena, retry lists and output buffer are reused
    GrowPipe pipe;
    Server *server = nullptr;  // query serving (mscd_serve_start)
    FullState *full = nullptr;  // last run of the full method (mscd_full_run)
    char last_error[160] = "";  // where the last failed run stopped
};

namespace {

void free_run(mscd_ctx *c) {
    cudaFree(c->alphas);
    cudaFree(c->seeds);
    cudaFree(c->init_ptr);
    cudaFree(c->init_nodes);
    c->init_ptr = nullptr;
    c->init_nodes = nullptr;
    cudaFree(c->uoff);
    cudaFree(c->ulen);
    cudaFree(c->uhash);
    cudaFree(c->uf);
    cudaFree(c->ustat);
    cudaFree(c->ustatus);
    c->alphas = nullptr;
    c->seeds = nullptr;
    c->uoff = nullptr;
    c->ulen = nullptr;
    c->uhash = nullptr;
    c->uf = nullptr;
    c->ustat = nullptr;
    c->ustatus = nullptr;
    for (auto &s : c->scales) scale_result_free(&s);
    c->scales.clear();
    c->nmi_succ.clear();
    c->win3.clear();
    c->win5.clear();
    c->have = false;
}

void free_graph(GraphRec &g) {
    cudaFree(g.rp);
    cudaFree(g.col);
    cudaFree(g.w);
    cudaFree(g.wfx);
    cudaFree(g.k);
    cudaFree(g.logk);
    cudaFree(g.part_off);
    g = GraphRec{};
}

int add_graph(mscd_ctx *c, const GraphRec &g, int32_t *graph_id);

GraphRec *find_graph(mscd_ctx *c, int32_t id) {
    if (!c || id < 0 || id >= (int32_t)c->graphs.size() || !c->graphs[id].live) return nullptr;
    return &c->graphs[id];
}

void window_means(const std::vector<double> &nmi, int32_t S, int p, std::vector<double> &out) {
    out.assign(S, NAN);
    for (int32_t i = 0; i < S; ++i) {
        int32_t lo = i - (p - 1) / 2, hi = lo + p - 1;
        lo = std::max(lo, 0);
        hi = std::min(hi, S - 1);
        double s = 0.0;
        int cnt = 0;
        for (int32_t j = lo; j + 1 <= hi; ++j) {
            s += nmi[j];
            ++cnt;
        }
        out[i] = cnt ? s / cnt : NAN;
    }
}


}  // namespace

bool ctx_graph(mscd_ctx *c, int32_t graph_id, DevGraph *g, int *device) {
    GraphRec *r = find_graph(c, graph_id);
    if (!r) return false;
    *g = r->g;
    *device = c->device;
    return true;
}

Server **ctx_server(mscd_ctx *c) { return &c->server; }
FullState **ctx_full(mscd_ctx *c) { return &c->full; }

GrowPipe *ctx_pipe(mscd_ctx *c, cudaStream_t st) {
    c->pipe.p = c->p;
    c->pipe.p.schedule = MSCD_SCHED_PERSISTENT;
    c->pipe.st = st ? st : c->own;
    c->pipe.stats = nullptr;
    return &c->pipe;
}

bool ctx_graph_part(mscd_ctx *c, int32_t id, DevGraph *g, i64 *max_part_n) {
    GraphRec *r = find_graph(c, id);
    if (!r) return false;
    *g = r->g;
    *max_part_n = r->max_part_n;
    return true;
}

int ctx_device_of(mscd_ctx *c) { return c->device; }
int ctx_sm_count_of(mscd_ctx *c) { return c->sm_count; }
mscd_params ctx_params_of(mscd_ctx *c) { return c->p; }

extern "C" {

const char *mscd_strerror(int s) {
    switch (s) {
    case MSCD_OK: return "ok";
    case MSCD_EINVAL: return "invalid argument or malformed CSR structure";
    case MSCD_ENOTSYM: return "CSR is not symmetric (missing reverse entry or unequal weight)";
    case MSCD_ESELFLOOP: return "CSR has a self-loop";
    case MSCD_EDUP: return "CSR row has a repeated entry";
    case MSCD_ERANGE: return "exact fixed-point weights exceed 62 bits";
    case MSCD_ENOMEM: return "device memory allocation failed";
    case MSCD_EDEVICE: return "CUDA device error";
    case MSCD_ETIMEOUT: return "a unit hit the grow/prune repetition cap";
    case MSCD_ESMALL: return "output buffer too small";
    case MSCD_EUNDECIDED: return "a comparison could not be decided by any certified stage";
    case MSCD_EUNSORTED: return "CSR row not in ascending column order";
    case MSCD_EWEIGHT: return "edge weight not finite and positive";
    case MSCD_ENORESULT: return "no successful run to read results from";
    case MSCD_EBUSY: return "in use (a graph that queries still need, or a running server)";
    default: return "unknown status";
    }
}

int mscd_version(void) { return 200; }

int64_t mscd_launch_count(void) { return (int64_t)g_launches.load(std::memory_order_relaxed); }

int mscd_create(mscd_ctx **out, int device, const mscd_params *params) {
    if (!out) return MSCD_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return MSCD_EDEVICE;
    if (device < 0 || device >= ndev) return MSCD_EINVAL;
    if (params && params->struct_size != (int32_t)sizeof(mscd_params)) return MSCD_EINVAL;
    MSCD_CUDA(cudaSetDevice(device));
    mscd_ctx *c = new (std::nothrow) mscd_ctx();
    if (!c) return MSCD_ENOMEM;
    c->device = device;
    if (params) c->p = *params;
    if (c->p.warps_per_block <= 0) c->p.warps_per_block = 8;
    if (c->p.max_rounds <= 0) c->p.max_rounds = 1000000;
    if (c->p.smem_slots < 0) c->p.smem_slots = 0;
    if (c->p.mid_slots < 0) c->p.mid_slots = 0;
    if (c->p.global_warps_per_sm <= 0) c->p.global_warps_per_sm = 16;
    if (c->p.list_hash_bits < 0 || c->p.list_hash_bits > 63 || c->p.global_slots < 0 ||
        (c->p.global_slots & (c->p.global_slots - 1)) ||
        (c->p.schedule != MSCD_SCHED_PERSISTENT && c->p.schedule != MSCD_SCHED_PER_SCALE)) {
        delete c;
        return MSCD_EINVAL;
    }
    if (c->p.warps_per_block > GROW_MAX_THREADS / 32 || (c->p.smem_slots & (c->p.smem_slots - 1)) ||
        (c->p.smem_slots > 0 && c->p.smem_slots < 32) || (c->p.mid_slots & (c->p.mid_slots - 1)) ||
        (c->p.mid_slots > 0 && c->p.mid_slots < 32)) {
        delete c;
        return MSCD_EINVAL;
    }
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    c->pipe.sm_count = c->sm_count;
    if (cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking) != cudaSuccess) {
        delete c;
        return MSCD_EDEVICE;
    }
    *out = c;
    return MSCD_OK;
}

int mscd_destroy(mscd_ctx *c) {
    if (!c) return MSCD_EINVAL;
    serve_destroy(c->server);
    c->server = nullptr;
    full_state_free(c->full);
    c->full = nullptr;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->own);
    free_run(c);
    for (auto &g : c->graphs) free_graph(g);
    pipe_free(c->pipe);
    cudaStreamDestroy(c->own);
    delete c;
    return MSCD_OK;
}

int mscd_graph_load_csr(mscd_ctx *c, int64_t n, const int64_t *row_ptr, const int32_t *col, const float *w,
                        uint32_t flags, int32_t *graph_id) {
    if (!c || !row_ptr || !graph_id || n < 0 || n >= (int64_t)INT32_MAX) return MSCD_EINVAL;
    MSCD_CUDA(cudaSetDevice(c->device));
    const bool dev = flags & MSCD_DEVICE_PTRS;
    const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaStream_t st = c->own;
    i64 nnz = 0;
    if (dev) MSCD_CUDA(cudaMemcpy(&nnz, row_ptr + n, sizeof(i64), cudaMemcpyDeviceToHost));
    else nnz = row_ptr[n];
    if (nnz < 0 || (nnz > 0 && !col)) return MSCD_EINVAL;
    GraphRec g;
    int rc = MSCD_OK;
    do {
        if ((rc = cuda_status(cudaMalloc((void **)&g.rp, (size_t)(n + 1) * sizeof(i64))))) break;
        if ((rc = cuda_status(cudaMalloc((void **)&g.col, (size_t)std::max<i64>(nnz, 1) * sizeof(i32))))) break;
        if ((rc = cuda_status(cudaMemcpyAsync(g.rp, row_ptr, (size_t)(n + 1) * sizeof(i64), kind, st)))) break;
        if (nnz > 0 && (rc = cuda_status(cudaMemcpyAsync(g.col, col, (size_t)nnz * sizeof(i32), kind, st)))) break;
        if (w) {
            if ((rc = cuda_status(cudaMalloc((void **)&g.w, (size_t)std::max<i64>(nnz, 1) * sizeof(float))))) break;
            if (nnz > 0 && (rc = cuda_status(cudaMemcpyAsync(g.w, w, (size_t)nnz * sizeof(float), kind, st)))) break;
        }
        rc = graph_prepare(n, g.rp, g.col, g.w, &g.g, &g.wfx, &g.k, &g.logk, st);
    } while (0);
    if (rc != MSCD_OK) {
        cudaStreamSynchronize(st);
        free_graph(g);
        return rc;
    }
    cudaFree(g.w);  // the exact fixed-point copy replaces it
    g.w = nullptr;
    g.live = true;
    g.parts = {0, n};
    g.max_part_n = n;
    return add_graph(c, g, graph_id);
}

int mscd_graph_union(mscd_ctx *c, const int32_t *graph_ids, int32_t n_parts, int32_t *union_id) {
    if (!c || !graph_ids || n_parts < 1 || !union_id) return MSCD_EINVAL;
    std::vector<DevGraph> parts;
    i64 max_part = 0;
    for (int32_t i = 0; i < n_parts; ++i) {
        GraphRec *r = find_graph(c, graph_ids[i]);
        if (!r || r->part_off) return MSCD_EINVAL;  // parts are graphs loaded from one CSR
        parts.push_back(r->g);
        max_part = std::max(max_part, r->g.n);
    }
    MSCD_CUDA(cudaSetDevice(c->device));
    GraphRec g;
    int rc = graph_union(parts, &g.g, &g.rp, &g.col, &g.wfx, &g.k, &g.logk, &g.parts, c->own);
    if (rc) return rc;
    rc = cuda_status(cudaMalloc((void **)&g.part_off, g.parts.size() * sizeof(i64)));
    if (!rc)
        rc = cuda_status(cudaMemcpy(g.part_off, g.parts.data(), g.parts.size() * sizeof(i64), cudaMemcpyHostToDevice));
    if (rc) {
        free_graph(g);
        return rc;
    }
    g.max_part_n = max_part;
    g.live = true;
    return add_graph(c, g, union_id);
}

int mscd_graph_parts(mscd_ctx *c, int32_t graph_id, int64_t *node_offset, int32_t cap, int32_t *n_parts) {
    GraphRec *g = find_graph(c, graph_id);
    if (!g || !n_parts || cap < 0 || (cap > 0 && !node_offset)) return MSCD_EINVAL;
    const int32_t P = (int32_t)g->parts.size() - 1;
    *n_parts = P;
    if (cap < P + 1) return MSCD_ESMALL;
    std::copy(g->parts.begin(), g->parts.end(), node_offset);
    return MSCD_OK;
}

}  // extern "C"

namespace {

int add_graph(mscd_ctx *c, const GraphRec &g, int32_t *graph_id) {
    int32_t id = -1;
    for (size_t i = 0; i < c->graphs.size(); ++i)
        if (!c->graphs[i].live) {
            id = (int32_t)i;
            break;
        }
    if (id < 0) {
        id = (int32_t)c->graphs.size();
        c->graphs.push_back(g);
    } else {
        c->graphs[id] = g;
    }
    *graph_id = id;
    return MSCD_OK;
}

}  // namespace

extern "C" {

int mscd_graph_free(mscd_ctx *c, int32_t graph_id) {
    GraphRec *g = find_graph(c, graph_id);
    if (!g) return MSCD_EINVAL;
    if (serve_graph_busy(c->server, graph_id)) return MSCD_EBUSY;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->own);
    free_graph(*g);
    return MSCD_OK;
}

int mscd_graph_info(mscd_ctx *c, int32_t graph_id, int64_t *n, int64_t *nnz, int32_t *unit_exp, int64_t *volume) {
    GraphRec *g = find_graph(c, graph_id);
    if (!g) return MSCD_EINVAL;
    if (n) *n = g->g.n;
    if (nnz) *nnz = g->g.nnz;
    if (unit_exp) *unit_exp = g->g.unit_exp;
    if (volume) *volume = g->g.volume;
    return MSCD_OK;
}

int mscd_graph_degrees(mscd_ctx *c, int32_t graph_id, int64_t *k) {
    GraphRec *g = find_graph(c, graph_id);
    if (!g || !k) return MSCD_EINVAL;
    MSCD_CUDA(cudaSetDevice(c->device));
    if (g->g.n > 0) MSCD_CUDA(cudaMemcpy(k, g->g.k, (size_t)g->g.n * sizeof(i64), cudaMemcpyDeviceToHost));
    return MSCD_OK;
}

int mscd_scales_logspaced(double vmin, double a, int32_t x, double *out) {
    if (x < 1 || !out || !(vmin > 0.0) || !(a >= vmin) || !std::isfinite(a)) return MSCD_EINVAL;
    if (x == 1) {
        out[0] = a;
        return MSCD_OK;
    }
    const double lx = std::log((double)x);
    for (int32_t k = 1; k <= x; ++k) out[k - 1] = vmin + (a - vmin) * (1.0 - std::log((double)k) / lx);
    return MSCD_OK;
}

}  // extern "C"

namespace {

// The whole path of mscd_run; growth_only stops after the growth (autotuning).
int run_impl(mscd_ctx *c, int32_t graph_id, const double *alphas, int32_t n_scales, const int32_t *seeds,
             int64_t n_seeds, uint32_t flags, void *cuda_stream, bool growth_only, const int64_t *init_ptr = nullptr,
             const int32_t *init_nodes = nullptr) {
    GraphRec *gr = find_graph(c, graph_id);
    if (!gr || !alphas || n_scales < 1) return MSCD_EINVAL;
    MSCD_CUDA(cudaSetDevice(c->device));
    cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : c->own;
    const bool dev = flags & MSCD_DEVICE_PTRS;
    const DevGraph &G = gr->g;
    const i64 N = seeds ? n_seeds : G.n;
    if (N < 0) return MSCD_EINVAL;
    std::vector<double> ha(n_scales);
    if (dev) MSCD_CUDA(cudaMemcpy(ha.data(), alphas, n_scales * sizeof(double), cudaMemcpyDeviceToHost));
    else std::memcpy(ha.data(), alphas, n_scales * sizeof(double));
    for (double a : ha)
        if (!(a > 0.0) || !std::isfinite(a)) return MSCD_EINVAL;
    free_run(c);
    c->stats = mscd_run_stats{};
    c->S = n_scales;
    c->N = N;
    c->U = (i64)n_scales * N;
    c->n_nodes_graph = G.n;
    const i64 U = c->U;
    cudaEvent_t ev[4];
    for (auto &e : ev) cudaEventCreate(&e);
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> dedup_ev;  // around each group's dedup
    char stage[96];
    snprintf(stage, sizeof(stage), "setup");
    unsigned char *big_seed = nullptr;
    int rc = MSCD_OK;
    cudaEventRecord(ev[0], st);
    do {
        if ((rc = cuda_status(cudaMalloc((void **)&c->alphas, n_scales * sizeof(double))))) break;
        if ((rc = cuda_status(cudaMemcpyAsync(c->alphas, ha.data(), n_scales * sizeof(double), cudaMemcpyHostToDevice,
                                              st))))
            break;
        if (seeds && N > 0) {
            if ((rc = cuda_status(cudaMalloc((void **)&c->seeds, N * sizeof(i32))))) break;
            if ((rc = cuda_status(cudaMemcpyAsync(c->seeds, seeds, N * sizeof(i32),
                                                  dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st))))
                break;
        }
        const size_t U1 = (size_t)std::max<i64>(U, 1);
        if ((rc = cuda_status(cudaMalloc((void **)&c->uoff, U1 * sizeof(i64))))) break;
        if ((rc = cuda_status(cudaMalloc((void **)&c->ulen, U1 * sizeof(i32))))) break;
        if ((rc = cuda_status(cudaMalloc((void **)&c->uhash, U1 * sizeof(u64))))) break;
        if ((rc = cuda_status(cudaMalloc((void **)&c->uf, U1 * sizeof(double))))) break;
        if ((rc = cuda_status(cudaMalloc((void **)&c->ustat, U1 * MSCD_NSTATS * sizeof(i64))))) break;
        if ((rc = cuda_status(cudaMalloc((void **)&c->ustatus, U1 * sizeof(i32))))) break;
        c->pipe.st = st;
        if ((rc = pipe_reserve(c->pipe, (i64)U1))) break;
        Counters *ctr = c->pipe.ctr;
        if ((rc = cuda_status(cudaMalloc((void **)&big_seed, (size_t)std::max<i64>(N, 1))))) break;
        if ((rc = cuda_status(cudaMemsetAsync(big_seed, 0, (size_t)std::max<i64>(N, 1), st)))) break;
        if (init_ptr && N > 0) {
            // initial member lists (copied; checked on the device below)
            i64 m = 0;
            if (dev) MSCD_CUDA(cudaMemcpy(&m, init_ptr + N, sizeof(i64), cudaMemcpyDeviceToHost));
            else m = init_ptr[N];
            if (m < 0 || (m > 0 && !init_nodes)) { rc = MSCD_EINVAL; break; }
            const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
            if ((rc = cuda_status(cudaMalloc((void **)&c->init_ptr, (N + 1) * sizeof(i64))))) break;
            if ((rc = cuda_status(cudaMalloc((void **)&c->init_nodes, (size_t)std::max<i64>(m, 1) * sizeof(i32)))))
                break;
            if ((rc = cuda_status(cudaMemcpyAsync(c->init_ptr, init_ptr, (N + 1) * sizeof(i64), kind, st)))) break;
            if (m > 0 && (rc = cuda_status(cudaMemcpyAsync(c->init_nodes, init_nodes, m * sizeof(i32), kind, st))))
                break;
        }
        if (c->seeds) {
            if ((rc = cuda_status(cudaMemsetAsync(ctr, 0, sizeof(Counters), st)))) break;
            check_seeds<<<152 * 8, 256, 0, st>>>(c->seeds, N, G.n, &ctr->error_flags); note_launch();
            if (c->init_ptr) {
                check_init<<<152 * 8, 256, 0, st>>>(c->init_ptr, N, c->init_nodes, G.n, &ctr->error_flags);
                note_launch();
            }
            u32 bad = 0;
            if ((rc = cuda_status(cudaMemcpyAsync(&bad, &ctr->error_flags, sizeof(u32), cudaMemcpyDeviceToHost, st))))
                break;
            if ((rc = cuda_status(cudaStreamSynchronize(st)))) break;
            if (bad) { rc = MSCD_EINVAL; break; }
        }
        // ---- growth ----
        std::vector<int> ladder;
        std::vector<bool> in_smem;
        if ((rc = make_ladder(G, gr->max_part_n, c->p, &ladder, &in_smem))) break;
        // Scale groups.  The member lists of a group's units go to one output
        // buffer; once the group is grown, each of its scales is deduplicated
        // and its units are pointed at their community's list (the lists are
        // equal), so the buffer is free again for the next group.  A group is
        // as many scales as fit 35% of the free memory at the expected list
        // length (1024 entries per unit, or twice the largest group mean seen:
        // lists grow towards the coarse scales); the persistent schedule
        // usually needs one group, the plain form takes one scale at a time.
        const bool per_scale = c->p.schedule == MSCD_SCHED_PER_SCALE;
        size_t free_mem = 0, total_mem = 0;
        cudaMemGetInfo(&free_mem, &total_mem);
        i64 out_budget = (i64)(free_mem / 10 * 4 / sizeof(i32));
        double per_unit = std::max(1.0, std::min<double>(1024.0, (double)gr->max_part_n));
        GrowArgs proto{};
        proto.G = G;
        proto.alphas = c->alphas;
        proto.seeds = c->seeds;
        proto.n_seeds = N;
        proto.max_rounds = c->p.max_rounds;
        proto.uoff = c->uoff;
        proto.ulen = c->ulen;
        proto.uhash = c->uhash;
        proto.uf = c->uf;
        proto.ustat = c->ustat;
        proto.ustatus = c->ustatus;
        proto.big_seed = c->init_ptr ? nullptr : big_seed;  // sizes from {seed} do not predict these
        proto.init_ptr = c->init_ptr;
        proto.init_nodes = c->init_nodes;
        proto.log_kmax = G.kmax > 1 ? (float)std::log((double)G.kmax) : 0.0f;
        proto.hash_clear = c->p.list_hash_bits > 0 ? ~(((u64)1 << c->p.list_hash_bits) - 1) : 0;
        c->pipe.p = c->p;
        c->pipe.st = st;
        c->pipe.stats = &c->stats;
        int32_t s0 = 0;
        while (s0 < n_scales && rc == MSCD_OK) {
        {
            // 35% of what is free, counting the output buffer being reused
            size_t fr = 0, tot = 0;
            cudaMemGetInfo(&fr, &tot);
            out_budget = (i64)((double)(fr + (size_t)c->pipe.out_cap * sizeof(i32)) * 0.35 / sizeof(i32));
        }
        int32_t s1 = s0 + 1;
        if (!per_scale && N > 0)
            s1 = (int32_t)std::min<i64>(n_scales, s0 + std::max<i64>(1, (i64)(out_budget / (per_unit * N))));
        else if (!per_scale)
            s1 = n_scales;
        const i64 group_units = (i64)(s1 - s0) * N;
        unsigned long long cursor = 0;
        proto.unit_base = (i64)s0 * N;
        snprintf(stage, sizeof(stage), "growth of scales %d..%d", s0, s1 - 1);
        rc = grow_units(c->pipe, proto, group_units, ladder, in_smem, per_scale, out_budget, gr->max_part_n, &cursor);
        if (rc) break;
        if (group_units > 0)
            per_unit = std::max(per_unit, 2.0 * (double)cursor / (double)group_units);
        if (!growth_only) {
            // dedup the group's scales; point their units at the community lists
            cudaEvent_t d0, d1;
            cudaEventCreate(&d0);
            cudaEventCreate(&d1);
            dedup_ev.push_back({d0, d1});
            cudaEventRecord(d0, st);
            c->scales.resize(n_scales);
            for (int32_t s = s0; s < s1 && rc == MSCD_OK; ++s) {
                snprintf(stage, sizeof(stage), "dedup of scale %d", s);
                rc = dedup_scale(c->uoff + s * N, c->ulen + s * N, c->uhash + s * N, c->uf + s * N,
                                 c->pipe.out_nodes, N, &c->scales[s], st);
                if (rc == MSCD_OK && N > 0) {
                    point_units<<<152 * 4, 256, 0, st>>>(c->scales[s].seed2comm, c->scales[s].comm_ptr, N,
                                                          c->uoff + s * N); note_launch();
                }
            }
            cudaEventRecord(d1, st);
        }
        s0 = s1;
        }  // scale groups
        if (rc) break;
        // a large output buffer is not kept past the growth (the lists now live
        // in the deduplicated communities)
        if (!growth_only && c->pipe.out_cap > ((i64)1 << 28)) pipe_release_output(c->pipe);
        cudaEventRecord(ev[1], st);
        // ---- totals ----
        unsigned long long *tot = nullptr;
        if ((rc = cuda_status(cudaMallocAsync((void **)&tot, 8 * sizeof(unsigned long long), st)))) break;
        cudaMemsetAsync(tot, 0, 8 * sizeof(unsigned long long), st);
        if (U > 0) { sum_unit_stats<<<152 * 4, 256, 0, st>>>(c->ustat, c->ulen, c->ustatus, U, tot); note_launch(); }
        unsigned long long ht[8];
        cudaMemcpyAsync(ht, tot, sizeof(ht), cudaMemcpyDeviceToHost, st);
        cudaFreeAsync(tot, st);
        if ((rc = cuda_status(cudaStreamSynchronize(st)))) break;
        c->stats.units = U;
        c->stats.edges_scanned = (i64)ht[0];
        c->stats.adds = (i64)ht[1];
        c->stats.removes = (i64)ht[2];
        c->stats.slow_decisions = (i64)ht[3];
        c->stats.undecided = (i64)ht[4];
        c->stats.member_entries = (i64)ht[7];
        const i64 n_timeout = (i64)ht[5], n_undecided = (i64)ht[6];
        if (growth_only) {
            cudaEventRecord(ev[2], st);
            cudaEventRecord(ev[3], st);
            if ((rc = cuda_status(cudaEventSynchronize(ev[3])))) break;
            float ms = 0;
            cudaEventElapsedTime(&ms, ev[0], ev[1]);
            c->stats.ms_grow = c->stats.ms_total = ms;
            if (n_undecided) rc = MSCD_EUNDECIDED;
            else if (n_timeout) rc = MSCD_ETIMEOUT;
            break;
        }
        cudaEventRecord(ev[2], st);
        // ---- stability ----
        // per part: successive-scale NMI and window means
        const int32_t P = (int32_t)gr->parts.size() - 1;
        const int32_t S1 = std::max(n_scales - 1, 0);
        c->n_parts = P;
        c->nmi_succ.assign((size_t)P * S1, NAN);
        {
            std::vector<double> pn(P);
            for (int32_t s = 0; s + 1 < n_scales && rc == MSCD_OK; ++s) {
                snprintf(stage, sizeof(stage), "stability between scales %d and %d", s, s + 1);
                rc = nmi_between(c->scales[s], c->scales[s + 1], G.n, gr->part_off, P, pn.data(), st);
                for (int32_t p = 0; p < P; ++p) c->nmi_succ[(size_t)p * S1 + s] = pn[p];
            }
        }
        if (rc) break;
        c->win3.assign((size_t)P * n_scales, NAN);
        c->win5.assign((size_t)P * n_scales, NAN);
        for (int32_t p = 0; p < P; ++p) {
            std::vector<double> one(c->nmi_succ.begin() + (size_t)p * S1, c->nmi_succ.begin() + (size_t)(p + 1) * S1);
            std::vector<double> w;
            window_means(one, n_scales, 3, w);
            std::copy(w.begin(), w.end(), c->win3.begin() + (size_t)p * n_scales);
            window_means(one, n_scales, 5, w);
            std::copy(w.begin(), w.end(), c->win5.begin() + (size_t)p * n_scales);
        }
        cudaEventRecord(ev[3], st);
        if ((rc = cuda_status(cudaEventSynchronize(ev[3])))) break;
        float ms = 0, md = 0;
        for (auto &d : dedup_ev) {
            cudaEventElapsedTime(&ms, d.first, d.second);
            md += ms;
        }
        cudaEventElapsedTime(&ms, ev[0], ev[1]);
        c->stats.ms_grow = ms - md;  // growth with its totals, the dedup of the groups taken out
        c->stats.ms_dedup = md;
        cudaEventElapsedTime(&ms, ev[2], ev[3]);
        c->stats.ms_stability = ms;
        cudaEventElapsedTime(&ms, ev[0], ev[3]);
        c->stats.ms_total = ms;
        c->have = true;
        if (n_undecided) rc = MSCD_EUNDECIDED;
        else if (n_timeout) rc = MSCD_ETIMEOUT;
    } while (0);
    cudaStreamSynchronize(st);
    cudaFree(big_seed);
    for (auto &e : ev) cudaEventDestroy(e);
    for (auto &d : dedup_ev) {
        cudaEventDestroy(d.first);
        cudaEventDestroy(d.second);
    }
    if (rc != MSCD_OK && !c->have) free_run(c);
    if (rc != MSCD_OK)
        snprintf(c->last_error, sizeof(c->last_error), "mscd_run: %s: %s", stage, mscd_strerror(rc));
    return rc;
}

// Graph shape class of the autotuner's cache: size (log2 n), weighted, slot width.
u64 tune_key(const DevGraph &g) {
    int lg = 0;
    while (lg < 62 && ((i64)1 << lg) < g.n) ++lg;
    return (u64)lg | (g.wfx ? 1ull << 8 : 0ull) | (g.kmax < 65536 ? 1ull << 9 : 0ull);
}

}  // namespace

extern "C" {

int mscd_run(mscd_ctx *c, int32_t graph_id, const double *alphas, int32_t n_scales, const int32_t *seeds,
             int64_t n_seeds, uint32_t flags, void *cuda_stream) {
    return run_impl(c, graph_id, alphas, n_scales, seeds, n_seeds, flags, cuda_stream, false);
}

int mscd_run_init(mscd_ctx *c, int32_t graph_id, const double *alphas, int32_t n_scales, const int32_t *seeds,
                  int64_t n_seeds, const int64_t *init_ptr, const int32_t *init_nodes, uint32_t flags,
                  void *cuda_stream) {
    if (!seeds || !init_ptr) return MSCD_EINVAL;
    return run_impl(c, graph_id, alphas, n_scales, seeds, n_seeds, flags, cuda_stream, false, init_ptr, init_nodes);
}

int mscd_autotune(mscd_ctx *c, int32_t graph_id, const double *alphas, int32_t n_scales, int64_t n_sample,
                  uint32_t flags, mscd_params *best, double *best_ms) {
    GraphRec *gr = find_graph(c, graph_id);
    if (!gr || !alphas || n_scales < 1 || n_sample < 0) return MSCD_EINVAL;
    const u64 key = tune_key(gr->g);
    if ((flags & MSCD_TUNE_CACHED) && c->tune_cache.count(key)) {
        const mscd_params &p = c->tune_cache[key].first;
        if (best) *best = p;
        if (best_ms) *best_ms = c->tune_cache[key].second;
        if (flags & MSCD_TUNE_APPLY) c->p = p;
        return MSCD_OK;
    }
    // evenly spaced seeds over the graph (every part of a union alike)
    const i64 n = gr->g.n;
    const i64 m = std::min<i64>(n, n_sample > 0 ? n_sample : 20000);
    if (m < 1) return MSCD_EINVAL;
    std::vector<i32> seeds(m);
    for (i64 i = 0; i < m; ++i) seeds[i] = (i32)((__int128)i * n / m);
    const mscd_params saved = c->p;
    mscd_params cur = c->p;
    int rc = MSCD_OK;
    auto time_it = [&](const mscd_params &p, double *ms) -> int {
        c->p = p;
        int r = run_impl(c, graph_id, alphas, n_scales, seeds.data(), m, 0, nullptr, true);
        *ms = c->stats.ms_grow;
        return r;
    };
    double cur_ms = 0.0, ms = 0.0;
    if ((rc = time_it(cur, &cur_ms))) {  // also the warm-up
        c->p = saved;
        free_run(c);
        return rc;
    }
    if ((rc = time_it(cur, &cur_ms)) == MSCD_OK) {
        // coordinate search: first shared-memory class, first global class, global residency
        const int smem_c[] = {256, 512, 1024, 2048};
        const int glob_c[] = {0, 4096, 8192, 16384};
        const int warps_c[] = {8, 12, 16, 24, 32};
        for (int axis = 0; axis < 3 && rc == MSCD_OK; ++axis) {
            const int count = axis == 0 ? 4 : axis == 1 ? 4 : 5;
            for (int i = 0; i < count && rc == MSCD_OK; ++i) {
                mscd_params p = cur;
                if (axis == 0) p.smem_slots = smem_c[i];
                if (axis == 1) p.global_slots = glob_c[i];
                if (axis == 2) p.global_warps_per_sm = warps_c[i];
                if (axis == 1 && p.global_slots && p.global_slots <= std::max(p.smem_slots, 1024)) continue;
                if (std::memcmp(&p, &cur, sizeof(p)) == 0) continue;
                if ((rc = time_it(p, &ms))) break;
                if (ms < cur_ms) {
                    cur = p;
                    cur_ms = ms;
                }
            }
        }
    }
    free_run(c);
    c->p = saved;
    if (rc) return rc;
    c->tune_cache[key] = {cur, cur_ms};
    if (flags & MSCD_TUNE_APPLY) c->p = cur;
    if (best) *best = cur;
    if (best_ms) *best_ms = cur_ms;
    return MSCD_OK;
}

int mscd_get_membership(mscd_ctx *c, int32_t scale_idx, int64_t seed_idx, int32_t *buf, int64_t cap, int64_t *len,
                        double *fitness) {
    if (!c || !len) return MSCD_EINVAL;
    if (!c->have) return MSCD_ENORESULT;
    if (scale_idx < 0 || scale_idx >= c->S || seed_idx < 0 || seed_idx >= c->N) return MSCD_EINVAL;
    MSCD_CUDA(cudaSetDevice(c->device));
    const i64 u = (i64)scale_idx * c->N + seed_idx;
    i64 off = 0;
    i32 m = 0;
    MSCD_CUDA(cudaMemcpy(&off, c->uoff + u, sizeof(i64), cudaMemcpyDeviceToHost));
    MSCD_CUDA(cudaMemcpy(&m, c->ulen + u, sizeof(i32), cudaMemcpyDeviceToHost));
    if (fitness) MSCD_CUDA(cudaMemcpy(fitness, c->uf + u, sizeof(double), cudaMemcpyDeviceToHost));
    *len = m;
    if (cap < m || (m > 0 && !buf)) return MSCD_ESMALL;
    if (m > 0)
        MSCD_CUDA(cudaMemcpy(buf, c->scales[scale_idx].comm_nodes + off, (size_t)m * sizeof(i32),
                             cudaMemcpyDeviceToHost));
    return MSCD_OK;
}

int mscd_get_memberships(mscd_ctx *c, int32_t scale_idx, int64_t *ptr, int32_t *nodes, int64_t nodes_cap,
                         double *fitness, int64_t *stats, int64_t *n_nodes) {
    if (!c || !n_nodes) return MSCD_EINVAL;
    if (!c->have) return MSCD_ENORESULT;
    if (scale_idx < 0 || scale_idx >= c->S) return MSCD_EINVAL;
    MSCD_CUDA(cudaSetDevice(c->device));
    cudaStream_t st = c->own;
    const i64 N = c->N, base = (i64)scale_idx * N;
    i64 *dptr = nullptr;
    i32 *dnodes = nullptr;
    int rc = MSCD_OK;
    do {
        if ((rc = cuda_status(cudaMallocAsync((void **)&dptr, (N + 1) * sizeof(i64), st)))) break;
        if (N > 0) { widen_len<<<152 * 4, 256, 0, st>>>(c->ulen + base, N, dptr); note_launch(); }
        if ((rc = scan_exclusive_i64(dptr, dptr, N, dptr + N, st))) break;
        i64 total = 0;
        if ((rc = cuda_status(cudaMemcpyAsync(&total, dptr + N, sizeof(i64), cudaMemcpyDeviceToHost, st)))) break;
        if ((rc = cuda_status(cudaStreamSynchronize(st)))) break;
        *n_nodes = total;
        if (ptr && (rc = cuda_status(cudaMemcpy(ptr, dptr, (N + 1) * sizeof(i64), cudaMemcpyDeviceToHost)))) break;
        if (fitness && N > 0 &&
            (rc = cuda_status(cudaMemcpy(fitness, c->uf + base, N * sizeof(double), cudaMemcpyDeviceToHost))))
            break;
        if (stats && N > 0 &&
            (rc = cuda_status(cudaMemcpy(stats, c->ustat + base * MSCD_NSTATS, N * MSCD_NSTATS * sizeof(i64),
                                         cudaMemcpyDeviceToHost))))
            break;
        if (nodes_cap < total || (total > 0 && !nodes)) { rc = MSCD_ESMALL; break; }
        if (total > 0) {
            if ((rc = cuda_status(cudaMallocAsync((void **)&dnodes, total * sizeof(i32), st)))) break;
            gather_lists<<<152 * 8, 256, 0, st>>>(c->uoff + base, c->ulen + base, dptr,
                                                  c->scales[scale_idx].comm_nodes, N, dnodes); note_launch();
            if ((rc = cuda_status(cudaMemcpyAsync(nodes, dnodes, total * sizeof(i32), cudaMemcpyDeviceToHost, st))))
                break;
        }
        rc = cuda_status(cudaStreamSynchronize(st));
    } while (0);
    cudaFreeAsync(dptr, st);
    if (dnodes) cudaFreeAsync(dnodes, st);
    cudaStreamSynchronize(st);
    return rc;
}

int mscd_get_communities(mscd_ctx *c, int32_t scale_idx, int64_t *ptr, int64_t ptr_cap, int32_t *nodes,
                         int64_t nodes_cap, double *fitness, int32_t *seed2comm, int64_t *n_comms, int64_t *n_nodes) {
    if (!c || !n_comms || !n_nodes) return MSCD_EINVAL;
    if (!c->have) return MSCD_ENORESULT;
    if (scale_idx < 0 || scale_idx >= c->S) return MSCD_EINVAL;
    MSCD_CUDA(cudaSetDevice(c->device));
    const ScaleResult &r = c->scales[scale_idx];
    *n_comms = r.n_comms;
    *n_nodes = r.n_nodes;
    if (seed2comm && c->N > 0)
        MSCD_CUDA(cudaMemcpy(seed2comm, r.seed2comm, c->N * sizeof(i32), cudaMemcpyDeviceToHost));
    if (fitness && r.n_comms > 0)
        MSCD_CUDA(cudaMemcpy(fitness, r.comm_f, r.n_comms * sizeof(double), cudaMemcpyDeviceToHost));
    if (ptr_cap < r.n_comms + 1 || nodes_cap < r.n_nodes || !ptr || (r.n_nodes > 0 && !nodes)) return MSCD_ESMALL;
    MSCD_CUDA(cudaMemcpy(ptr, r.comm_ptr, (r.n_comms + 1) * sizeof(i64), cudaMemcpyDeviceToHost));
    if (r.n_nodes > 0) MSCD_CUDA(cudaMemcpy(nodes, r.comm_nodes, r.n_nodes * sizeof(i32), cudaMemcpyDeviceToHost));
    return MSCD_OK;
}

int mscd_get_stability_part(mscd_ctx *c, int32_t part, double *nmi_succ, double *nmi_win3, double *nmi_win5) {
    if (!c) return MSCD_EINVAL;
    if (!c->have) return MSCD_ENORESULT;
    if (part < 0 || part >= c->n_parts) return MSCD_EINVAL;
    const size_t S = (size_t)c->S, S1 = S ? S - 1 : 0;
    if (nmi_succ) std::copy_n(c->nmi_succ.begin() + part * S1, S1, nmi_succ);
    if (nmi_win3) std::copy_n(c->win3.begin() + part * S, S, nmi_win3);
    if (nmi_win5) std::copy_n(c->win5.begin() + part * S, S, nmi_win5);
    return MSCD_OK;
}

int mscd_get_stability(mscd_ctx *c, double *nmi_succ, double *nmi_win3, double *nmi_win5) {
    return mscd_get_stability_part(c, 0, nmi_succ, nmi_win3, nmi_win5);
}

int mscd_window_means(const double *nmi_succ, int32_t n_scales, int32_t p, double *out) {
    if (n_scales < 1 || p < 2 || !out || (n_scales > 1 && !nmi_succ)) return MSCD_EINVAL;
    std::vector<double> nmi, w;
    if (n_scales > 1) nmi.assign(nmi_succ, nmi_succ + (n_scales - 1));
    window_means(nmi, n_scales, p, w);
    std::copy(w.begin(), w.end(), out);
    return MSCD_OK;
}

const char *mscd_last_error(mscd_ctx *c) { return c ? c->last_error : ""; }

int mscd_get_run_stats(mscd_ctx *c, mscd_run_stats *out) {
    if (!c || !out) return MSCD_EINVAL;
    if (!c->have) return MSCD_ENORESULT;
    *out = c->stats;
    return MSCD_OK;
}

}  // extern "C"
