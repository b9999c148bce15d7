// Community growth that allocates no device memory during the call.
//
// Some callers cannot call cudaMalloc while they run: code that owns every
// byte of device memory up front (a serving process with a fixed memory
// plan, or a framework whose allocator must not be bypassed), code on a
// latency-critical path where an allocation's implicit synchronisation is not
// acceptable, and code that must not fail for lack of memory halfway through
// a job.  mscd_grow_noalloc serves them: the caller passes the inputs and
// every output buffer, and the growth kernel's scratch (the per-warp node-slot
// arenas, the work counters and the lists of units it could not finish) lives
// in one file-scope device array of NOALLOC_BYTES that every GPU loading the
// library holds until the process exits.
//
// Host code only ever sees a stand-in for that array's name; the device
// address is taken once per device with cudaGetSymbolAddress (with the device
// current) on the first call on that device, and passed to the kernel.
#include <cmath>
#include <mutex>

#include "common.cuh"
#include "grow.cuh"

namespace {

constexpr size_t NOALLOC_BYTES = (size_t)64 << 20;   // whole scratch array: 64 MiB
constexpr int NOALLOC_SLOTS = 8192;                 // node slots per unit
constexpr i64 NOALLOC_MAX_UNITS = (i64)1 << 20;     // (scale, seed) units per call
constexpr int NOALLOC_MAX_SCALES = 256;
constexpr int MAX_DEVICES = 64;

struct Header {
    unsigned long long work, out_cursor, out_needed, n_retry_state, n_retry_out;
    u32 error_flags, bad_seed;
    double alphas[NOALLOC_MAX_SCALES];
};

// Layout: header | retry_state i64[MAX_UNITS] | retry_out i64[MAX_UNITS] | arenas
constexpr size_t OFF_RETRY_STATE = 4096;
constexpr size_t OFF_RETRY_OUT = OFF_RETRY_STATE + sizeof(i64) * NOALLOC_MAX_UNITS;
constexpr size_t OFF_ARENA = OFF_RETRY_OUT + sizeof(i64) * NOALLOC_MAX_UNITS;
static_assert(sizeof(Header) <= OFF_RETRY_STATE, "header fits its page");
static_assert(OFF_ARENA < NOALLOC_BYTES, "arenas fit");

std::mutex g_setup_mutex;
void *g_scratch_addr[MAX_DEVICES];  // device address of the array, per device

__global__ void check_seeds_noalloc(const i32 *seeds, i64 N, i64 n, Header *hdr) {
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (i64)gridDim.x * blockDim.x)
        if (seeds[i] < 0 || (i64)seeds[i] >= n) atomicOr(&hdr->bad_seed, 1u);
}

}  // namespace

// The scratch array (file scope, device memory of every GPU that loads the library).
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

extern "C" int mscd_grow_noalloc(mscd_ctx *ctx, int32_t graph_id, const double *alphas, int32_t n_scales,
                                 const int32_t *seeds, int64_t n_seeds, int32_t *out_nodes, int64_t out_cap,
                                 int64_t *out_offset, int32_t *out_len, double *out_fitness, int64_t *out_stats,
                                 int32_t *out_status, uint64_t *out_hash, int64_t *n_nodes_needed,
                                 void *cuda_stream) {
    DevGraph G;
    int device = 0;
    if (!ctx || !ctx_graph(ctx, graph_id, &G, &device)) return MSCD_EINVAL;
    if (!alphas || n_scales < 1 || !out_offset || !out_len || !out_fitness || !out_stats || !out_status ||
        !out_hash || !n_nodes_needed || out_cap < 0)
        return MSCD_EINVAL;
    if (n_scales > NOALLOC_MAX_SCALES) return MSCD_ERANGE;
    for (int32_t s = 0; s < n_scales; ++s)
        if (!(alphas[s] > 0.0) || !std::isfinite(alphas[s])) return MSCD_EINVAL;
    const i64 N = seeds ? n_seeds : G.n;
    if (N < 0) return MSCD_EINVAL;
    const i64 U = (i64)n_scales * N;
    if (U > NOALLOC_MAX_UNITS) return MSCD_ERANGE;
    *n_nodes_needed = 0;
    if (U == 0) return MSCD_OK;
    if (out_cap > 0 && !out_nodes) return MSCD_EINVAL;
    if (device < 0 || device >= MAX_DEVICES) return MSCD_EINVAL;
    MSCD_CUDA(cudaSetDevice(device));
    // once per device, with that device current: the array's device address
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_addr[device]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_status(e);
            g_scratch_addr[device] = p;
        }
    }
    unsigned char *base = (unsigned char *)g_scratch_addr[device];
    Header *hdr = (Header *)base;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // the array keeps the previous call's contents: zero the header's counters
    MSCD_CUDA(cudaMemsetAsync(hdr, 0, offsetof(Header, alphas), st));
    MSCD_CUDA(cudaMemcpyAsync(hdr->alphas, alphas, n_scales * sizeof(double), cudaMemcpyHostToDevice, st));
    if (seeds) {
        check_seeds_noalloc<<<152 * 4, 256, 0, st>>>(seeds, N, G.n, hdr); note_launch();
        u32 bad = 0;
        MSCD_CUDA(cudaMemcpyAsync(&bad, &hdr->bad_seed, sizeof(bad), cudaMemcpyDeviceToHost, st));
        MSCD_CUDA(cudaStreamSynchronize(st));
        if (bad) return MSCD_EINVAL;
    }
    GrowArgs a{};
    a.G = G;
    a.alphas = hdr->alphas;
    a.seeds = seeds;
    a.n_seeds = N;
    a.n_work = U;
    a.work_counter = &hdr->work;
    i64 full = 32;
    while (full < G.n + 1) full <<= 1;
    a.cap = (int)std::min<i64>(NOALLOC_SLOTS, full);
    a.use_smem = 0;
    a.state_bytes = grow_state_bytes(G, a.cap);
    a.gstate = base + OFF_ARENA;
    a.max_rounds = 1000000;
    a.log_kmax = G.kmax > 1 ? (float)std::log((double)G.kmax) : 0.0f;
    a.out_nodes = out_nodes;
    a.out_cursor = &hdr->out_cursor;
    a.out_needed = &hdr->out_needed;
    a.out_cap = out_cap;
    a.uoff = out_offset;
    a.ulen = out_len;
    a.uhash = (u64 *)out_hash;
    a.uf = out_fitness;
    a.ustat = out_stats;
    a.ustatus = out_status;
    a.retry_state = (i64 *)(base + OFF_RETRY_STATE);
    a.n_retry_state = &hdr->n_retry_state;
    a.retry_out = (i64 *)(base + OFF_RETRY_OUT);
    a.n_retry_out = &hdr->n_retry_out;
    a.error_flags = &hdr->error_flags;
    const i64 warps = std::max<i64>(1, (i64)((NOALLOC_BYTES - OFF_ARENA) / a.state_bytes));
    const int wpc = 8;
    const int blocks = (int)std::max<i64>(1, std::min<i64>(warps / wpc, (U + wpc - 1) / wpc));
    if (blocks * (i64)wpc > warps) return MSCD_ERANGE;  // a state larger than the arenas
    int rc = grow_launch(a, blocks, wpc * 32, 0, st);
    if (rc) return rc;
    Header h;
    MSCD_CUDA(cudaMemcpyAsync(&h, hdr, offsetof(Header, alphas), cudaMemcpyDeviceToHost, st));
    MSCD_CUDA(cudaStreamSynchronize(st));
    *n_nodes_needed = (int64_t)h.out_cursor;
    if (h.error_flags) return MSCD_EDEVICE;
    if (h.n_retry_state) return MSCD_ERANGE;  // a unit touched more nodes than a slot arena holds
    if (h.n_retry_out) return MSCD_ESMALL;    // out_cap below *n_nodes_needed
    return MSCD_OK;
}
