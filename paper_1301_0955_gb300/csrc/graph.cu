// Graph preparation on the device: checks of the CSR input, exact
// fixed-point weights, weighted degrees k_u and log k_u.
//
// The method grows communities over an undirected weighted network with
// d_in + d_out = k_u (Sec. 2); sums of weights must be exact so that every
// decision is independent of summation order.  An FP32 weight is odd * 2^e;
// with the unit 2^ue, ue = the smallest such e over all weights (the largest
// power of two dividing every weight), each weight is the exact integer
// odd * 2^(e - ue).  Totals must stay below 2^62 (else MSCD_ERANGE).
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace {

enum : u32 {
    CAT_STRUCT = 1u,
    CAT_WEIGHT = 2u,
    CAT_SELF = 4u,
    CAT_UNSORTED = 8u,
    CAT_DUP = 16u,
    CAT_NOTSYM = 32u,
    CAT_RANGE = 64u,
};

struct PrepState {
    u32 mask;
    int min_lowbit;
    unsigned long long total;  // exact volume (valid while total_d < 2^63)
    double total_d;            // coarse volume, guards against wrap-around
    unsigned long long kmax;   // largest degree
};

__global__ void check_row_ptr(const i64 *rp, i64 n, PrepState *ps) {
    i64 u = (i64)blockIdx.x * blockDim.x + threadIdx.x;
    if (u > n) return;
    bool bad = (u == 0) ? (rp[0] != 0) : (rp[u] < rp[u - 1]);
    if (bad) atomicOr(&ps->mask, CAT_STRUCT);
}

// lowbit exponent of a positive finite FP32 value: w = odd * 2^lowbit
__device__ __forceinline__ int f32_lowbit(float w, u32 *odd) {
    u32 bits = __float_as_uint(w);
    u32 E = (bits >> 23) & 0xffu, M = bits & 0x7fffffu;
    u32 sig = E ? (M | 0x800000u) : M;
    int e0 = E ? (int)E - 150 : -149;
    int tz = __ffs((int)sig) - 1;
    *odd = sig >> tz;
    return e0 + tz;
}

// Warp per row: per-entry checks (column range, weight, self-loop, order,
// duplicate, symmetric partner with the same weight) and the smallest lowbit.
__global__ void check_entries(const i64 *rp, const i32 *col, const float *w, i64 n, PrepState *ps) {
    const int lane = threadIdx.x & 31;
    const i64 warps = (i64)gridDim.x * (blockDim.x >> 5);
    u32 mask = 0;
    int lowbit = INT32_MAX;
    for (i64 u = (i64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < n; u += warps) {
        const i64 rs = rp[u], re = rp[u + 1];
        for (i64 e = rs + lane; e < re; e += 32) {
            const i32 c = col[e];
            if (c < 0 || (i64)c >= n) {
                mask |= CAT_STRUCT;
                continue;
            }
            float we = 0.0f;
            if (w) {
                we = w[e];
                if (!(isfinite(we) && we > 0.0f)) mask |= CAT_WEIGHT;
                else {
                    u32 odd;
                    lowbit = min(lowbit, f32_lowbit(we, &odd));
                }
            }
            if ((i64)c == u) mask |= CAT_SELF;
            if (e > rs) {
                const i32 p = col[e - 1];
                if (c < p) mask |= CAT_UNSORTED;
                else if (c == p) mask |= CAT_DUP;
            }
            // partner entry c -> u by binary search in row c
            i64 lo = rp[c], hi = rp[(i64)c + 1];
            while (lo < hi) {
                i64 mid = lo + ((hi - lo) >> 1);
                if ((i64)col[mid] < u) lo = mid + 1;
                else hi = mid;
            }
            if (lo >= rp[(i64)c + 1] || (i64)col[lo] != u) mask |= CAT_NOTSYM;
            else if (w && !(w[lo] == we)) mask |= CAT_NOTSYM;
        }
    }
    mask = __reduce_or_sync(FULL_MASK, mask);
    lowbit = __reduce_min_sync(FULL_MASK, lowbit);
    if (lane == 0) {
        if (mask) atomicOr(&ps->mask, mask);
        if (lowbit != INT32_MAX) atomicMin(&ps->min_lowbit, lowbit);
    }
}

__global__ void fixed_weights(const float *w, i64 nnz, int ue, i64 *wfx, PrepState *ps) {
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (i64)gridDim.x * blockDim.x) {
        u32 odd;
        int sh = f32_lowbit(w[e], &odd) - ue;  // >= 0
        int len = 32 - __clz((int)odd);
        bool ok = (odd == 1u) ? (sh <= 62) : (len + sh <= 62);
        if (!ok) {
            atomicOr(&ps->mask, CAT_RANGE);
            wfx[e] = 0;
        } else {
            wfx[e] = (i64)odd << sh;
        }
    }
}

// Warp per row: k_u = sum of weights (exact), log k_u, and the volume.
__global__ void degrees(const i64 *rp, const i64 *wfx, i64 n, i64 *k, float *logk, PrepState *ps) {
    const int lane = threadIdx.x & 31;
    const i64 warps = (i64)gridDim.x * (blockDim.x >> 5);
    unsigned long long tot = 0, kmax = 0;
    double tot_d = 0.0;
    for (i64 u = (i64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < n; u += warps) {
        const i64 rs = rp[u], re = rp[u + 1];
        unsigned long long s = 0;
        double sd = 0.0;
        if (wfx) {
            for (i64 e = rs + lane; e < re; e += 32) {
                s += (unsigned long long)wfx[e];
                sd += (double)wfx[e];
            }
            for (int o = 16; o; o >>= 1) {
                s += __shfl_xor_sync(FULL_MASK, s, o);
                sd += __shfl_xor_sync(FULL_MASK, sd, o);
            }
        } else {
            s = (unsigned long long)(re - rs);
            sd = (double)(re - rs);
        }
        if (lane == 0) {
            k[u] = (i64)s;
            logk[u] = s ? logf((float)(i64)s) : 0.0f;
            tot += s;
            kmax = s > kmax ? s : kmax;
            tot_d += sd;
        }
    }
    if (lane == 0) {
        atomicAdd(&ps->total, tot);
        atomicAdd(&ps->total_d, tot_d);
        atomicMax(&ps->kmax, kmax);
    }
}

int first_category(u32 mask) {
    if (mask & CAT_STRUCT) return MSCD_EINVAL;
    if (mask & CAT_WEIGHT) return MSCD_EWEIGHT;
    if (mask & CAT_SELF) return MSCD_ESELFLOOP;
    if (mask & CAT_UNSORTED) return MSCD_EUNSORTED;
    if (mask & CAT_DUP) return MSCD_EDUP;
    if (mask & CAT_NOTSYM) return MSCD_ENOTSYM;
    if (mask & CAT_RANGE) return MSCD_ERANGE;
    return MSCD_OK;
}

}  // namespace

int graph_prepare(i64 n, const i64 *rp, const i32 *col, const float *w, DevGraph *g, i64 **wfx_out, i64 **k_out,
                  float **logk_out, cudaStream_t st) {
    *wfx_out = nullptr;
    *k_out = nullptr;
    *logk_out = nullptr;
    PrepState *ps = nullptr;
    PrepState init{0u, INT32_MAX, 0ull, 0.0, 0ull};
    MSCD_CUDA(cudaMallocAsync((void **)&ps, sizeof(PrepState), st));
    int rc = MSCD_OK;
    PrepState h{};
    i64 nnz = 0;
    do {
        if ((rc = cuda_status(cudaMemcpyAsync(ps, &init, sizeof(init), cudaMemcpyHostToDevice, st)))) break;
        check_row_ptr<<<(unsigned)((n + 1 + 255) / 256), 256, 0, st>>>(rp, n, ps); note_launch();
        if ((rc = cuda_status(cudaMemcpyAsync(&h, ps, sizeof(h), cudaMemcpyDeviceToHost, st)))) break;
        if ((rc = cuda_status(cudaStreamSynchronize(st)))) break;
        if (h.mask) { rc = MSCD_EINVAL; break; }
        if ((rc = cuda_status(cudaMemcpyAsync(&nnz, rp + n, sizeof(i64), cudaMemcpyDeviceToHost, st)))) break;
        if ((rc = cuda_status(cudaStreamSynchronize(st)))) break;
        const unsigned row_blocks = (unsigned)std::max<i64>(1, std::min<i64>((n + 7) / 8, 152 * 64));
        if (n > 0) { check_entries<<<row_blocks, 256, 0, st>>>(rp, col, w, n, ps); note_launch(); }
        if ((rc = cuda_status(cudaMemcpyAsync(&h, ps, sizeof(h), cudaMemcpyDeviceToHost, st)))) break;
        if ((rc = cuda_status(cudaStreamSynchronize(st)))) break;
        if ((rc = first_category(h.mask))) break;
        int ue = 0;
        if (w && nnz > 0) {
            ue = h.min_lowbit;
            if ((rc = cuda_status(cudaMalloc((void **)wfx_out, (size_t)nnz * sizeof(i64))))) break;
            fixed_weights<<<(unsigned)std::min<i64>((nnz + 255) / 256, 152 * 32), 256, 0, st>>>(w, nnz, ue,
                                                                                             *wfx_out, ps); note_launch();
        }
        if ((rc = cuda_status(cudaMalloc((void **)k_out, (size_t)std::max<i64>(n, 1) * sizeof(i64))))) break;
        if ((rc = cuda_status(cudaMalloc((void **)logk_out, (size_t)std::max<i64>(n, 1) * sizeof(float))))) break;
        if (n > 0) { degrees<<<row_blocks, 256, 0, st>>>(rp, *wfx_out, n, *k_out, *logk_out, ps); note_launch(); }
        if ((rc = cuda_status(cudaMemcpyAsync(&h, ps, sizeof(h), cudaMemcpyDeviceToHost, st)))) break;
        if ((rc = cuda_status(cudaStreamSynchronize(st)))) break;
        if ((rc = first_category(h.mask))) break;
        if (h.total_d >= 0x1p63 || h.total >= (1ull << 62)) { rc = MSCD_ERANGE; break; }
        g->n = n;
        g->nnz = nnz;
        g->rp = rp;
        g->col = col;
        g->wfx = *wfx_out;
        g->k = *k_out;
        g->logk = *logk_out;
        g->unit_exp = ue;
        g->volume = (i64)h.total;
        g->kmax = (i64)h.kmax;
    } while (0);
    cudaFreeAsync(ps, st);
    if (rc != MSCD_OK) {
        cudaStreamSynchronize(st);
        if (*wfx_out) cudaFree(*wfx_out);
        if (*k_out) cudaFree(*k_out);
        if (*logk_out) cudaFree(*logk_out);
        *wfx_out = nullptr;
        *k_out = nullptr;
        *logk_out = nullptr;
    }
    return rc;
}
