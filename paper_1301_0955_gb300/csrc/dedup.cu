// Deduplication of the communities of one scale.
//
// Communities grown from different seeds are the same community iff their
// sorted member lists are equal (the paper keeps community nodes sorted,
// Sec. 3).  Units are grouped by the 64-bit hash of their list in a device
// hash table; the representative of a group is its smallest unit (= seed)
// index; every unit's list is compared element by element with its
// representative's, and the rare unit whose list differs despite an equal
// hash is regrouped exactly by a warp-parallel pass over those units.  Unique communities are
// numbered in order of their representative (smallest generating seed index).
#include <algorithm>

#include "common.cuh"
#include "dedup.cuh"

namespace {

__global__ void table_insert(const u64 *uhash, i64 N, u64 *tkey, i64 *trep, i64 tmask, i64 *uent, u32 *err) {
    for (i64 u = (i64)blockIdx.x * blockDim.x + threadIdx.x; u < N; u += (i64)gridDim.x * blockDim.x) {
        const u64 key = uhash[u];
        i64 h = (i64)(key & (u64)tmask);
        i64 p = 0;
        for (; p <= tmask; ++p) {
            const u64 old = atomicCAS((unsigned long long *)&tkey[h], 0ull, (unsigned long long)key);
            if (old == 0ull || old == key) break;
            h = (h + 1) & tmask;
        }
        if (p > tmask) {
            atomicOr(err, 1u);
            h = 0;
        }
        uent[u] = h;
        atomicMin((long long *)&trep[h], (long long)u);
    }
}

// Warp per unit: compare the list with the representative's.
__global__ void verify(const i64 *uoff, const i32 *ulen, const i32 *nodes, const i64 *uent, const i64 *trep, i64 N,
                       i64 *urep, unsigned long long *n_coll) {
    const int lane = threadIdx.x & 31;
    const i64 warps = (i64)gridDim.x * (blockDim.x >> 5);
    for (i64 u = (i64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < N; u += warps) {
        const i64 r = trep[uent[u]];
        bool same = true;
        if (r != u) {
            same = ulen[u] == ulen[r];
            if (same) {
                const i32 *a = nodes + uoff[u], *b = nodes + uoff[r];
                const int m = ulen[u];
                bool diff = false;
                for (int i = lane; i < m; i += 32) diff |= a[i] != b[i];
                same = !__any_sync(FULL_MASK, diff);
            }
        }
        if (lane == 0) {
            urep[u] = same ? r : -1;
            if (!same) atomicAdd(n_coll, 1ull);
        }
    }
}

// Exact regrouping of the units whose list differed from their hash group's
// representative (equal lists have equal hashes, so every equal-list class
// of such units lies inside this set).  The set is listed in ascending unit
// order; a warp per listed unit finds the first listed unit with the same
// hash, length and list (itself at the latest), which is the smallest unit of
// its class: every class gets its smallest unit as representative, as the
// sequential pairwise pass would.
__global__ void flag_collisions(const i64 *urep, i64 N, i64 *flag) {
    for (i64 u = (i64)blockIdx.x * blockDim.x + threadIdx.x; u < N; u += (i64)gridDim.x * blockDim.x)
        flag[u] = urep[u] == -1 ? 1 : 0;
}

__global__ void list_collisions(const i64 *flag, const i64 *pos, i64 N, i64 *list) {
    for (i64 u = (i64)blockIdx.x * blockDim.x + threadIdx.x; u < N; u += (i64)gridDim.x * blockDim.x)
        if (flag[u]) list[pos[u]] = u;
}

__global__ void regroup_collisions(const i64 *list, const i64 *n_list, const u64 *uhash, const i64 *uoff,
                                   const i32 *ulen, const i32 *nodes, i64 *urep) {
    const int lane = threadIdx.x & 31;
    const i64 X = *n_list;
    const i64 warps = (i64)gridDim.x * (blockDim.x >> 5);
    for (i64 j = (i64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < X; j += warps) {
        const i64 u = list[j];
        const u64 hu = uhash[u];
        const i32 lu = ulen[u];
        const i32 *a = nodes + uoff[u];
        i64 rep = u;
        for (i64 b = 0; b < j; b += 32) {
            // candidates of this chunk with the same hash and length, then each
            // compared in ascending order until one equals
            const i64 i = b + lane;
            const i64 v = i < j ? list[i] : -1;
            u32 cand = __ballot_sync(FULL_MASK, v >= 0 && uhash[v] == hu && ulen[v] == lu);
            bool found = false;
            while (cand) {
                const int l = __ffs(cand) - 1;
                cand &= cand - 1;
                const i64 w = __shfl_sync(FULL_MASK, v, l);
                const i32 *c = nodes + uoff[w];
                bool diff = false;
                for (i32 k = lane; k < lu; k += 32) diff |= a[k] != c[k];
                if (!__any_sync(FULL_MASK, diff)) {
                    rep = w;
                    found = true;
                    break;
                }
            }
            if (found) break;
        }
        if (lane == 0) urep[u] = rep;
    }
}

__global__ void mark_reps(const i64 *urep, i64 N, i64 *flag) {
    for (i64 u = (i64)blockIdx.x * blockDim.x + threadIdx.x; u < N; u += (i64)gridDim.x * blockDim.x)
        flag[u] = urep[u] == u ? 1 : 0;
}

__global__ void fill_comms(const i64 *urep, const i64 *cid, const i32 *ulen, const double *uf, const u64 *uhash,
                           i64 N, i64 *clen, double *cf, u64 *chash, i64 *crep, i32 *seed2comm) {
    for (i64 u = (i64)blockIdx.x * blockDim.x + threadIdx.x; u < N; u += (i64)gridDim.x * blockDim.x) {
        const i64 r = urep[u];
        seed2comm[u] = (i32)cid[r];
        if (r == u) {
            const i64 c = cid[u];
            clen[c] = ulen[u];
            cf[c] = uf[u];
            chash[c] = uhash[u];
            crep[c] = u;
        }
    }
}

__global__ void copy_lists(const i64 *crep, const i64 *cptr, const i64 *uoff, const i32 *nodes, i64 C, i32 *cnodes) {
    const int lane = threadIdx.x & 31;
    const i64 warps = (i64)gridDim.x * (blockDim.x >> 5);
    for (i64 c = (i64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < C; c += warps) {
        const i32 *src = nodes + uoff[crep[c]];
        i32 *dst = cnodes + cptr[c];
        const i64 m = cptr[c + 1] - cptr[c];
        for (i64 i = lane; i < m; i += 32) dst[i] = src[i];
    }
}

}  // namespace

void scale_result_free(ScaleResult *r) {
    cudaFree(r->comm_ptr);
    cudaFree(r->comm_nodes);
    cudaFree(r->comm_f);
    cudaFree(r->seed2comm);
    cudaFree(r->comm_hash);
    *r = ScaleResult{};
}

int dedup_scale(const i64 *uoff, const i32 *ulen, const u64 *uhash, const double *uf, const i32 *nodes, i64 N,
                ScaleResult *out, cudaStream_t st) {
    *out = ScaleResult{};
    if (N <= 0) {
        MSCD_CUDA(cudaMalloc((void **)&out->comm_ptr, sizeof(i64)));
        MSCD_CUDA(cudaMemsetAsync(out->comm_ptr, 0, sizeof(i64), st));
        return MSCD_OK;
    }
    i64 T = 1;
    while (T < 2 * N) T <<= 1;
    u64 *tkey = nullptr;
    i64 *trep = nullptr, *uent = nullptr, *urep = nullptr, *flag = nullptr, *cid = nullptr, *clen = nullptr,
        *crep = nullptr, *tot = nullptr;
    unsigned long long *ncoll = nullptr;
    u32 *err = nullptr;
    int rc = MSCD_OK;
    const unsigned blocks = (unsigned)std::min<i64>((N + 255) / 256, 152 * 16);
    const unsigned wblocks = (unsigned)std::min<i64>((N + 7) / 8, 152 * 16);
    do {
        if ((rc = cuda_status(cudaMallocAsync((void **)&tkey, T * sizeof(u64), st)))) break;
        if ((rc = cuda_status(cudaMallocAsync((void **)&trep, T * sizeof(i64), st)))) break;
        if ((rc = cuda_status(cudaMallocAsync((void **)&uent, N * sizeof(i64), st)))) break;
        if ((rc = cuda_status(cudaMallocAsync((void **)&urep, N * sizeof(i64), st)))) break;
        if ((rc = cuda_status(cudaMallocAsync((void **)&flag, (N + 1) * sizeof(i64), st)))) break;
        if ((rc = cuda_status(cudaMallocAsync((void **)&cid, (N + 1) * sizeof(i64), st)))) break;
        if ((rc = cuda_status(cudaMallocAsync((void **)&tot, 2 * sizeof(i64) + 2 * sizeof(unsigned long long), st))))
            break;
        ncoll = (unsigned long long *)(tot + 1);
        err = (u32 *)(tot + 2);
        if ((rc = cuda_status(cudaMemsetAsync(tkey, 0, T * sizeof(u64), st)))) break;
        if ((rc = cuda_status(cudaMemsetAsync(trep, 0x7f, T * sizeof(i64), st)))) break;
        if ((rc = cuda_status(cudaMemsetAsync(tot, 0, 2 * sizeof(i64) + 2 * sizeof(unsigned long long), st)))) break;
        table_insert<<<blocks, 256, 0, st>>>(uhash, N, tkey, trep, T - 1, uent, err); note_launch();
        verify<<<wblocks, 256, 0, st>>>(uoff, ulen, nodes, uent, trep, N, urep, ncoll); note_launch();
        unsigned long long h_coll = 0;
        u32 h_err = 0;
        if ((rc = cuda_status(cudaMemcpyAsync(&h_coll, ncoll, sizeof(h_coll), cudaMemcpyDeviceToHost, st)))) break;
        if ((rc = cuda_status(cudaMemcpyAsync(&h_err, err, sizeof(h_err), cudaMemcpyDeviceToHost, st)))) break;
        if ((rc = cuda_status(cudaStreamSynchronize(st)))) break;
        if (h_err) { rc = MSCD_EDEVICE; break; }
        if (h_coll) {
            // flag is reused below (mark_reps overwrites it); cid holds the positions
            flag_collisions<<<blocks, 256, 0, st>>>(urep, N, flag); note_launch();
            if ((rc = scan_exclusive_i64(flag, cid, N, tot, st))) break;
            list_collisions<<<blocks, 256, 0, st>>>(flag, cid, N, uent); note_launch();  // uent is free now
            const unsigned rblocks = (unsigned)std::max<u64>(1, std::min<u64>((h_coll + 7) / 8, 152 * 16));
            regroup_collisions<<<rblocks, 256, 0, st>>>(uent, tot, uhash, uoff, ulen, nodes, urep); note_launch();
        }
        mark_reps<<<blocks, 256, 0, st>>>(urep, N, flag); note_launch();
        if ((rc = scan_exclusive_i64(flag, cid, N, tot, st))) break;
        i64 C = 0;
        if ((rc = cuda_status(cudaMemcpyAsync(&C, tot, sizeof(i64), cudaMemcpyDeviceToHost, st)))) break;
        if ((rc = cuda_status(cudaStreamSynchronize(st)))) break;
        out->n_comms = C;
        if ((rc = cuda_status(cudaMallocAsync((void **)&clen, (C + 1) * sizeof(i64), st)))) break;
        if ((rc = cuda_status(cudaMallocAsync((void **)&crep, (C + 1) * sizeof(i64), st)))) break;
        if ((rc = cuda_status(cudaMalloc((void **)&out->comm_ptr, (C + 1) * sizeof(i64))))) break;
        if ((rc = cuda_status(cudaMalloc((void **)&out->comm_f, std::max<i64>(C, 1) * sizeof(double))))) break;
        if ((rc = cuda_status(cudaMalloc((void **)&out->seed2comm, N * sizeof(i32))))) break;
        if ((rc = cuda_status(cudaMalloc((void **)&out->comm_hash, std::max<i64>(C, 1) * sizeof(u64))))) break;
        fill_comms<<<blocks, 256, 0, st>>>(urep, cid, ulen, uf, uhash, N, clen, out->comm_f, out->comm_hash, crep,
                                           out->seed2comm); note_launch();
        if ((rc = scan_exclusive_i64(clen, out->comm_ptr, C, out->comm_ptr + C, st))) break;
        i64 total = 0;
        if ((rc = cuda_status(cudaMemcpyAsync(&total, out->comm_ptr + C, sizeof(i64), cudaMemcpyDeviceToHost, st))))
            break;
        if ((rc = cuda_status(cudaStreamSynchronize(st)))) break;
        out->n_nodes = total;
        if ((rc = cuda_status(cudaMalloc((void **)&out->comm_nodes, std::max<i64>(total, 1) * sizeof(i32))))) break;
        const unsigned cblocks = (unsigned)std::max<i64>(1, std::min<i64>((C + 7) / 8, 152 * 16));
        if (C > 0) { copy_lists<<<cblocks, 256, 0, st>>>(crep, out->comm_ptr, uoff, nodes, C, out->comm_nodes); note_launch(); }
        rc = cuda_status(cudaGetLastError());
    } while (0);
    cudaFreeAsync(tkey, st);
    cudaFreeAsync(trep, st);
    cudaFreeAsync(uent, st);
    cudaFreeAsync(urep, st);
    cudaFreeAsync(flag, st);
    cudaFreeAsync(cid, st);
    cudaFreeAsync(clen, st);
    cudaFreeAsync(crep, st);
    cudaFreeAsync(tot, st);
    if (rc != MSCD_OK) {
        cudaStreamSynchronize(st);
        scale_result_free(out);
    }
    return rc;
}
