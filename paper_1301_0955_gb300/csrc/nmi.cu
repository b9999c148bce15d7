// Overlapping NMI between the community sets of two scales (Sec. 4 measures
// the change between successive sets with the NMI for overlapping
// communities of Lancichinetti, Fortunato & Kertesz).
//
// Each community is a binary variable over the n nodes; h(p) = -p log2 p.
//   H(X_k|Y_l) = H(X_k, Y_l) - H(Y_l), admitted only if
//                h(P11) + h(P00) > h(P01) + h(P10)
//                (not admitted when {n11, n00} = {n01, n10} as multisets)
//   H(X_k|Y)   = min over admitted l, else H(X_k)
//   H(X|Y)     = mean_k H(X_k|Y) / H(X_k)   (0 for a community of all n nodes)
//   N          = 1 - [H(X|Y) + H(Y|X)] / 2
//
// Only two kinds of pair can be admitted, so only they are evaluated:
//   * pairs that share a node (counted through the node -> communities map);
//   * disjoint pairs with |X_k| + |Y_l| > n/2.  For a disjoint pair with
//     s = (|X_k| + |Y_l|)/n <= 1/2: h(P00) = h(1-s) <= h(s) (h(1-s) <= h(s)
//     on [0, 1/2]) <= h(P10) + h(P01) (h concave with h(0) = 0 is
//     subadditive), and h(P11) = 0, so the admission test fails.
// Per-k results are reduced in a fixed order, so the value is deterministic.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "dedup.cuh"

namespace {

__device__ __forceinline__ double hterm(i64 c, double inv_n) {
    if (c <= 0) return 0.0;
    const double p = (double)c * inv_n;
    return -p * log2(p);
}

// Candidate H(X_k|Y_l) if admitted, else +inf.
__device__ __forceinline__ double cond_candidate(i64 n11, i64 sx, i64 sy, i64 n, double inv_n) {
    const i64 n10 = sx - n11, n01 = sy - n11, n00 = n - n11 - n10 - n01;
    const i64 lo1 = min(n11, n00), hi1 = max(n11, n00), lo2 = min(n01, n10), hi2 = max(n01, n10);
    if (lo1 == lo2 && hi1 == hi2) return __builtin_huge_val();
    const double h11 = hterm(n11, inv_n), h00 = hterm(n00, inv_n), h01 = hterm(n01, inv_n), h10 = hterm(n10, inv_n);
    if (!(h11 + h00 > h01 + h10)) return __builtin_huge_val();
    return (h11 + h10 + h01 + h00) - (hterm(sy, inv_n) + hterm(n - sy, inv_n));
}

__global__ void count_memberships(const i32 *nodes, i64 m, i32 *cnt) {
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (i64)gridDim.x * blockDim.x)
        atomicAdd(&cnt[nodes[e]], 1);
}

__global__ void widen_i32(const i32 *a, i64 n, i64 *b) {
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) b[i] = a[i];
}

// Warp per community l of Y: append l to the list of each member.
__global__ void fill_memberships(const i64 *cptr, const i32 *nodes, i64 C, const i64 *mptr, i32 *cursor, i32 *mlist) {
    const int lane = threadIdx.x & 31;
    const i64 warps = (i64)gridDim.x * (blockDim.x >> 5);
    for (i64 l = (i64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); l < C; l += warps)
        for (i64 e = cptr[l] + lane; e < cptr[l + 1]; e += 32) {
            const i32 u = nodes[e];
            mlist[mptr[u] + atomicAdd(&cursor[u], 1)] = (i32)l;
        }
}

// Warp per community k of X: table size for the communities of Y it meets.
__global__ void table_sizes(const i64 *xptr, const i32 *xnodes, i64 CX, const i32 *ycnt, i64 CY, i64 *tsz) {
    const int lane = threadIdx.x & 31;
    const i64 warps = (i64)gridDim.x * (blockDim.x >> 5);
    for (i64 k = (i64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); k < CX; k += warps) {
        i64 s = 0;
        for (i64 e = xptr[k] + lane; e < xptr[k + 1]; e += 32) s += ycnt[xnodes[e]];
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(FULL_MASK, s, o);
        s = min(s, CY);
        i64 t = 2;
        while (t < 2 * s) t <<= 1;
        if (lane == 0) tsz[k] = t;
    }
}

__device__ __forceinline__ u32 hash_comm(i32 l) { return (u32)l * 0x9E3779B1u; }

// Warp per community k of X: intersections with every Y_l it meets, then
// the minimum admitted conditional entropy, normalised.
__global__ void cond_entropy(const i64 *xptr, const i32 *xnodes, i64 CX, const i64 *yptr, i64 CY, const i64 *mptr,
                             const i32 *mlist, const i64 *toff, i32 *tkey, i32 *tcnt, const i32 *big, i64 nbig, i64 n,
                             double *term) {
    const int lane = threadIdx.x & 31;
    const i64 warps = (i64)gridDim.x * (blockDim.x >> 5);
    const double inv_n = 1.0 / (double)n;
    for (i64 k = (i64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); k < CX; k += warps) {
        const i64 sx = xptr[k + 1] - xptr[k];
        i32 *keys = tkey + toff[k];
        i32 *cnts = tcnt + toff[k];
        const u32 tm = (u32)(toff[k + 1] - toff[k] - 1);
        for (i64 e = xptr[k] + lane; e < xptr[k + 1]; e += 32) {
            const i32 u = xnodes[e];
            for (i64 j = mptr[u]; j < mptr[u + 1]; ++j) {
                const i32 l = mlist[j];
                u32 h = hash_comm(l) & tm;
                for (u32 p = 0; p <= tm; ++p) {
                    const i32 old = atomicCAS(&keys[h], -1, l);
                    if (old == -1 || old == l) {
                        atomicAdd(&cnts[h], 1);
                        break;
                    }
                    h = (h + 1u) & tm;
                }
            }
        }
        __syncwarp();
        const double Hx = hterm(sx, inv_n) + hterm(n - sx, inv_n);
        double best = Hx;
        for (u32 t = lane; t <= tm; t += 32) {
            const i32 l = keys[t];
            if (l < 0) continue;
            best = min(best, cond_candidate(cnts[t], sx, yptr[l + 1] - yptr[l], n, inv_n));
        }
        // disjoint partners that can be admitted: |X_k| + |Y_l| > n/2
        for (i64 b = lane; b < nbig; b += 32) {
            const i32 l = big[b];
            const i64 sy = yptr[l + 1] - yptr[l];
            if (2 * (sx + sy) <= n) continue;
            u32 h = hash_comm(l) & tm;
            bool met = false;
            for (u32 p = 0; p <= tm; ++p) {
                const i32 x = keys[h];
                if (x == -1) break;
                if (x == l) {
                    met = true;
                    break;
                }
                h = (h + 1u) & tm;
            }
            if (!met) best = min(best, cond_candidate(0, sx, sy, n, inv_n));
        }
        for (int o = 16; o; o >>= 1) best = min(best, __shfl_xor_sync(FULL_MASK, best, o));
        if (lane == 0) term[k] = Hx > 0.0 ? best / Hx : 0.0;
    }
}

// Fixed-order sum of term[0..m) by one block.
__global__ void sum_fixed(const double *term, i64 m, double *out) {
    __shared__ double part[1024];
    double s = 0.0;
    for (i64 i = threadIdx.x; i < m; i += blockDim.x) s += term[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = part[0];
}

__global__ void list_big(const i64 *yptr, i64 CY, i64 n, i32 *big, unsigned long long *nbig) {
    // communities of Y with 2|Y_l| > n - 2: the only ones that can meet the
    // disjoint admission condition with some X_k of size >= 1
    for (i64 l = (i64)blockIdx.x * blockDim.x + threadIdx.x; l < CY; l += (i64)gridDim.x * blockDim.x)
        if (2 * (yptr[l + 1] - yptr[l] + 1) > n) big[atomicAdd(nbig, 1ull)] = (i32)l;
}

int cond_norm(const ScaleResult &X, const ScaleResult &Y, i64 n, double *out_mean, cudaStream_t st) {
    const i64 CX = X.n_comms, CY = Y.n_comms;
    i32 *ycnt = nullptr, *cursor = nullptr, *mlist = nullptr, *tkey = nullptr, *tcnt = nullptr, *big = nullptr;
    i64 *mptr = nullptr, *tsz = nullptr, *toff = nullptr, *tmp = nullptr;
    double *term = nullptr, *sum = nullptr;
    unsigned long long *nbig = nullptr;
    int rc = MSCD_OK;
    const unsigned gb = 152 * 16;
    do {
        if ((rc = cuda_status(cudaMallocAsync((void **)&ycnt, n * sizeof(i32), st)))) break;
        if ((rc = cuda_status(cudaMallocAsync((void **)&cursor, n * sizeof(i32), st)))) break;
        if ((rc = cuda_status(cudaMallocAsync((void **)&mptr, (n + 1) * sizeof(i64), st)))) break;
        if ((rc = cuda_status(cudaMallocAsync((void **)&tmp, (n + 1) * sizeof(i64), st)))) break;
        if ((rc = cuda_status(cudaMemsetAsync(ycnt, 0, n * sizeof(i32), st)))) break;
        if ((rc = cuda_status(cudaMemsetAsync(cursor, 0, n * sizeof(i32), st)))) break;
        count_memberships<<<gb, 256, 0, st>>>(Y.comm_nodes, Y.n_nodes, ycnt);
        widen_i32<<<gb, 256, 0, st>>>(ycnt, n, tmp);
        if ((rc = scan_exclusive_i64(tmp, mptr, n, mptr + n, st))) break;
        if ((rc = cuda_status(cudaMallocAsync((void **)&mlist, std::max<i64>(Y.n_nodes, 1) * sizeof(i32), st)))) break;
        fill_memberships<<<gb, 256, 0, st>>>(Y.comm_ptr, Y.comm_nodes, CY, mptr, cursor, mlist);
        if ((rc = cuda_status(cudaMallocAsync((void **)&tsz, (CX + 1) * sizeof(i64), st)))) break;
        if ((rc = cuda_status(cudaMallocAsync((void **)&toff, (CX + 1) * sizeof(i64), st)))) break;
        table_sizes<<<gb, 256, 0, st>>>(X.comm_ptr, X.comm_nodes, CX, ycnt, CY, tsz);
        if ((rc = scan_exclusive_i64(tsz, toff, CX, toff + CX, st))) break;
        i64 TT = 0;
        if ((rc = cuda_status(cudaMemcpyAsync(&TT, toff + CX, sizeof(i64), cudaMemcpyDeviceToHost, st)))) break;
        if ((rc = cuda_status(cudaStreamSynchronize(st)))) break;
        if ((rc = cuda_status(cudaMallocAsync((void **)&tkey, std::max<i64>(TT, 1) * sizeof(i32), st)))) break;
        if ((rc = cuda_status(cudaMallocAsync((void **)&tcnt, std::max<i64>(TT, 1) * sizeof(i32), st)))) break;
        if ((rc = cuda_status(cudaMemsetAsync(tkey, 0xff, TT * sizeof(i32), st)))) break;
        if ((rc = cuda_status(cudaMemsetAsync(tcnt, 0, TT * sizeof(i32), st)))) break;
        if ((rc = cuda_status(cudaMallocAsync((void **)&big, std::max<i64>(CY, 1) * sizeof(i32), st)))) break;
        if ((rc = cuda_status(cudaMallocAsync((void **)&nbig, sizeof(unsigned long long), st)))) break;
        if ((rc = cuda_status(cudaMemsetAsync(nbig, 0, sizeof(unsigned long long), st)))) break;
        list_big<<<gb, 256, 0, st>>>(Y.comm_ptr, CY, n, big, nbig);
        unsigned long long h_nbig = 0;
        if ((rc = cuda_status(cudaMemcpyAsync(&h_nbig, nbig, sizeof(h_nbig), cudaMemcpyDeviceToHost, st)))) break;
        if ((rc = cuda_status(cudaMallocAsync((void **)&term, std::max<i64>(CX, 1) * sizeof(double), st)))) break;
        if ((rc = cuda_status(cudaMallocAsync((void **)&sum, sizeof(double), st)))) break;
        if ((rc = cuda_status(cudaStreamSynchronize(st)))) break;
        cond_entropy<<<gb, 256, 0, st>>>(X.comm_ptr, X.comm_nodes, CX, Y.comm_ptr, CY, mptr, mlist, toff, tkey, tcnt,
                                         big, (i64)h_nbig, n, term);
        sum_fixed<<<1, 1024, 0, st>>>(term, CX, sum);
        double h_sum = 0.0;
        if ((rc = cuda_status(cudaMemcpyAsync(&h_sum, sum, sizeof(double), cudaMemcpyDeviceToHost, st)))) break;
        if ((rc = cuda_status(cudaStreamSynchronize(st)))) break;
        *out_mean = h_sum / (double)CX;
    } while (0);
    cudaFreeAsync(ycnt, st);
    cudaFreeAsync(cursor, st);
    cudaFreeAsync(mptr, st);
    cudaFreeAsync(tmp, st);
    cudaFreeAsync(mlist, st);
    cudaFreeAsync(tsz, st);
    cudaFreeAsync(toff, st);
    cudaFreeAsync(tkey, st);
    cudaFreeAsync(tcnt, st);
    cudaFreeAsync(big, st);
    cudaFreeAsync(nbig, st);
    cudaFreeAsync(term, st);
    cudaFreeAsync(sum, st);
    return rc;
}

}  // namespace

int nmi_between(const ScaleResult &X, const ScaleResult &Y, i64 n, double *nmi, cudaStream_t st) {
    if (X.n_comms <= 0 || Y.n_comms <= 0 || n <= 0) {
        *nmi = __builtin_nan("");
        return MSCD_OK;
    }
    double hxy = 0.0, hyx = 0.0;
    int rc = cond_norm(X, Y, n, &hxy, st);
    if (rc == MSCD_OK) rc = cond_norm(Y, X, n, &hyx, st);
    if (rc != MSCD_OK) return rc;
    *nmi = 1.0 - 0.5 * (hxy + hyx);
    return MSCD_OK;
}
