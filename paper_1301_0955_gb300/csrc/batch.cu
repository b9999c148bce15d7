// Many independent graphs as one: the disjoint union of loaded graphs.
//
// Units on different parts never interact (a community grows only inside the
// component of its seed, and every decision depends only on K, V, d and k of
// that community), so all seeds of all parts run in the same persistent
// launches, the per-scale dedup of the union is the concatenation of the
// parts' dedups, and the stability is measured per part (the NMI takes n as
// its part's node count).  Node ids of part p are shifted by its node offset.
//
// Weighted parts are brought to the smallest weight unit 2^e of all parts
// (exact left shifts of the fixed-point values); the decisions are invariant
// under a common scale factor of a part's weights (both sides of every test
// scale by the same power), and the reported fitness is converted back to
// real weight units, so results per part are unchanged.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace {

__global__ void rows_with_offset(const i64 *src, i64 m, i64 add, i64 *dst) {
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (i64)gridDim.x * blockDim.x)
        dst[i] = src[i] + add;
}

__global__ void cols_with_offset(const i32 *src, i64 m, i32 add, i32 *dst) {
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (i64)gridDim.x * blockDim.x)
        dst[i] = src[i] + add;
}

__global__ void shift_left(const i64 *src, i64 m, int s, i64 *dst) {
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (i64)gridDim.x * blockDim.x)
        dst[i] = src[i] << s;
}

// Same expression as the degree kernel of graph preparation.
__global__ void log_degrees(const i64 *k, i64 m, float *logk) {
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (i64)gridDim.x * blockDim.x)
        logk[i] = k[i] ? logf((float)k[i]) : 0.0f;
}

unsigned grid_for(i64 m) { return (unsigned)std::max<i64>(1, std::min<i64>((m + 255) / 256, 152 * 8)); }

}  // namespace

int graph_union(const std::vector<DevGraph> &parts, DevGraph *out, i64 **rp_out, i32 **col_out, i64 **wfx_out,
                i64 **k_out, float **logk_out, std::vector<i64> *node_off, cudaStream_t st) {
    *rp_out = nullptr;
    *col_out = nullptr;
    *wfx_out = nullptr;
    *k_out = nullptr;
    *logk_out = nullptr;
    if (parts.empty()) return MSCD_EINVAL;
    const bool weighted = parts[0].wfx != nullptr;
    i64 n = 0, nnz = 0, kmax = 0;
    int ue = parts[0].unit_exp;
    for (const DevGraph &g : parts) {
        if ((g.wfx != nullptr) != weighted) return MSCD_EINVAL;
        n += g.n;
        nnz += g.nnz;
        ue = std::min(ue, g.unit_exp);
    }
    if (n >= (i64)INT32_MAX) return MSCD_ERANGE;
    // exact volume and largest degree after the shifts; the same 2^62 bound as a load
    long double vol = 0.0L;
    for (const DevGraph &g : parts) {
        const int s = weighted ? g.unit_exp - ue : 0;
        if (s > 62) return MSCD_ERANGE;
        vol += std::ldexp((long double)g.volume, s);
        kmax = std::max<i64>(kmax, g.kmax == 0 ? 0 : (i64)std::min<long double>(std::ldexp((long double)g.kmax, s),
                                                                              (long double)INT64_MAX));
    }
    if (vol >= std::ldexp(1.0L, 62)) return MSCD_ERANGE;
    int rc = MSCD_OK;
    do {
        if ((rc = cuda_status(cudaMalloc((void **)rp_out, (size_t)(n + 1) * sizeof(i64))))) break;
        if ((rc = cuda_status(cudaMalloc((void **)col_out, (size_t)std::max<i64>(nnz, 1) * sizeof(i32))))) break;
        if ((rc = cuda_status(cudaMalloc((void **)k_out, (size_t)std::max<i64>(n, 1) * sizeof(i64))))) break;
        if ((rc = cuda_status(cudaMalloc((void **)logk_out, (size_t)std::max<i64>(n, 1) * sizeof(float))))) break;
        if (weighted &&
            (rc = cuda_status(cudaMalloc((void **)wfx_out, (size_t)std::max<i64>(nnz, 1) * sizeof(i64)))))
            break;
        node_off->assign(1, 0);
        i64 no = 0, eo = 0;
        for (const DevGraph &g : parts) {
            const int s = weighted ? g.unit_exp - ue : 0;
            if (g.n > 0) {
                rows_with_offset<<<grid_for(g.n), 256, 0, st>>>(g.rp, g.n, eo, *rp_out + no); note_launch();
            }
            if (g.nnz > 0) {
                cols_with_offset<<<grid_for(g.nnz), 256, 0, st>>>(g.col, g.nnz, (i32)no, *col_out + eo); note_launch();
                if (weighted) {
                    shift_left<<<grid_for(g.nnz), 256, 0, st>>>(g.wfx, g.nnz, s, *wfx_out + eo); note_launch();
                }
            }
            if (g.n > 0) {
                if (s == 0) {
                    if ((rc = cuda_status(cudaMemcpyAsync(*k_out + no, g.k, g.n * sizeof(i64),
                                                          cudaMemcpyDeviceToDevice, st))))
                        break;
                    if ((rc = cuda_status(cudaMemcpyAsync(*logk_out + no, g.logk, g.n * sizeof(float),
                                                          cudaMemcpyDeviceToDevice, st))))
                        break;
                } else {
                    shift_left<<<grid_for(g.n), 256, 0, st>>>(g.k, g.n, s, *k_out + no); note_launch();
                    log_degrees<<<grid_for(g.n), 256, 0, st>>>(*k_out + no, g.n, *logk_out + no); note_launch();
                }
            }
            no += g.n;
            eo += g.nnz;
            node_off->push_back(no);
        }
        if (rc) break;
        if ((rc = cuda_status(cudaMemcpyAsync(*rp_out + n, &nnz, sizeof(i64), cudaMemcpyHostToDevice, st)))) break;
        if ((rc = cuda_status(cudaStreamSynchronize(st)))) break;
        if ((rc = cuda_status(cudaGetLastError()))) break;
        out->n = n;
        out->nnz = nnz;
        out->rp = *rp_out;
        out->col = *col_out;
        out->wfx = *wfx_out;
        out->k = *k_out;
        out->logk = *logk_out;
        out->kmax = kmax;
        out->unit_exp = weighted ? ue : 0;
        out->volume = (i64)vol;
    } while (0);
    if (rc) {
        cudaStreamSynchronize(st);
        cudaFree(*rp_out);
        cudaFree(*col_out);
        cudaFree(*wfx_out);
        cudaFree(*k_out);
        cudaFree(*logk_out);
        *rp_out = nullptr;
        *col_out = nullptr;
        *wfx_out = nullptr;
        *k_out = nullptr;
        *logk_out = nullptr;
    }
    return rc;
}
