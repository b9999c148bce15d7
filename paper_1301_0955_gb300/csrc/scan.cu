// Exclusive prefix sum of int64 on the device (tiles of 1024, block sums
// scanned recursively, then added back).  Used for output offsets.
#include "common.cuh"

namespace {
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__global__ void __launch_bounds__(SCAN_THREADS) scan_tiles(const i64 *in, i64 *out, i64 n, i64 *tile_sums) {
    __shared__ i64 warp_tot[SCAN_THREADS / 32];
    const i64 base = (i64)blockIdx.x * SCAN_TILE + (i64)threadIdx.x * SCAN_ITEMS;
    i64 v[SCAN_ITEMS];
    i64 tsum = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        v[j] = (base + j < n) ? in[base + j] : 0;
        tsum += v[j];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    i64 x = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        i64 y = __shfl_up_sync(FULL_MASK, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        i64 t = lane < SCAN_THREADS / 32 ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            i64 y = __shfl_up_sync(FULL_MASK, t, o);
            if (lane >= o) t += y;
        }
        if (lane < SCAN_THREADS / 32) warp_tot[lane] = t;
    }
    __syncthreads();
    i64 excl = x - tsum + (w > 0 ? warp_tot[w - 1] : 0);
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        if (base + j < n) out[base + j] = excl;
        excl += v[j];
    }
    if (threadIdx.x == SCAN_THREADS - 1) tile_sums[blockIdx.x] = excl;
}

__global__ void __launch_bounds__(SCAN_THREADS) add_tile_offsets(i64 *out, i64 n, const i64 *offs) {
    const i64 base = (i64)blockIdx.x * SCAN_TILE + (i64)threadIdx.x * SCAN_ITEMS;
    const i64 o = offs[blockIdx.x];
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j)
        if (base + j < n) out[base + j] += o;
}
}  // namespace

int scan_exclusive_i64(const i64 *in, i64 *out, i64 n, i64 *total_dev, cudaStream_t st) {
    if (n <= 0) {
        if (total_dev) MSCD_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(i64), st));
        return MSCD_OK;
    }
    const i64 nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    i64 *sums = nullptr;
    MSCD_CUDA(cudaMallocAsync((void **)&sums, (size_t)nb * sizeof(i64), st));
    scan_tiles<<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, out, n, sums); note_launch();
    int rc = MSCD_OK;
    if (nb > 1) {
        rc = scan_exclusive_i64(sums, sums, nb, total_dev, st);
        if (rc == MSCD_OK) { add_tile_offsets<<<(unsigned)nb, SCAN_THREADS, 0, st>>>(out, n, sums); note_launch(); }
    } else if (total_dev) {
        cudaMemcpyAsync(total_dev, sums, sizeof(i64), cudaMemcpyDeviceToDevice, st);
    }
    cudaFreeAsync(sums, st);
    if (rc != MSCD_OK) return rc;
    return cuda_status(cudaGetLastError());
}
