// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <vector>
#include <stdint.h>

#include "mscd.h"

typedef int64_t i64;
typedef uint64_t u64;
typedef int32_t i32;
typedef uint32_t u32;

#define FULL_MASK 0xffffffffu

// Resident graph on the device (all arrays owned by the context).
struct DevGraph {
    i64 n = 0, nnz = 0;
    const i64 *rp = nullptr;     // int64[n+1]
    const i32 *col = nullptr;    // int32[nnz]
    const i64 *wfx = nullptr;    // int64[nnz] exact fixed-point weights, null = unweighted
    const i64 *k = nullptr;      // int64[n] weighted degree (weight units)
    const float *logk = nullptr;   // float[n] logf(k) (0 where k = 0), for the binary32 priority keys
    i64 kmax = 0;                  // largest k_u
    int unit_exp = 0;            // weight unit 2^unit_exp
    i64 volume = 0;              // sum of k
};

static inline int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return MSCD_OK;
    if (e == cudaErrorMemoryAllocation) return MSCD_ENOMEM;
    return MSCD_EDEVICE;
}

#define MSCD_CUDA(x)                               \
    do {                                           \
        cudaError_t _e = (x);                      \
        if (_e != cudaSuccess) return cuda_status(_e); \
    } while (0)

// Count one kernel launch of this library (process-wide, see mscd_launch_count).
void note_launch();

// Device-side exclusive scan of int64 (in place allowed); returns the total
// through *total_dev (device pointer, may be null).  Work buffer handled inside.
int scan_exclusive_i64(const i64 *in, i64 *out, i64 n, i64 *total_dev, cudaStream_t st);

// A context's resident graph and device (false for an unknown id).
struct mscd_ctx;
bool ctx_graph(mscd_ctx *c, int32_t graph_id, DevGraph *g, int *device);

// Graph preparation (checks, exact weights, degrees, log degrees).
int graph_prepare(i64 n, const i64 *rp_dev, const i32 *col_dev, const float *w_dev, DevGraph *g, i64 **wfx_out,
                  i64 **k_out, float **logk_out, cudaStream_t st);

// Disjoint union of graphs as one graph (node ids of part p shifted by the
// nodes of the parts before it); node_off gets the n_parts+1 offsets.  All parts
// weighted or none; MSCD_ERANGE when the total exceeds the ranges of a load.
int graph_union(const std::vector<DevGraph> &parts, DevGraph *out, i64 **rp_out, i32 **col_out, i64 **wfx_out,
                i64 **k_out, float **logk_out, std::vector<i64> *node_off, cudaStream_t st);
