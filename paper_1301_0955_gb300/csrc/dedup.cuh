// Per-scale deduplicated communities and the stability measure between scales.
#pragma once

#include "common.cuh"

struct ScaleResult {
    i64 n_comms = 0, n_nodes = 0;
    i64 *comm_ptr = nullptr;   // [n_comms+1]
    i32 *comm_nodes = nullptr; // [n_nodes]
    double *comm_f = nullptr;  // [n_comms]
    i32 *seed2comm = nullptr;  // [n_seeds]
    u64 *comm_hash = nullptr;  // [n_comms] hash of the member list
};

void scale_result_free(ScaleResult *r);

// Units of one scale: uoff/ulen/uhash/uf indexed 0..N-1 (seed order), lists in nodes.
int dedup_scale(const i64 *uoff, const i32 *ulen, const u64 *uhash, const double *uf, const i32 *nodes, i64 N,
                ScaleResult *out, cudaStream_t st);

// Overlapping NMI between two deduplicated community sets over n nodes.
// nmi[p] for each part p of a graph that is a disjoint union (part_off:
// device int64[n_parts+1] node offsets), or nmi[0] for the whole graph of n
// nodes when part_off is null.  NaN where a side has no community.
int nmi_between(const ScaleResult &X, const ScaleResult &Y, i64 n, const i64 *part_off, int32_t n_parts, double *nmi,
                cudaStream_t st);
