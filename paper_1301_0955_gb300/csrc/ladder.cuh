// One growth pipeline: the node-slot class ladder and the buffers it reuses.
//
// Units start in the first (shared-memory) class; a unit that touches more
// nodes than its class holds stops and is grown again from scratch in the
// next class; a unit whose list finds the output buffer full is grown again
// once the buffer has been enlarged.  A context's runs use one pipeline; each
// serving worker owns another (its own stream and buffers).
#pragma once
#include <vector>

#include "common.cuh"
#include "grow.cuh"

struct Counters {
    unsigned long long work, out_cursor, out_needed, n_retry_state, n_retry_out;
    u32 error_flags;
    u32 pad;
};

struct GrowPipe {
    int sm_count = 1;
    mscd_params p{};
    cudaStream_t st = nullptr;
    Counters *ctr = nullptr;
    i64 *retry_a = nullptr, *retry_b = nullptr;  // units to grow again (class / output)
    i64 retry_cap = 0;
    unsigned char *arena = nullptr;               // global-arena class states
    size_t arena_bytes = 0;
    i32 *out_nodes = nullptr;                     // member lists
    i64 out_cap = 0;
    mscd_run_stats *stats = nullptr;              // launch records (may be null)
};

// Counters and retry lists for up to `units` units per call.
int pipe_reserve(GrowPipe &w, i64 units);
// Output buffer of at least `need` entries keeping the first `keep`.
int pipe_output(GrowPipe &w, i64 need, i64 keep);
void pipe_free(GrowPipe &w);
// Drop the output buffer (it is allocated again on the next use).
void pipe_release_output(GrowPipe &w);

// The ladder of node-slot capacities for a graph whose parts hold at most
// max_part_n nodes: shared-memory classes, then global arenas growing 8x up to
// the first power of two above max_part_n (a class that never overflows).
int make_ladder(const DevGraph &G, i64 max_part_n, const mscd_params &p, std::vector<int> *ladder,
                std::vector<bool> *in_smem);

// Grow n_units units through the ladder.  `proto` carries the graph, the scale
// and seed mapping (alphas/seeds/n_seeds/unit_base, or unit_alpha with seeds
// per unit), the per-unit outputs, max_rounds, log_kmax and big_seed; lists are
// written from output entry 0 and *cursor_out gets the entries used.  `plain`:
// one statically mapped unit per warp (no persistence).  out_budget: entries
// the output may take before units wait for a larger buffer.
int grow_units(GrowPipe &w, const GrowArgs &proto, i64 n_units, const std::vector<int> &ladder,
               const std::vector<bool> &in_smem, bool plain, i64 out_budget, i64 max_part_n,
               unsigned long long *cursor_out);
