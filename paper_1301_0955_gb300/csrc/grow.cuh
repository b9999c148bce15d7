// Launch interface of the growth kernel.
#pragma once

#include "common.cuh"

#define GROW_MAX_THREADS 512
#define GLOBAL_CTA_THREADS 256  // threads per CTA of the global-arena classes

struct GrowArgs {
    DevGraph G;
    const double *alphas;   // [n_scales]
    const i32 *seeds;       // [n_seeds] or null = node ids 0..n_seeds-1
    i64 n_seeds;
    // per-unit scales (serving batches mix queries): unit u grows from
    // seeds[u] at unit_alpha[u]; null = unit u is (scale u / n_seeds, seed u % n_seeds)
    const double *unit_alpha;
    // optional initial members per seed index (init_ptr[si]..init_ptr[si+1])
    const i64 *init_ptr;
    const i32 *init_nodes;
    int single_round;       // one grow call of Alg. 1 (the full method repeats it itself)
    // work: units 0..n_work-1, or the listed units
    const i64 *work_list;
    i64 n_work;
    unsigned long long *work_counter;
    // plain (non-persistent) form: warp w of the grid takes work item
    // work_base + w, and unit unit_base + item when there is no list
    int plain;
    i64 work_base, unit_base;
    // per-warp node-slot state
    int cap;                // node slots per unit (power of 2, >= 32)
    int use_smem;           // 1: dynamic shared memory, 0: global arena
    int bounds_smem;        // global arena with the group bounds in dynamic shared memory
    int hash_smem;          // ... and the hash table too (after the bounds)
    size_t smem_per_warp;   // dynamic shared memory of one warp in a global-arena class
    unsigned char *big_seed;  // per seed: outgrew this class at a finer scale (first class only; may be null)
    unsigned char *gstate;  // global arena (warps * state_bytes)
    size_t state_bytes;     // per warp
    i64 max_rounds;
    float log_kmax;         // log of the largest degree (bounds the binary32 key error)
    // outputs (unit-indexed)
    i32 *out_nodes;
    unsigned long long *out_cursor;
    unsigned long long *out_needed;
    i64 out_cap;
    i64 *uoff;
    i32 *ulen;
    u64 *uhash;
    u64 hash_clear;         // bits cleared in every list hash (0; set only by tests of the collision path)
    double *uf;
    i64 *ustat;
    i32 *ustatus;
    // units to grow again: slot capacity exceeded / output buffer full
    i64 *retry_state;
    unsigned long long *n_retry_state;
    i64 *retry_out;
    unsigned long long *n_retry_out;
    u32 *error_flags;
};

// Bytes of one unit's state at `cap` node slots on graph G.
size_t grow_state_bytes(const DevGraph &G, int cap);
// One unit per warp; `threads` = 32 * warps per CTA.
int grow_launch(const GrowArgs &a, int blocks, int threads, size_t smem, cudaStream_t st);
int grow_occupancy(const GrowArgs &a, int threads, size_t smem, int *blocks_per_sm);
