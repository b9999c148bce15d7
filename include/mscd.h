/*
 * mscd.h — C ABI of the GB300 multi-scale local-criterion community growth
 * library (libmscd.so).
 *
 * The method is that of Le Martelot & Hankin, "Fast Multi-Scale Community
 * Detection based on Local Criteria within a Multi-Threaded Algorithm":
 * for every scale alpha and every seed node, a community grows from {seed}
 * by the greedy rule of Algorithm 1 (max priority queue ranked by
 * 2 d_in / (d_in + d_out)^alpha, add a node iff it raises the LFK fitness
 * f_c = k_in / (k_in + k_out)^alpha of Eq. 1, Eq. 2 as a strict test, then
 * prune members whose removal raises f), repeated while a grow pass adds
 * something ("while changes can be made", Algorithm 2).  Identical
 * communities found from different seeds are deduplicated per scale, and
 * successive scales are compared with the overlapping NMI cited in Sec. 4,
 * averaged over windows of 3 and 5 scales.
 *
 * Conventions shared by every entry point:
 *   - Every function returns an int status: MSCD_OK (0) or a negative code
 *     below; mscd_strerror() gives its text.  Nothing is fixed silently.
 *   - Array arguments are host pointers unless a function takes `flags` and
 *     MSCD_DEVICE_PTRS is set, in which case they are device pointers on the
 *     context's device.  Input arrays are copied before the call returns; the
 *     caller keeps ownership of everything it passes.
 *   - Outputs go to caller-owned buffers.  A buffer that is too small gives
 *     MSCD_ESMALL with the required length written back; cap = 0 queries it.
 *   - A context is not thread-safe: calls on one context must not overlap.
 *   - Exact decisions: every add / remove / priority decision is the exact
 *     sign of log(a1/a2) - alpha*log(b1/b2) over integer operands (weights
 *     are converted exactly to int64 multiples of the largest power of two
 *     dividing all of them), so memberships are independent of thread, warp
 *     and launch order.
 */
#ifndef MSCD_H
#define MSCD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define MSCD_OK 0
#define MSCD_EINVAL (-1)      /* bad argument or malformed CSR structure          */
#define MSCD_ENOTSYM (-2)     /* CSR not symmetric, or unequal weights u->v, v->u */
#define MSCD_ESELFLOOP (-3)   /* an entry u -> u                                  */
#define MSCD_EDUP (-4)        /* a repeated entry inside one row                  */
#define MSCD_ERANGE (-5)      /* exact fixed-point weights need more than 62 bits */
#define MSCD_ENOMEM (-6)      /* device allocation failed                         */
#define MSCD_EDEVICE (-7)     /* CUDA error (device, launch or copy)              */
#define MSCD_ETIMEOUT (-8)    /* a unit hit the grow/prune repetition cap         */
#define MSCD_ESMALL (-9)      /* output buffer too small; length written back     */
#define MSCD_EUNDECIDED (-10) /* a decision no certified stage could settle       */
#define MSCD_EUNSORTED (-11)  /* a CSR row is not in ascending column order       */
#define MSCD_EWEIGHT (-12)    /* a weight that is not finite and > 0              */
#define MSCD_ENORESULT (-13)  /* no successful run to read results from           */
#define MSCD_EBUSY (-14)      /* in use: a graph queries still need, or a server
                                 already running                                 */

/* ---- flags ------------------------------------------------------------- */
#define MSCD_DEVICE_PTRS 1u   /* array arguments are device pointers             */

/* Per-unit statistics (int64 each, in this order): CSR entries scanned
 * (seed row + rows of every added and removed node), nodes added, nodes
 * removed, grow/prune rounds, final K (internal degree sum, weight units),
 * final V (volume, weight units), decisions taken by a slow stage, undecided
 * flag. */
#define MSCD_STAT_EDGES 0
#define MSCD_STAT_ADDS 1
#define MSCD_STAT_REMOVES 2
#define MSCD_STAT_ROUNDS 3
#define MSCD_STAT_K 4
#define MSCD_STAT_V 5
#define MSCD_STAT_SLOW 6
#define MSCD_STAT_UNDECIDED 7
#define MSCD_NSTATS 8

typedef struct mscd_ctx mscd_ctx;

/* Tuning and limits.  Zero fields take the defaults. */
typedef struct mscd_params {
    int32_t struct_size;     /* sizeof(mscd_params)                                     */
    int32_t warps_per_block; /* reserved (0)                                             */
    int32_t smem_slots;      /* node slots of the first shared-memory class (power of 2
                                >= 32; 0 = 1024, or 512 when weighted slots do not fit) */
    int32_t blocks_per_sm;   /* first class: CTAs per SM (0 = from occupancy)           */
    int32_t mid_slots;       /* node slots of an optional second shared-memory class
                                (power of 2 >= 32; 0 = none)                            */
    int32_t global_warps_per_sm; /* global-arena classes: resident units per SM (16)     */
    int32_t global_slots;    /* node slots of the first global-arena class (power of 2;
                                0 = 8 times the last shared-memory class)                */
    int64_t max_rounds;      /* grow/prune repetitions per unit before ETIMEOUT (1e6)     */
    int32_t schedule;        /* MSCD_SCHED_PERSISTENT (0): every scale's units in one
                                persistent launch per slot class, warps taking units from a
                                global counter.  MSCD_SCHED_PER_SCALE (1): the plain form,
                                one launch per scale and slot class, one unit per warp,
                                statically mapped (no persistence, no work stealing); the
                                results are identical, only the speed differs           */
    int32_t hash_smem_slots; /* global-arena classes of at most this many slots keep
                                their hash table (and group bounds) in shared memory,
                                the slot arrays in the arena (0 = none)               */
    int32_t list_hash_bits;  /* testing only: keep this many low bits (1..63) of each
                                member list's 64-bit hash, so that different lists
                                share hashes and dedup's exact comparison and
                                regrouping run on every scale (0 = all 64 bits; the
                                results are the same either way)                       */
} mscd_params;

#define MSCD_SCHED_PERSISTENT 0
#define MSCD_SCHED_PER_SCALE 1

/* mscd_autotune flags */
#define MSCD_TUNE_APPLY 1u   /* make the result the context's parameters          */
#define MSCD_TUNE_CACHED 2u  /* reuse a result for the same graph shape if present */

/* Totals of the last run. */
typedef struct mscd_run_stats {
    int64_t units;            /* (scale, seed) units grown                         */
    int64_t edges_scanned;    /* sum of MSCD_STAT_EDGES                            */
    int64_t adds, removes;    /* sums over units                                   */
    int64_t slow_decisions;   /* decisions settled by the tie test or double-double */
    int64_t undecided;        /* units with an undecided decision (expected 0)     */
    int64_t overflow_units;   /* units re-grown in a larger node-slot class        */
    int64_t grow_launches;    /* growth kernel launches                            */
    int64_t member_entries;   /* total member-list length over all units           */
    double ms_grow, ms_dedup, ms_stability, ms_total; /* device time per stage    */
    /* the first 8 growth launches: node slots per unit, shared memory (1) or
     * global arena (0), units, ms */
    int32_t launch_cap[8], launch_smem[8];
    int64_t launch_units[8];
    double launch_ms[8];
} mscd_run_stats;

/* Text of a status code (static storage). */
const char *mscd_strerror(int status);

/* Library version, major*10000 + minor*100 + patch.  0.2.0 (200) added
 * mscd_params.list_hash_bits, the last two fields of mscd_serve_stats and
 * mscd_serve_batch_intervals; structs of 0.1.x have other sizes. */
int mscd_version(void);

/* Number of kernels this library has launched in the calling process so far
 * (all contexts); the difference around a call counts its launches. */
int64_t mscd_launch_count(void);

/* Create a context on CUDA device `device`.  params may be NULL.  Errors:
 * EINVAL (bad device or params), EDEVICE, ENOMEM. */
int mscd_create(mscd_ctx **out, int device, const mscd_params *params);

/* Free a context and every graph and result it holds. */
int mscd_destroy(mscd_ctx *ctx);

/* Load an undirected graph in CSR form (the paper's input network, Alg. 2).
 *   n        number of nodes (0 <= n < 2^31)
 *   row_ptr  int64[n+1], row_ptr[0] = 0, non-decreasing
 *   col      int32[row_ptr[n]], each row strictly ascending, no u -> u
 *   w        float32[row_ptr[n]] edge weights (finite, > 0), or NULL for an
 *            unweighted graph (every weight 1)
 * The CSR must be symmetric with equal weights in both directions.  Checks
 * run on the device in a fixed category order and the first failing
 * category is returned: EINVAL (structure), EWEIGHT, ESELFLOOP, EUNSORTED,
 * EDUP, ENOTSYM, ERANGE.  On success *graph_id names the resident graph
 * (arrays copied to device memory; degrees and exact weights precomputed). */
int mscd_graph_load_csr(mscd_ctx *ctx, int64_t n, const int64_t *row_ptr, const int32_t *col,
                        const float *w, uint32_t flags, int32_t *graph_id);

/* Release a resident graph.  EINVAL for an unknown id. */
int mscd_graph_free(mscd_ctx *ctx, int32_t graph_id);

/* Batching of independent graphs.  Every community grows on its own from its
 * seed (Alg. 1), so many graphs form one problem: the disjoint union of the
 * resident graphs graph_ids[0..n_parts) becomes a new resident graph whose
 * node ids are those of part p shifted by the node counts of the parts before
 * it (offsets from mscd_graph_parts).  A run on it grows every seed of every
 * part in the same launches; the deduplicated communities of a scale are the
 * parts' communities one after another; the stability is per part
 * (mscd_get_stability_part: the NMI of Sec. 4 with n = the part's node count).
 * Results per part equal those of the part run alone.  The parts stay resident
 * and owned by the caller (the union holds copies).  EINVAL: an unknown id, a
 * part that is itself a union, weighted and unweighted parts mixed; ERANGE:
 * 2^31 - 1 nodes or more, or a total volume of 2^62 weight units or more once
 * weighted parts share the smallest weight unit. */
int mscd_graph_union(mscd_ctx *ctx, const int32_t *graph_ids, int32_t n_parts, int32_t *union_id);

/* Part node offsets of a resident graph: node_offset int64[n_parts+1] (cap
 * entries); a graph loaded from one CSR is one part {0, n}.  ESMALL with
 * *n_parts set when cap < n_parts + 1. */
int mscd_graph_parts(mscd_ctx *ctx, int32_t graph_id, int64_t *node_offset, int32_t cap, int32_t *n_parts);

/* Facts of a resident graph: node and entry counts, the weight unit 2^unit_exp
 * of the exact fixed-point weights, total volume in weight units. */
int mscd_graph_info(mscd_ctx *ctx, int32_t graph_id, int64_t *n, int64_t *nnz, int32_t *unit_exp,
                    int64_t *volume);

/* Weighted degrees k_u in weight units, host int64[n]. */
int mscd_graph_degrees(mscd_ctx *ctx, int32_t graph_id, int64_t *k);

/* The logarithmic scale list of Sec. 4, read as
 *   alpha_k = vmin + (a - vmin) (1 - log k / log x),  k = 1..x,
 * i.e. a first (finest scale, smallest communities) down to vmin (coarsest);
 * x = 1 gives {a}.  out: host double[x].  EINVAL unless x >= 1, 0 < vmin <= a. */
int mscd_scales_logspaced(double vmin, double a, int32_t x, double *out);

/* Grow one community per (scale, seed) unit, deduplicate per scale and compare
 * successive scales (Alg. 1 per unit, Sec. 4 for the stability measure).
 *   alphas   double[n_scales], each finite and > 0 (ordered as the caller wants
 *            successive scales compared; Sec. 4 lists them fine to coarse)
 *   seeds    int32[n_seeds] node ids, or NULL for every node (n_seeds ignored)
 *   flags    MSCD_DEVICE_PTRS: alphas and seeds are device pointers
 *   cuda_stream  cudaStream_t to order the work on, or NULL for the context's
 * Synchronous: returns when results are ready.  Unit index = scale * n_seeds +
 * seed index.  Errors: EINVAL, ENOMEM, EDEVICE; ETIMEOUT or EUNDECIDED when a
 * unit hit the round cap or an undecided comparison (results still readable,
 * the unit's statistics say which). */
int mscd_run(mscd_ctx *ctx, int32_t graph_id, const double *alphas, int32_t n_scales, const int32_t *seeds,
             int64_t n_seeds, uint32_t flags, void *cuda_stream);

/* The same, each community starting from its seed plus given initial members
 * (Alg. 2: "a set of initial communities is given in input"): init_ptr
 * int64[n_seeds+1] (init_ptr[0] = 0, non-decreasing) and init_nodes
 * int32[init_ptr[n_seeds]] list the members for seed i at
 * init_ptr[i]..init_ptr[i+1] (any order; repeats and the seed are ignored).
 * The members join before the first grow pass (not counted as additions);
 * the seed stays pinned; a community that no addition improves is returned
 * as given (prune passes follow additions only, Alg. 1).  seeds must not be
 * NULL.  Host or device pointers as flags say. */
int mscd_run_init(mscd_ctx *ctx, int32_t graph_id, const double *alphas, int32_t n_scales, const int32_t *seeds,
                  int64_t n_seeds, const int64_t *init_ptr, const int32_t *init_nodes, uint32_t flags,
                  void *cuda_stream);

/* Membership of one unit: the sorted member list (host int32, cap entries),
 * its length and its fitness f (Eq. 1 in the original weight units). */
int mscd_get_membership(mscd_ctx *ctx, int32_t scale_idx, int64_t seed_idx, int32_t *buf, int64_t cap,
                        int64_t *len, double *fitness);

/* All memberships of one scale, concatenated in seed order: ptr int64[n_seeds+1],
 * nodes int32[nodes_cap], fitness double[n_seeds] (may be NULL), stats
 * int64[n_seeds * MSCD_NSTATS] (may be NULL).  *n_nodes gets the total length. */
int mscd_get_memberships(mscd_ctx *ctx, int32_t scale_idx, int64_t *ptr, int32_t *nodes, int64_t nodes_cap,
                         double *fitness, int64_t *stats, int64_t *n_nodes);

/* Deduplicated communities of one scale, numbered in order of their smallest
 * generating seed index: ptr int64[n_comms+1] (ptr_cap entries), nodes
 * int32[nodes_cap], fitness double[n_comms] (may be NULL), seed2comm
 * int32[n_seeds] (may be NULL).  *n_comms and *n_nodes get the sizes. */
int mscd_get_communities(mscd_ctx *ctx, int32_t scale_idx, int64_t *ptr, int64_t ptr_cap, int32_t *nodes,
                         int64_t nodes_cap, double *fitness, int32_t *seed2comm, int64_t *n_comms,
                         int64_t *n_nodes);

/* Autotuner (no counterpart in the paper, whose growth runs one community
 * per CPU thread).  Times the growth alone on n_sample evenly spaced seeds of
 * graph_id (0 = min(n, 20000)) at the given scales under candidate schedules
 * and keeps the fastest: the node-slot capacity of the shared-memory class
 * (256..2048), of the first global-arena class (4096..16384, or 8 times the
 * first), and the resident units per SM of the global-arena classes (8..32),
 * searched one coordinate at a time from the context's current parameters.
 * The results of a run do not depend on any of these (only its speed).  The
 * winner goes to *best (may be NULL) with its growth time on the sample in
 * *best_ms (may be NULL), into a per-context cache keyed by the graph's shape
 * (log2 n, weighted, degree width), and with MSCD_TUNE_APPLY into the context's
 * parameters; MSCD_TUNE_CACHED returns a cached result without timing.  Clears
 * the context's last run (MSCD_ENORESULT for the getters until the next run).
 * alphas is a host array. */
int mscd_autotune(mscd_ctx *ctx, int32_t graph_id, const double *alphas, int32_t n_scales, int64_t n_sample,
                  uint32_t flags, mscd_params *best, double *best_ms);

/* Stability across scales (Sec. 4): nmi_succ double[n_scales-1] with the
 * overlapping NMI between deduplicated sets of scales i and i+1; nmi_win3 and
 * nmi_win5 double[n_scales] with its mean over the window of 3 (5) scales
 * centred on scale i (clipped at the ends; NaN when the window holds no pair).
 * Any pointer may be NULL. */
int mscd_get_stability(mscd_ctx *ctx, double *nmi_succ, double *nmi_win3, double *nmi_win5);

/* The window means of mscd_get_stability for any list of successive-scale
 * NMI values (Sec. 4: "averaged over p successive scales"): out[i] is the
 * mean of nmi_succ[j] (the pair of scales j, j+1) over the pairs inside the
 * window of p scales centred on scale i, clipped at the ends; NaN when the
 * window holds no pair.  nmi_succ host double[n_scales-1] (may be NULL when
 * n_scales = 1), out host double[n_scales].  EINVAL unless n_scales >= 1 and
 * p >= 2.  Host code only (no context, no GPU), e.g. for the NMI of merged
 * shards (mscd_merge_shards + mscd_nmi_covers). */
int mscd_window_means(const double *nmi_succ, int32_t n_scales, int32_t p, double *out);

/* The same for part `part` of a union graph (mscd_graph_union); part 0 is what
 * mscd_get_stability returns.  A part without seeds in the run gets NaN.
 * EINVAL for a part outside the last run's graph. */
int mscd_get_stability_part(mscd_ctx *ctx, int32_t part, double *nmi_succ, double *nmi_win3, double *nmi_win5);

/* Totals of the last run. */
int mscd_get_run_stats(mscd_ctx *ctx, mscd_run_stats *out);

/* The overlapping NMI of Sec. 4 between two covers of n nodes given on the
 * host (ptr int64[n_x+1], nodes int32: each list non-empty, strictly
 * ascending, ids in [0, n); EINVAL otherwise), e.g. a scale's communities
 * against a reference partition.  NaN if a cover is empty. */
int mscd_nmi_covers(mscd_ctx *ctx, int64_t n, const int64_t *ptr_a, const int32_t *nodes_a, int64_t n_a,
                    const int64_t *ptr_b, const int32_t *nodes_b, int64_t n_b, double *nmi);

/* ---- seeds split across GPUs --------------------------------------------
 * Units are independent (each grows from its own seed, Alg. 1), so one job's
 * seeds can be split across GPUs (one process each) and every process runs
 * mscd_run on its share.  What each returns for a scale is its shard of the
 * deduplicated communities; mscd_merge_shards joins the shards of one scale
 * into exactly what one mscd_run over all the seeds returns for it: the
 * distinct member lists, numbered in order of their smallest generating seed
 * index in the whole job, and the community of every seed.  Host code only:
 * it needs no context and no GPU, so it runs wherever the shards were
 * gathered. */
typedef struct mscd_cover_shard {
    int64_t n_seeds;           /* seeds this shard grew                              */
    const int64_t *seed_index; /* int64[n_seeds]: each seed's index in the whole job */
    const int32_t *seed2comm;  /* int32[n_seeds]: its community in this shard        */
    int64_t n_comms;           /* communities of this shard                          */
    const int64_t *ptr;        /* int64[n_comms+1], ptr[0] = 0                       */
    const int32_t *nodes;      /* int32[ptr[n_comms]], each list non-empty and
                                  strictly ascending, ids >= 0                       */
    const double *fitness;     /* double[n_comms], or NULL                           */
} mscd_cover_shard;

/* Merge n_shards shards of one scale (host pointers).  The seed indices of
 * all shards together must be 0..n_seeds_total-1, each exactly once, and
 * every community of a shard must be the community of one of its seeds;
 * MSCD_EINVAL otherwise (also for a malformed list).  A list found in several
 * shards is one community; its fitness is taken from the shard holding its
 * smallest seed (the device computes f from exact integer sums, so every
 * shard has the same value).  Outputs: ptr int64[n_comms+1] (ptr_cap
 * entries), nodes int32[nodes_cap], fitness double[n_comms] (may be NULL;
 * then shards may omit theirs), seed2comm int32[n_seeds_total] (may be
 * NULL).  *n_comms and *n_nodes always get the sizes; a buffer too small
 * gives MSCD_ESMALL and nothing else is written. */
int mscd_merge_shards(const mscd_cover_shard *shards, int32_t n_shards, int64_t n_seeds_total, int64_t *ptr,
                      int64_t ptr_cap, int32_t *nodes, int64_t nodes_cap, double *fitness, int32_t *seed2comm,
                      int64_t *n_comms, int64_t *n_nodes);

/* Where the last failed mscd_run stopped and why ("" if none failed), e.g.
 * "mscd_run: dedup of scale 3: device memory allocation failed".  The string
 * belongs to the context and stays valid until its next failed run. */
const char *mscd_last_error(mscd_ctx *ctx);

/* Growth of every (scale, seed) unit without allocating device memory during
 * the call.  The paper has no counterpart: this entry point exists for
 * callers that cannot call cudaMalloc while they run (a process with a fixed
 * device-memory plan, an allocator that must not be bypassed, a latency
 * path that cannot take an allocation's synchronisation).  It grows the same
 * communities as mscd_run (no dedup, no stability) and allocates nothing:
 * the growth scratch lives in one 64 MiB device array built into the library,
 * which every GPU that loads the library holds until the process exits.
 *   graph_id   a graph resident in ctx (loaded earlier by mscd_graph_load_csr)
 *   alphas     host double[n_scales], finite and > 0, n_scales <= 256
 *   seeds      device int32[n_seeds] node ids, or NULL for every node
 *   outputs    device buffers owned by the caller, unit u = scale*n_seeds+seed:
 *              out_nodes int32[out_cap] (member lists, each ascending, at
 *              out_offset[u], length out_len[u]), out_fitness double[U],
 *              out_stats int64[U*MSCD_NSTATS], out_status int32[U],
 *              out_hash uint64[U] (hash of each member list)
 *   *n_nodes_needed  total member-list length of all units (host); set on
 *              MSCD_OK and MSCD_ESMALL only (after MSCD_ERANGE it leaves out
 *              the units that did not finish)
 *   cuda_stream      stream to order the work on (NULL = default stream)
 * Limits and errors: MSCD_ERANGE for more than 2^20 units or 256 scales in
 * one call, and for a unit that touches more than 8192 nodes (the per-unit
 * slot arena of the array); MSCD_ESMALL when out_cap < *n_nodes_needed;
 * MSCD_EINVAL for bad arguments or seeds.  The array holds the states of
 * about 270 (weighted graphs) to 380 (unweighted) units at once, so a call
 * keeps a fraction of a large GPU busy: it suits small and medium batches.
 * The call waits for its stream (cudaStreamSynchronize) after the seed check,
 * when seeds are given, and once more to read its counters back; it returns
 * with the outputs written.  The first call on a device looks up the array's
 * device address once (make that first call before any stream capture).
 * Every call reuses the same array, which keeps the previous call's contents
 * (the call clears what must start at zero): calls that overlap on the GPU,
 * on any stream or context of one device, race on it and must not be
 * issued. */
int mscd_grow_noalloc(mscd_ctx *ctx, int32_t graph_id, const double *alphas, int32_t n_scales,
                      const int32_t *seeds, int64_t n_seeds, int32_t *out_nodes, int64_t out_cap,
                      int64_t *out_offset, int32_t *out_len, double *out_fitness, int64_t *out_stats,
                      int32_t *out_status, uint64_t *out_hash, int64_t *n_nodes_needed, void *cuda_stream);

/* ------------------------------------------------------------- full method
 * The paper's whole algorithm (Alg. 2 with the growth of Alg. 3) rather than
 * one independent community per (scale, seed): seeds chosen by rule 1 (a
 * seed's neighbours cannot be seeds) or rule 2 (nor their neighbours) from the
 * nodes with at least two neighbours, taken in the order `prio` gives (the
 * paper's random order, passed in: int32[n], lower first, ties by id); or
 * given initial communities (init_ptr int64[n_init+1] from 0, init_nodes; the
 * first listed node of each is its seed).  For every scale in the given
 * order, while changes can be made: every community is grown once by Alg. 1
 * from its current members (seed kept) unless it already shares at least
 * eta * min(|c|, |c'|) nodes with another community c'; grown communities that
 * changed and the flagged ones are checked, each finding its first such
 * partner in the scan order of Alg. 2 (members ascending); the pairs merge in
 * rounds of disjoint pairs (the partner joins the checked community, which
 * keeps its seed).  The communities at the end of a scale start the next.
 * Every step is deterministic: seeds are chosen in rounds of local minima of
 * (prio, id), which equals the sequential greedy choice; a community's partner
 * is the first other community whose shared-node count reaches the ratio,
 * scanning its members ascending and each member's communities in index
 * order; a pair joins a merge round if neither side is already in it, and
 * later pairs rename the absorbed community to its absorber.
 * Host pointers.  ETIMEOUT: a scale needed more than max_iters iterations. */
typedef struct mscd_full_params {
    int32_t struct_size;  /* sizeof(mscd_full_params)                          */
    int32_t seed_rule;    /* 1 or 2 (0 = 1)                                    */
    double eta;           /* merge ratio in (0, 1] (0 = 0.5, Sec. 3's default) */
    int64_t max_iters;    /* iterations per scale before ETIMEOUT (0 = 1000)   */
} mscd_full_params;

int mscd_full_run(mscd_ctx *ctx, int32_t graph_id, const double *alphas, int32_t n_scales, const int32_t *prio,
                  const int64_t *init_ptr, const int32_t *init_nodes, int64_t n_init,
                  const mscd_full_params *params, void *cuda_stream);

/* Seeds of the last full run, in the order they were chosen. */
int mscd_full_get_seeds(mscd_ctx *ctx, int32_t *seeds, int64_t cap, int64_t *n);

/* Communities at the end of scale `scale`: ptr int64[n_comms+1], nodes int32
 * (each list ascending), seeds int32[n_comms] and fitness double[n_comms]
 * (either may be NULL).  ESMALL with the sizes when a buffer is short. */
int mscd_full_get_scale(mscd_ctx *ctx, int32_t scale, int64_t *ptr, int64_t ptr_cap, int32_t *nodes,
                        int64_t nodes_cap, int32_t *seeds, double *fitness, int64_t *n_comms, int64_t *n_nodes);

/* Iterations of the while loop, merges and growth calls at a scale, and the
 * overlapping NMI (Sec. 4) between its communities and the next scale's. */
int mscd_full_get_info(mscd_ctx *ctx, int32_t scale, int64_t *iterations, int64_t *merges, int64_t *grown,
                       double *nmi_next);

/* ------------------------------------------------------------------ serving
 * Local-community queries answered as they arrive (no counterpart in the
 * paper, whose method runs over all seeds at once; a query is the growth of
 * Alg. 1 from each of its seeds at one scale, the unit a run computes).
 *
 * mscd_serve_start starts `workers` host threads, each with its own CUDA
 * stream and growth buffers.  Waiting queries are batched continuously: a
 * free worker takes the oldest waiting query and every later one on the same
 * graph that fits its batch (max_batch_units seeds) and the memory budget,
 * and grows them in one persistent launch (plus the larger slot classes);
 * while it runs, other workers admit and launch the queries that arrive, so
 * batches overlap on the device.  Admission by memory: a query holds, until
 * its batch completes, its per-seed records plus its expected member lists
 * (the mean length seen on its graph, with a margin); a batch waits while the
 * holdings in flight would pass memory_budget (an oversized query runs alone).
 * Every seed is grown independently and exactly: a query's result is the same
 * alone and in any mix.  Graphs a waiting or running query uses cannot be
 * freed (MSCD_EBUSY).  The server's calls are thread-safe among themselves. */
typedef struct mscd_serve_params {
    int32_t struct_size;      /* sizeof(mscd_serve_params)                        */
    int32_t workers;          /* concurrent batches (0 = 4, at most 64)           */
    int64_t max_batch_units;  /* seeds per batch and per query (0 = 65536)        */
    int64_t memory_budget;    /* bytes batches in flight may hold (0 = a quarter
                                 of the free device memory at start)              */
} mscd_serve_params;

typedef struct mscd_serve_stats {
    int64_t queries_submitted, queries_done, units_done, batches;
    int64_t queued;               /* waiting now                                  */
    int64_t in_flight_bytes;      /* held by running batches now                  */
    int64_t max_in_flight_bytes;  /* largest holding seen                         */
    int64_t budget_bytes;
    int64_t max_concurrent_batches; /* most completed batches whose device
                                       intervals (first copy in to last copy
                                       out, timed by CUDA events on the
                                       worker's stream) overlapped at once   */
    int64_t overlap_us;           /* device time with two or more batches in
                                     flight, microseconds                     */
} mscd_serve_stats;

#define MSCD_Q_QUEUED 0
#define MSCD_Q_RUNNING 1
#define MSCD_Q_DONE 2

/* Start (EBUSY if running) / stop (waits for every queued and running query;
 * results not collected are dropped) the server of a context.  The node-slot
 * parameters of the context apply to its batches (persistent schedule). */
int mscd_serve_start(mscd_ctx *ctx, const mscd_serve_params *params);
int mscd_serve_stop(mscd_ctx *ctx);

/* Queue a query: seeds int32[n_seeds] (host, copied; 1 <= n_seeds <=
 * max_batch_units, else ERANGE; ids in [0, n) of the graph, else EINVAL) on
 * resident graph graph_id at scale alpha (finite, > 0).  *qid names it. */
int mscd_query_submit(mscd_ctx *ctx, int32_t graph_id, const int32_t *seeds, int32_t n_seeds, double alpha,
                      uint64_t *qid);

/* Device intervals of the completed batches, in completion order:
 * start_ms[i] and end_ms[i] (host double[cap]) are milliseconds after the
 * server started, from the batch's first host->device copy to its last
 * device->host copy, as CUDA events on the worker's stream timed them.
 * ESMALL with *n when cap is short. */
int mscd_serve_batch_intervals(mscd_ctx *ctx, double *start_ms, double *end_ms, int64_t cap, int64_t *n);

/* State of a query (MSCD_Q_*); wait: until done or timeout_us passed. */
int mscd_query_poll(mscd_ctx *ctx, uint64_t qid, int32_t *state);
int mscd_query_wait(mscd_ctx *ctx, uint64_t qid, int64_t timeout_us, int32_t *state);

/* Result of a done query (ENORESULT before): ptr int64[n_seeds+1] offsets of
 * each seed's sorted member list in nodes int32[nodes_cap], fitness
 * double[n_seeds] (may be NULL), *n_nodes the list entries; times_ms (may be
 * NULL) double[3] = queued, running, submit-to-done milliseconds.  ESMALL
 * (with *n_nodes) leaves the query in place; otherwise the query is released
 * and its status returned (OK, ETIMEOUT, EUNDECIDED, or the error that failed
 * its batch). */
int mscd_query_result(mscd_ctx *ctx, uint64_t qid, int64_t *ptr, int32_t *nodes, int64_t nodes_cap,
                      double *fitness, int64_t *n_nodes, double *times_ms);

int mscd_serve_get_stats(mscd_ctx *ctx, mscd_serve_stats *out);

#ifdef __cplusplus
}
#endif

#endif /* MSCD_H */
