// Community growth, one warp per (scale, seed) unit.
//
// Per unit the warp runs Alg. 1 repeated while a grow pass adds something
// (Alg. 2, "while changes can be made"), from c = {seed}:
//   grow : the max priority queue holds every frontier node (d_in > 0, not in
//          c), ranked by 2 d_in / k^alpha (Sec. 2), equal values by smaller
//          id.  Pop the best; add it iff f_{c+n} > f_c (Eq. 1-2, strict); on
//          an addition, update or add its outside neighbours in the queue.  A
//          rejected node leaves the queue until an addition touches it.
//   prune: only if the grow pass added something.  Passes over the members in
//          ascending id (seed excluded): remove n at once iff f_{c\n} > f_c;
//          repeat until a pass removes nothing.
//
// Pops are not done one at a time.  K and V change only when a node is
// added, so between two additions every pop faces the same add test: the
// node added next is the highest-ranked queued node that passes the test,
// and every queued node ranked before it is popped and rejected on the way.
// The warp finds it with one pass over the node slots (filter by a necessary
// condition, exact test on the survivors, exact argmax), so the cost of a
// long run of rejections is one pass instead of one pop each.  The common
// case (the top node passes) is a plain exact argmax.  Likewise a prune pass
// finds the smallest-id member that passes the remove test in one pass,
// removes it and continues after it.
//
// State per warp: node slots (id, d_in, k, priority key, flags) and an
// open-addressing hash node -> slot, either in shared memory (small class)
// or in a global-memory arena (large classes).  A unit whose touched nodes
// exceed the class capacity stops, is listed, and is grown again in a larger
// class; the result does not depend on the class.
#include "common.cuh"
#include "exact.cuh"
#include "grow.cuh"

namespace {

constexpr u32 F_MEMBER = 1u;
constexpr double NEG_INF = -__builtin_huge_val();

struct State {
    double *key;  // priority key (log d - alpha log k) while queued, else -inf
    i64 *din;     // d_in(u, c)
    i64 *kdeg;    // k_u
    i32 *id;      // node id
    i32 *hpos;    // hash bucket of the slot
    u32 *hsh;     // bucket -> slot + 1 (0 = empty)
    unsigned char *flag;
    int C, H;     // slot capacity, hash buckets (2C)
};

__device__ __forceinline__ State carve(unsigned char *base, int C) {
    State s;
    s.C = C;
    s.H = 2 * C;
    s.key = (double *)base;
    s.din = (i64 *)(base + 8ull * C);
    s.kdeg = (i64 *)(base + 16ull * C);
    s.id = (i32 *)(base + 24ull * C);
    s.hpos = (i32 *)(base + 28ull * C);
    s.hsh = (u32 *)(base + 32ull * C);
    s.flag = base + 40ull * C;
    return s;
}

__device__ __forceinline__ u32 lanemask_lt() {
    u32 m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ u32 hash_node(i32 v) { return (u32)v * 0x9E3779B1u; }

__device__ __forceinline__ u64 mix64(u64 x) {
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebull;
    x ^= x >> 31;
    return x;
}

struct Unit {
    i64 K, V;
    int ns;  // slots in use
    i32 seed;
    double alpha, E2;
    i64 edges, adds, removes, rounds;
    u32 xflags;  // EXACT_* of every decision
    bool ovf;    // slot capacity exceeded
    bool err;    // internal probe bound hit (cannot happen at load <= 1/2)
};

// Look up (and insert if absent) node v for every active lane.  Warp-collective.
__device__ int lookup_insert(const State &st, Unit &U, i32 v, bool active, const i64 *kglob) {
    const u32 hm = (u32)st.H - 1u;
    int slot = -1;
    u32 h = 0;
    bool need = false;
    if (active) {
        h = hash_node(v) & hm;
        int p = 0;
        for (; p < st.H; ++p) {
            u32 x = st.hsh[h];
            if (x == 0u) {
                need = true;
                break;
            }
            if (st.id[x - 1] == v) {
                slot = (int)x - 1;
                break;
            }
            h = (h + 1u) & hm;
        }
        if (p == st.H) U.err = true;
    }
    const u32 ball = __ballot_sync(FULL_MASK, need);
    if (ball) {
        const int cnt = __popc(ball);
        if (U.ns + cnt > st.C) {
            U.ovf = true;
            __syncwarp();
            return -1;
        }
        if (need) {
            slot = U.ns + __popc(ball & lanemask_lt());
            st.id[slot] = v;
            st.din[slot] = 0;
            st.kdeg[slot] = kglob[v];
            st.key[slot] = NEG_INF;
            st.flag[slot] = 0;
            st.hpos[slot] = -1;
            int p = 0;
            for (; p < st.H; ++p) {
                if (atomicCAS(&st.hsh[h], 0u, (u32)(slot + 1)) == 0u) {
                    st.hpos[slot] = (i32)h;
                    break;
                }
                h = (h + 1u) & hm;
            }
            if (p == st.H) U.err = true;
        }
        U.ns += cnt;
    }
    U.err = __any_sync(FULL_MASK, U.err);
    __syncwarp();
    return slot;
}

__device__ __forceinline__ double prio_key(i64 d, double logk, double alpha) {
    return log((double)d) - alpha * logk;
}

// Slot a ranks before slot b in the queue (exact; canonical argument order so
// that every lane evaluating the pair gets the same answer).
__device__ __forceinline__ bool ranks_before(const State &st, int a, double ka, int b, double kb, Unit &U) {
    const double diff = ka - kb;
    if (diff > U.E2) return true;
    if (diff < -U.E2) return false;
    const bool swap = a > b;
    const int x = swap ? b : a, y = swap ? a : b;
    int s = exact::sign_delta(st.din[x], st.din[y], st.kdeg[x], st.kdeg[y], U.alpha, &U.xflags);
    bool xfirst = s ? (s > 0) : (st.id[x] < st.id[y]);
    return swap ? !xfirst : xfirst;
}

__device__ __forceinline__ void warp_best(const State &st, int &best, double &bk, Unit &U) {
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        int ob = __shfl_xor_sync(FULL_MASK, best, off);
        double ok = __shfl_xor_sync(FULL_MASK, bk, off);
        if (ob >= 0 && (best < 0 || ranks_before(st, ob, ok, best, bk, U))) {
            best = ob;
            bk = ok;
        }
    }
    best = __shfl_sync(FULL_MASK, best, 0);
    bk = __shfl_sync(FULL_MASK, bk, 0);
}

// Highest-ranked queued slot, or -1.
__device__ int queue_top(const State &st, Unit &U) {
    const int lane = threadIdx.x & 31;
    int best = -1;
    double bk = NEG_INF;
    for (int i = lane; i < U.ns; i += 32) {
        const double k = st.key[i];
        if (k == NEG_INF) continue;
        if (best < 0 || ranks_before(st, i, k, best, bk, U)) {
            best = i;
            bk = k;
        }
    }
    warp_best(st, best, bk, U);
    return best;
}

// Highest-ranked queued slot that passes the add test at the current K, V.
__device__ int best_passing(const State &st, Unit &U) {
    const int lane = threadIdx.x & 31;
    int best = -1;
    double bk = NEG_INF;
    for (int i = lane; i < U.ns; i += 32) {
        const double k = st.key[i];
        if (k == NEG_INF) continue;
        const i64 d = st.din[i], kd = st.kdeg[i];
        if (!exact::add_possible(U.K, U.V, d, kd, U.alpha)) continue;
        if (!exact::add_test(U.K, U.V, d, kd, U.alpha, &U.xflags)) continue;
        if (best < 0 || ranks_before(st, i, k, best, bk, U)) {
            best = i;
            bk = k;
        }
    }
    warp_best(st, best, bk, U);
    return best;
}

// Pop (reject) every queued slot ranked before `best` (all of them if best < 0).
__device__ void drop_before(const State &st, int best, Unit &U) {
    const int lane = threadIdx.x & 31;
    const double bk = best >= 0 ? st.key[best] : 0.0;
    for (int i = lane; i < U.ns; i += 32) {
        const double k = st.key[i];
        if (k == NEG_INF) continue;
        if (best < 0 || ranks_before(st, i, k, best, bk, U)) st.key[i] = NEG_INF;
    }
    __syncwarp();
}

// Scan node u's row, adding sign*w to d_in of every neighbour; with requeue,
// (re)insert outside neighbours in the queue with their new key.
__device__ void expand(const State &st, const DevGraph &G, Unit &U, i32 u, int sign, bool requeue) {
    const int lane = threadIdx.x & 31;
    const i64 rs = G.rp[u], re = G.rp[u + 1];
    for (i64 b = rs; b < re; b += 32) {
        const i64 e = b + lane;
        const bool act = e < re;
        i32 v = 0;
        i64 w = 0;
        if (act) {
            v = G.col[e];
            w = G.wfx ? G.wfx[e] : 1;
        }
        const int s = lookup_insert(st, U, v, act, G.k);
        if (U.ovf || U.err) return;
        if (act) {
            const i64 d = st.din[s] + sign * w;
            st.din[s] = d;
            if (requeue && !(st.flag[s] & F_MEMBER)) st.key[s] = prio_key(d, G.logk[v], U.alpha);
        }
    }
    __syncwarp();
    U.edges += re - rs;
}

__device__ void accept(const State &st, const DevGraph &G, Unit &U, int s) {
    const i64 d = st.din[s], kd = st.kdeg[s];
    const i32 u = st.id[s];
    __syncwarp();
    if ((threadIdx.x & 31) == 0) {
        st.flag[s] |= F_MEMBER;
        st.key[s] = NEG_INF;
    }
    __syncwarp();
    U.K += 2 * d;
    U.V += kd;
    U.adds++;
    expand(st, G, U, u, +1, true);
}

// Smallest-id member (not the seed, id > last) whose removal raises f; -1 if none.
__device__ int first_removable(const State &st, Unit &U, i32 last) {
    const int lane = threadIdx.x & 31;
    i32 bid = INT32_MAX;
    int bslot = -1;
    for (int i = lane; i < U.ns; i += 32) {
        if (!(st.flag[i] & F_MEMBER)) continue;
        const i32 u = st.id[i];
        if (u == U.seed || u <= last || u >= bid) continue;
        const i64 d = st.din[i], kd = st.kdeg[i];
        if (!exact::remove_possible(U.K, U.V, d, kd, U.alpha)) continue;
        if (!exact::remove_test(U.K, U.V, d, kd, U.alpha, &U.xflags)) continue;
        bid = u;
        bslot = i;
    }
    const i32 m = __reduce_min_sync(FULL_MASK, bid);
    const u32 who = __ballot_sync(FULL_MASK, bid == m && bslot >= 0);
    if (!who) return -1;
    return __shfl_sync(FULL_MASK, bslot, __ffs(who) - 1);
}

__device__ void remove_node(const State &st, const DevGraph &G, Unit &U, int s) {
    const i64 d = st.din[s], kd = st.kdeg[s];
    const i32 u = st.id[s];
    __syncwarp();
    if ((threadIdx.x & 31) == 0) st.flag[s] &= ~F_MEMBER;
    __syncwarp();
    U.K -= 2 * d;
    U.V -= kd;
    U.removes++;
    expand(st, G, U, u, -1, false);
}

__device__ void clear_hash(const State &st, const Unit &U) {
    __syncwarp();
    if (U.err) {
        for (int i = threadIdx.x & 31; i < st.H; i += 32) st.hsh[i] = 0u;
    } else {
        for (int i = threadIdx.x & 31; i < U.ns; i += 32)
            if (st.hpos[i] >= 0) st.hsh[st.hpos[i]] = 0u;
    }
    __syncwarp();
}

// Sort the members ascending into scratch (the key array viewed as int32[2C]),
// hash the list and write it out.  Returns false if the output buffer is full.
__device__ bool emit(const State &st, const GrowArgs &a, const DevGraph &G, Unit &U, i64 unit, int status) {
    const int lane = threadIdx.x & 31;
    i32 *scr = (i32 *)st.key;
    int m = 0;
    __syncwarp();
    for (int b = 0; b < U.ns; b += 32) {
        const int i = b + lane;
        const bool mem = i < U.ns && (st.flag[i] & F_MEMBER);
        const u32 ball = __ballot_sync(FULL_MASK, mem);
        i32 v = mem ? st.id[i] : 0;
        __syncwarp();
        if (mem) scr[m + __popc(ball & lanemask_lt())] = v;
        m += __popc(ball);
    }
    int P = 1;
    while (P < m) P <<= 1;
    for (int i = m + lane; i < P; i += 32) scr[i] = INT32_MAX;
    __syncwarp();
    for (int kk = 2; kk <= P; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < P; i += 32) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const i32 x = scr[i], y = scr[ixj];
                    const bool up = (i & kk) == 0;
                    if ((x > y) == up) {
                        scr[i] = y;
                        scr[ixj] = x;
                    }
                }
            }
            __syncwarp();
        }
    }
    u64 h = 0;
    for (int i = lane; i < m; i += 32) h += mix64((u64)(u32)scr[i] + 0x9E3779B97F4A7C15ull * (u64)(i + 1));
#pragma unroll
    for (int o = 16; o; o >>= 1) h += __shfl_xor_sync(FULL_MASK, h, o);
    h ^= mix64((u64)m);
    if (h == 0) h = 1;
    unsigned long long off = 0;
    if (lane == 0) off = atomicAdd(a.out_cursor, (unsigned long long)m);
    off = __shfl_sync(FULL_MASK, off, 0);
    if ((i64)(off + m) > a.out_cap) {
        if (lane == 0) atomicAdd(a.out_needed, (unsigned long long)m);
        return false;
    }
    for (int i = lane; i < m; i += 32) a.out_nodes[off + i] = scr[i];
    if (lane == 0) {
        a.uoff[unit] = (i64)off;
        a.ulen[unit] = m;
        a.uhash[unit] = h;
        double f = 0.0;
        if (U.K > 0) {
            const double LN2 = 0.6931471805599453;
            f = exp(log((double)U.K) - U.alpha * log((double)U.V) + (1.0 - U.alpha) * (double)G.unit_exp * LN2);
        }
        a.uf[unit] = f;
        i64 *stt = a.ustat + unit * MSCD_NSTATS;
        stt[MSCD_STAT_EDGES] = U.edges;
        stt[MSCD_STAT_ADDS] = U.adds;
        stt[MSCD_STAT_REMOVES] = U.removes;
        stt[MSCD_STAT_ROUNDS] = U.rounds;
        stt[MSCD_STAT_K] = U.K;
        stt[MSCD_STAT_V] = U.V;
        stt[MSCD_STAT_SLOW] = (U.xflags & EXACT_SLOW) ? 1 : 0;
        stt[MSCD_STAT_UNDECIDED] = (U.xflags & EXACT_UNDECIDED) ? 1 : 0;
        a.ustatus[unit] = status;
    }
    return true;
}

__device__ void grow_unit(const State &st, const GrowArgs &a, i64 unit) {
    const int lane = threadIdx.x & 31;
    const DevGraph &G = a.G;
    Unit U;
    const i64 si = unit % a.n_seeds;
    U.alpha = a.alphas[unit / a.n_seeds];
    U.seed = a.seeds ? a.seeds[si] : (i32)si;
    U.E2 = 2.0 * 0x1p-44 * (1.0 + U.alpha);
    U.K = 0;
    U.V = G.k[U.seed];
    U.ns = 0;
    U.edges = U.adds = U.removes = U.rounds = 0;
    U.xflags = 0;
    U.ovf = U.err = false;
    int status = MSCD_OK;

    lookup_insert(st, U, U.seed, lane == 0, G.k);  // slot 0
    if (lane == 0) st.flag[0] = F_MEMBER;
    __syncwarp();
    expand(st, G, U, U.seed, +1, false);

    while (!U.ovf && !U.err) {
        if (U.rounds >= a.max_rounds) {
            status = MSCD_ETIMEOUT;
            break;
        }
        U.rounds++;
        // queue = whole frontier
        for (int i = lane; i < U.ns; i += 32) {
            const i64 d = st.din[i];
            st.key[i] = (!(st.flag[i] & F_MEMBER) && d > 0) ? prio_key(d, G.logk[st.id[i]], U.alpha) : NEG_INF;
        }
        __syncwarp();
        i64 added = 0;
        for (;;) {
            const int top = queue_top(st, U);
            if (top < 0) break;
            int s = top;
            if (!exact::add_test(U.K, U.V, st.din[top], st.kdeg[top], U.alpha, &U.xflags)) {
                s = best_passing(st, U);
                drop_before(st, s, U);
                if (s < 0) break;
            }
            accept(st, G, U, s);
            added++;
            if (U.ovf || U.err) break;
        }
        if (U.ovf || U.err || added == 0) break;
        for (;;) {  // prune passes
            i64 removed = 0;
            i32 last = -1;
            for (;;) {
                const int s = first_removable(st, U, last);
                if (s < 0) break;
                last = st.id[s];
                remove_node(st, G, U, s);
                removed++;
                if (U.ovf || U.err) break;
            }
            if (removed == 0 || U.ovf || U.err) break;
        }
    }
    U.xflags = __reduce_or_sync(FULL_MASK, U.xflags);
    if (U.err) {
        if (lane == 0) atomicOr(a.error_flags, 1u);
    } else if (U.ovf) {
        if (lane == 0) a.retry_state[atomicAdd(a.n_retry_state, 1ull)] = unit;
    } else {
        if (status == MSCD_OK && (U.xflags & EXACT_UNDECIDED)) status = MSCD_EUNDECIDED;
        if (!emit(st, a, G, U, unit, status)) {
            if (lane == 0) a.retry_out[atomicAdd(a.n_retry_out, 1ull)] = unit;
        }
    }
    clear_hash(st, U);
}

__global__ void __launch_bounds__(GROW_MAX_THREADS) grow_kernel(GrowArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const i64 gw = (i64)blockIdx.x * (blockDim.x >> 5) + wib;
    unsigned char *base = a.use_smem ? smem + (size_t)wib * a.state_bytes : a.gstate + (size_t)gw * a.state_bytes;
    const State st = carve(base, a.cap);
    for (int i = lane; i < st.H; i += 32) st.hsh[i] = 0u;
    __syncwarp();
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(a.work_counter, 1ull);
        t = __shfl_sync(FULL_MASK, t, 0);
        if ((i64)t >= a.n_work) break;
        const i64 unit = a.work_list ? a.work_list[t] : (i64)t;
        grow_unit(st, a, unit);
    }
}

}  // namespace

size_t grow_state_bytes(int cap) { return 41ull * (size_t)cap; }

int grow_launch(const GrowArgs &a, int blocks, int threads, size_t smem, cudaStream_t st) {
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(grow_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_status(e);
    }
    grow_kernel<<<blocks, threads, smem, st>>>(a);
    return cuda_status(cudaGetLastError());
}

int grow_occupancy(int threads, size_t smem, int *blocks_per_sm) {
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(grow_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_status(e);
    }
    return cuda_status(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, grow_kernel, threads, smem));
}
