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
// condition, exact test on the survivors, exact argmax), so a long run of
// rejections costs one pass instead of one pop each.  The common case (the
// top node passes) is an exact argmax over the queue.  Likewise a prune pass
// finds the smallest-id member that passes the remove test in one pass,
// removes it and continues after it.
//
// Ranking keys are binary32 log d - alpha log k, compared with a certified
// bound; pairs closer than the bound are ordered by the exact comparator.
// With u32 = 2^-24 and L = log of the largest degree, a key carries at most
// u32 (1+alpha) + 3 u32 |log d| + 5 u32 alpha |log k| <= 5 u32 (1+alpha)(1+L)
// of error (conversions, <= 1 ulp logf twice, fl(alpha), product,
// difference); E = 2^-20 (1+alpha)(1+L) per key is above it.
//
// Queue argmax: the slots are split into groups of 32 and each group keeps an
// upper bound of its largest key (raised by atomicMax when a key rises).  A
// pop recomputes exactly every group whose bound is within 2E of the largest
// bound, and repeats while the largest bound drops; the best node is then in
// a recomputed group (a group left out has a bound, hence a true maximum,
// below the true maximum minus 2E), so the result is the exact argmax at the
// cost of a few groups.  Bounds are made exact again wherever the kernel
// holds the keys anyway (the added node's group, groups the bulk rejection
// visits), so that a pop rarely meets a stale one.
//
// State per warp: node slots (d_in, key, id with the member flag in its sign
// bit; k_u is read from the graph's degree array, which every unit shares),
// a member list (slots in joining order, for the prune passes and the
// output), group bounds and an open-addressing hash node -> slot, in shared memory
// (first class) or in a global-memory arena (larger classes, run at high
// occupancy so that the dependent steps of one unit overlap with those of
// many others).  The hash table starts small and doubles (rehashing every
// slot) whenever it would pass a quarter full, up to twice the slot
// capacity: a unit's lookups touch a table sized to its own touched nodes,
// not to its class.  A unit whose touched nodes exceed the class capacity
// stops, is listed, and is grown again in a larger class; the result does
// not depend on the class, on the table size or on slot order.
#include "common.cuh"
#include "exact.cuh"
#include "grow.cuh"

namespace {

// A slot's id holds the node id (< 2^31) with the member flag in bit 31.
constexpr i32 MEMBER_BIT = (i32)0x80000000u;
__device__ __forceinline__ i32 node_of(i32 x) { return x & 0x7fffffff; }
constexpr int HASH_MIN = 256;  // buckets of a unit's table at its start

// Per-warp counters of the unit being grown (edges scanned, additions,
// removals), kept in shared memory by the warp's lane 0 rather than in
// registers of every lane.
__shared__ unsigned long long g_wcnt[GROW_MAX_THREADS / 32][3];

// Order-preserving int image of a binary32 value (no NaNs occur).
__device__ __forceinline__ int ord(float f) {
    const int b = __float_as_int(f);
    return b >= 0 ? b : b ^ 0x7fffffff;
}
__device__ __forceinline__ float unord(int o) { return __int_as_float(o >= 0 ? o : o ^ 0x7fffffff); }
constexpr int ORD_NEG_INF = (int)(0xff800000u ^ 0x7fffffffu);
constexpr float NEG_INF = -__builtin_huge_valf();

// VT: type of d_in in the slots; HT: type of a hash bucket (slot + 1).
template <class VT, class HT, bool WEIGHTED>
struct State {
    VT *din;              // [C] d_in(u, c)
    float *key;           // [C] ranking key while queued, else -inf
    i32 *id;              // [C] node id | MEMBER_BIT for members
    HT *hsh;              // [Hmax] bucket -> slot + 1 (0 = empty); the first H of the unit in use
    HT *mem;              // [C] slots of the members, in the order they joined
    int *gmax;            // [C/32] upper bound of the group's largest key (ord image)
    int *qmax;            // [C/32] upper bound of the group's largest d_in / k (ord image)
    const i64 *gk;        // the graph's k_u
    int C, Hmax;
};

// Layout: din | key | id | hash | member list | group bounds.  Rounded up to
// 128 bytes: per-warp states are laid end to end, and the 8-byte slot arrays
// must stay aligned for every warp; the table starts on a 16-byte boundary
// (C >= 32).
template <class VT, class HT, bool WEIGHTED>
__host__ __device__ __forceinline__ size_t state_bytes_t(int C) {
    const size_t per = sizeof(VT) + 4 + 4 + 3 * sizeof(HT);
    const size_t b = (size_t)C * per + 8 * (size_t)(C / 32);
    return (b + 127) & ~(size_t)127;
}

template <class VT, class HT, bool WEIGHTED>
__device__ __forceinline__ State<VT, HT, WEIGHTED> carve(unsigned char *base, int C, int *bounds, HT *hsh,
                                                         const i64 *gk) {
    State<VT, HT, WEIGHTED> s;
    s.C = C;
    s.Hmax = 2 * C;
    s.gk = gk;
    size_t o = 0;
    s.din = (VT *)(base + o);
    o += sizeof(VT) * (size_t)C;
    s.key = (float *)(base + o);
    o += 4 * (size_t)C;
    s.id = (i32 *)(base + o);
    o += 4 * (size_t)C;
    s.hsh = hsh ? hsh : (HT *)(base + o);  // the table may live in shared memory
    o += 2 * sizeof(HT) * (size_t)C;
    s.mem = (HT *)(base + o);
    o += sizeof(HT) * (size_t)C;
    s.gmax = (int *)(base + o);
    o += 4 * (size_t)(C / 32);
    s.qmax = (int *)(base + o);
    if (bounds) {  // group bounds kept apart (shared memory for a global-arena class)
        s.gmax = bounds;
        s.qmax = bounds + C / 32;
    }
    return s;
}

__device__ __forceinline__ u32 lanemask_lt() {
    u32 m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ u32 hash_node(i32 v) { return (u32)v * 0x9E3779B1u; }

__device__ __forceinline__ float rank_key(i64 d, i64 k, float alpha32) {
    return logf(exact::i2f(d)) - alpha32 * logf(exact::i2f(k));
}

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
    int nm;  // members (entries of the member list)
    int H;   // buckets of the hash table in use (a power of two, <= Hmax)
    i32 seed;
    double alpha;
    float alpha32, E2, kmaxf;
    i64 rounds;
    u32 xflags;  // EXACT_* of this lane's decisions
    bool ovf;    // slot capacity exceeded
    bool err;    // probe bound hit (cannot happen at load <= 1/2)
};

template <class VT>
struct SlotView {
    VT din;
    i64 kdeg;
    float logk;  // logf of k as a binary32 value (the graph's table)
    bool member;
};

// Zero the buckets [0, H) of a table (16-byte stores when the table allows).
template <class HT>
__device__ __forceinline__ void zero_table(HT *hsh, int H) {
    const int lane = threadIdx.x & 31;
    const size_t bytes = (size_t)H * sizeof(HT);
    if (((size_t)hsh & 15) == 0 && bytes % 512 == 0) {
        uint4 *q = (uint4 *)hsh;
        for (size_t i = lane; i < bytes / 16; i += 32) q[i] = make_uint4(0u, 0u, 0u, 0u);
    } else {
        for (int i = lane; i < H; i += 32) hsh[i] = 0;
    }
}

template <class HT>
__device__ __forceinline__ HT bucket_cas(HT *p, HT want) {
    if (sizeof(HT) == 2)
        return (HT)atomicCAS((unsigned short int *)p, (unsigned short int)0, (unsigned short int)want);
    return (HT)atomicCAS((unsigned int *)p, 0u, (unsigned int)want);
}

// Double the unit's table until `incoming` more slots keep it at most a
// quarter full (or it reaches Hmax), reinserting every slot.  Warp-collective.
template <class VT, class HT, bool WEIGHTED>
__device__ void rehash(const State<VT, HT, WEIGHTED> &st, Unit &U, int incoming) {
    int nH = U.H;
    while (4 * (U.ns + incoming) > nH && nH < st.Hmax) nH <<= 1;
    if (nH == U.H) return;
    __syncwarp();
    zero_table(st.hsh, U.H);  // buckets at and above U.H are zero already
    __syncwarp();
    const u32 hm = (u32)nH - 1u;
    for (int i = threadIdx.x & 31; i < U.ns; i += 32) {
        u32 h = hash_node(node_of(st.id[i])) & hm;
        int p = 0;
        while (bucket_cas(&st.hsh[h], (HT)(i + 1)) != 0 && ++p < nH) h = (h + 1u) & hm;
        if (p >= nH) U.err = true;
    }
    U.err = __any_sync(FULL_MASK, U.err);
    U.H = nH;
    __syncwarp();
}

// Look up (and insert if absent) node v for every active lane.  Warp-collective.
template <class VT, class HT, bool WEIGHTED>
__device__ int lookup_insert(const State<VT, HT, WEIGHTED> &st, const DevGraph &G, Unit &U, i32 v, bool active,
                             SlotView<VT> *sv = nullptr) {
    if (4 * (U.ns + 32) > U.H && U.H < st.Hmax) rehash(st, U, 32);
    const u32 hm = (u32)U.H - 1u;
    int slot = -1;
    u32 h = 0;
    bool need = false;
    if (active) {
        // k_v is loaded alongside the bucket: both depend only on v
        if (sv) {
            sv->kdeg = G.k[v];
            sv->logk = G.logk[v];
        }
        h = hash_node(v) & hm;
        int p = 0;
        for (; p < U.H; ++p) {
            const u32 x = st.hsh[h];
            if (x == 0u) {
                need = true;
                break;
            }
            const i32 idx = st.id[x - 1];
            VT dv = 0;
            if (sv) dv = st.din[x - 1];  // loaded with the id: one dependent step after the bucket
            if (node_of(idx) == v) {
                slot = (int)x - 1;
                if (sv) {
                    sv->din = dv;
                    sv->member = idx < 0;
                }
                break;
            }
            h = (h + 1u) & hm;
        }
        if (p == U.H) U.err = true;
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
            st.key[slot] = NEG_INF;
            if (sv) {
                sv->din = 0;
                sv->member = false;
            }
        }
        // Claim the empty buckets found.  Only this warp writes its table, so
        // lanes that found the same bucket are told apart with a match instead
        // of atomics: the lowest takes it, the others move on to the next empty
        // bucket; every round settles at least one lane.
        const int lane = threadIdx.x & 31;
        bool pending = need;
        for (int r = 0; r <= 32; ++r) {
            const u32 grp = __match_any_sync(FULL_MASK, pending ? h : 0xffffffffu - (u32)lane);
            if (pending && __ffs(grp) - 1 == lane) {
                st.hsh[h] = (HT)(slot + 1);
                pending = false;
            }
            __syncwarp();
            if (!__any_sync(FULL_MASK, pending)) break;
            if (pending) {
                int p = 0;
                do {
                    h = (h + 1u) & hm;
                    ++p;
                } while (st.hsh[h] != 0 && p < U.H);
                if (p >= U.H) {
                    U.err = true;
                    pending = false;
                }
            }
        }
        if (pending) U.err = true;
        U.ns += cnt;
    }
    U.err = __any_sync(FULL_MASK, U.err);
    __syncwarp();
    return slot;
}

// Slot a ranks before slot b (exact; canonical argument order so that every
// lane evaluating the pair gets the same answer).
template <class S>
__device__ __forceinline__ bool ranks_before(const S &st, int a, float ka, int b, float kb, Unit &U) {
    const float diff = ka - kb;
    if (diff > U.E2) return true;
    if (diff < -U.E2) return false;
    const bool swap = a > b;
    const int x = swap ? b : a, y = swap ? a : b;
    const i32 ix = node_of(st.id[x]), iy = node_of(st.id[y]);
    const int s = exact::sign_delta((i64)st.din[x], (i64)st.din[y], st.gk[ix], st.gk[iy], U.alpha, U.xflags);
    const bool xfirst = s ? (s > 0) : (ix < iy);
    return swap ? !xfirst : xfirst;
}

// Warp-wide best of the lanes' candidates (slot `best`, key `bk`; -1 none),
// returned to every lane.  The largest key comes from one integer max
// reduction; only lanes within E2 of it can rank first, and when there are
// several (rare) they are compared exactly in lane order.
template <class S>
__device__ __forceinline__ void warp_best(const S &st, int &best, float &bk, Unit &U) {
    const int om = __reduce_max_sync(FULL_MASK, best >= 0 ? ord(bk) : ORD_NEG_INF);
    if (om == ORD_NEG_INF) {
        best = -1;
        bk = NEG_INF;
        return;
    }
    const float mk = unord(om);
    u32 cand = __ballot_sync(FULL_MASK, best >= 0 && !(mk - bk > U.E2));
    int wb = -1;
    float wk = NEG_INF;
    while (cand) {
        const int l = __ffs(cand) - 1;
        cand &= cand - 1;
        const int b = __shfl_sync(FULL_MASK, best, l);
        const float k = __shfl_sync(FULL_MASK, bk, l);
        if (wb < 0 || ranks_before(st, b, k, wb, wk, U)) {
            wb = b;
            wk = k;
        }
    }
    best = wb;
    bk = wk;
}

constexpr int UNROLL = 4;

// Exact argmax over every queued slot (one pass).
template <class S>
__device__ int queue_top_flat(const S &st, Unit &U) {
    const int lane = threadIdx.x & 31;
    int best = -1;
    float bk = NEG_INF;
    for (int b = 0; b < U.ns; b += 32 * UNROLL) {
        float kv[UNROLL];
#pragma unroll
        for (int j = 0; j < UNROLL; ++j) {
            const int i = b + 32 * j + lane;
            kv[j] = i < U.ns ? st.key[i] : NEG_INF;
        }
#pragma unroll
        for (int j = 0; j < UNROLL; ++j) {
            if (kv[j] == NEG_INF) continue;
            const int i = b + 32 * j + lane;
            if (best < 0 || ranks_before(st, i, kv[j], best, bk, U)) {
                best = i;
                bk = kv[j];
            }
        }
    }
    warp_best(st, best, bk, U);
    return best;
}

template <class S>
__device__ __forceinline__ int max_bound(const S &st, int G) {
    int m = ORD_NEG_INF;
    for (int g = threadIdx.x & 31; g < G; g += 32) m = max(m, st.gmax[g]);
    return __reduce_max_sync(FULL_MASK, m);
}

// Queue = the whole frontier (outside nodes with d_in > 0): every slot's key
// and every group's two bounds, in one pass.
template <class S>
__device__ void build_queue(const S &st, const Unit &U) {
    const int lane = threadIdx.x & 31;
    const int G = (U.ns + 31) >> 5;
    for (int g = 0; g < G; ++g) {
        const int i = g * 32 + lane;
        float k = NEG_INF, q = NEG_INF;
        if (i < U.ns) {
            const i32 x = st.id[i];
            const i64 d = (i64)st.din[i];
            if (x >= 0 && d > 0) {
                const i64 kd = st.gk[x];
                k = rank_key(d, kd, U.alpha32);
                q = __fdividef(exact::i2f(d), exact::i2f(kd));
            }
            st.key[i] = k;
        }
        const int o = __reduce_max_sync(FULL_MASK, ord(k));
        const int qo = __reduce_max_sync(FULL_MASK, k == NEG_INF ? ORD_NEG_INF : ord(q));
        if (lane == 0) {
            st.gmax[g] = o;
            st.qmax[g] = qo;
        }
    }
    for (int g = G + lane; g < st.C / 32; g += 32) {
        st.gmax[g] = ORD_NEG_INF;
        st.qmax[g] = ORD_NEG_INF;
    }
    __syncwarp();
}

template <class S>
__device__ int queue_top(const S &st, Unit &U) {
    const int G = (U.ns + 31) >> 5;
    if (G <= 8) return queue_top_flat(st, U);
    const int lane = threadIdx.x & 31;
    int best = -1;
    float bk = NEG_INF;
    int M = max_bound(st, G);
    for (int iter = 0; iter < 64; ++iter) {
        if (M == ORD_NEG_INF) {
            warp_best(st, best, bk, U);
            return best;
        }
        const int othr = ord(unord(M) - 2.0f * U.E2);
        int mr = ORD_NEG_INF;  // largest refreshed (exact) bound
        for (int base = 0; base < G; base += 32) {
            const int g = base + lane;
            u32 ball = __ballot_sync(FULL_MASK, g < G && st.gmax[g] >= othr);
            while (ball) {
                const int gg = base + __ffs(ball) - 1;
                ball &= ball - 1;
                const int i = gg * 32 + lane;
                const float k = i < U.ns ? st.key[i] : NEG_INF;
                // the group's exact bound; candidates stay lane-local until the end
                const int o = __reduce_max_sync(FULL_MASK, k == NEG_INF ? ORD_NEG_INF : ord(k));
                if (lane == 0) st.gmax[gg] = o;
                mr = max(mr, o);
                if (k != NEG_INF && (best < 0 || ranks_before(st, i, k, best, bk, U))) {
                    best = i;
                    bk = k;
                }
            }
        }
        __syncwarp();
        // every other bound is below othr <= M, so an unchanged maximum means done
        bool done = mr == M;
        if (!done) {
            const int M2 = max_bound(st, G);
            done = M2 == M;
            M = M2;
        }
        if (done) {
            warp_best(st, best, bk, U);
            return best;
        }
    }
    return queue_top_flat(st, U);
}

// Highest-ranked queued slot that passes the add test at the current K, V.
// A node passes only if 2 d (V + k) > alpha K k (the filter below), so only if
// d / k > alpha K / (2 (V + k_max)): groups whose d/k bound is below that are
// skipped.  (The threshold and the d/k values carry errors of a few 2^-24
// each, the quotients being the fast division within 2 ulp; the 2^-16 margin
// keeps the skip one-sided.)
template <class S>
__device__ int best_passing(const S &st, Unit &U) {
    const int lane = threadIdx.x & 31;
    const int G = (U.ns + 31) >> 5;
    const float tau = U.alpha32 * exact::i2f(U.K) / (2.0f * (exact::i2f(U.V) + U.kmaxf)) * (1.0f - 0x1p-16f);
    const int otau = ord(tau);
    int best = -1;
    float bk = NEG_INF;
    for (int base = 0; base < G; base += 32) {
        const int g = base + lane;
        u32 ball = __ballot_sync(FULL_MASK, g < G && st.qmax[g] >= otau);
        while (ball) {
            const int gg = base + __ffs(ball) - 1;
            ball &= ball - 1;
            const int i = gg * 32 + lane;
            const float k = i < U.ns ? st.key[i] : NEG_INF;
            i64 d = 0, kd = 1;
            if (k != NEG_INF) {
                d = st.din[i];
                kd = st.gk[node_of(st.id[i])];
            }
            // the group's d/k bound made exact again (members and rejected
            // nodes have left the queue since it was last raised)
            const int qo =
                __reduce_max_sync(FULL_MASK, k == NEG_INF ? ORD_NEG_INF
                                                          : ord(__fdividef(exact::i2f(d), exact::i2f(kd))));
            if (lane == 0) st.qmax[gg] = qo;
            if (k == NEG_INF) continue;
            if (!exact::add_possible(U.K, U.V, d, kd, U.alpha32)) continue;
            if (!exact::add_test(U.K, U.V, d, kd, U.alpha, U.alpha32, U.xflags)) continue;
            if (best < 0 || ranks_before(st, i, k, best, bk, U)) {
                best = i;
                bk = k;
            }
        }
    }
    warp_best(st, best, bk, U);
    return best;
}

// Pop (reject) every queued slot ranked before `best`.  Such a slot has a key
// above key(best) - E2, so only groups whose bound reaches key(best) - 2 E2
// are visited; their bounds are recomputed, the others stay upper bounds.
template <class S>
__device__ void drop_before(const S &st, int best, Unit &U) {
    const int lane = threadIdx.x & 31;
    const int G = (U.ns + 31) >> 5;
    const float bk = st.key[best];
    const int othr = ord(bk - 2.0f * U.E2);
    for (int base = 0; base < G; base += 32) {
        const int g = base + lane;
        u32 ball = __ballot_sync(FULL_MASK, g < G && st.gmax[g] >= othr);
        while (ball) {
            const int gg = base + __ffs(ball) - 1;
            ball &= ball - 1;
            const int i = gg * 32 + lane;
            const float k = i < U.ns ? st.key[i] : NEG_INF;
            const bool drop = k != NEG_INF && ranks_before(st, i, k, best, bk, U);
            if (drop) st.key[i] = NEG_INF;
            // the group's key bound made exact again
            const int o = __reduce_max_sync(FULL_MASK, drop ? ORD_NEG_INF : ord(k));
            if (lane == 0) st.gmax[gg] = o;
        }
    }
    __syncwarp();
}

// Scan the row of the node in `slot`, adding sign*w to d_in of every
// neighbour; with requeue, (re)insert outside neighbours in the queue with
// their new key and fold them into their group's best.
// The first 32 entries of a row, loaded ahead by a caller that expects to
// expand it (valid = false: nothing loaded).
struct Chunk {
    i32 v;
    i64 w;
    bool valid;
};

template <bool WEIGHTED>
__device__ __forceinline__ Chunk load_chunk(const DevGraph &G, i64 rs, i64 re) {
    Chunk c;
    const i64 e = rs + (threadIdx.x & 31);
    c.v = 0;
    c.w = 0;
    if (e < re) {
        c.v = G.col[e];
        c.w = WEIGHTED ? G.wfx[e] : 1;
    }
    c.valid = true;
    return c;
}

template <class VT, class HT, bool WEIGHTED>
__device__ void expand(const State<VT, HT, WEIGHTED> &st, const GrowArgs &a, Unit &U, int slot, int sign,
                       bool requeue, i64 rs, i64 re, Chunk c0) {
    const DevGraph &G = a.G;
    const int lane = threadIdx.x & 31;
    if (rs < 0) {  // row bounds not loaded by the caller
        const i32 u = node_of(st.id[slot]);
        rs = G.rp[u];
        re = G.rp[u + 1];
    }
    for (i64 b = rs; b < re; b += 32) {
        const i64 e = b + lane;
        const bool act = e < re;
        i32 v = 0;
        i64 w = 0;
        if (b == rs && c0.valid) {
            v = c0.v;
            w = c0.w;
        } else if (act) {
            v = G.col[e];
            w = WEIGHTED ? G.wfx[e] : 1;
        }
        SlotView<VT> sv;
        const int s = lookup_insert(st, G, U, v, act, &sv);
        if (U.ovf || U.err) return;
        bool upd = false;
        float k = NEG_INF;
        i64 d = 0;
        if (act) {
            d = (i64)sv.din + sign * w;
            st.din[s] = (VT)d;
            if (requeue && !sv.member) {
                k = logf(exact::i2f(d)) - U.alpha32 * sv.logk;  // = rank_key(d, k_v)
                st.key[s] = k;
                upd = true;
            }
        }
        if (upd) {
            atomicMax(&st.gmax[s >> 5], ord(k));
            atomicMax(&st.qmax[s >> 5], ord(__fdividef(exact::i2f(d), exact::i2f(sv.kdeg))));
        }
    }
    __syncwarp();
    if (lane == 0) g_wcnt[threadIdx.x >> 5][0] += (unsigned long long)(re - rs);
}

// Add slot s to the community (an addition of the grow pass, or an initial
// member, which is not counted as one).
// With c0 valid, the caller also passes gkey, this lane's key of the group of
// s as it stands (s included): the group's bound is set to the exact largest
// key left once s leaves the queue, so that the next argmax does not meet a
// stale bound there.
template <class VT, class HT, bool WEIGHTED>
__device__ void accept(const State<VT, HT, WEIGHTED> &st, const GrowArgs &a, Unit &U, int s, i32 u, i64 d, i64 kd,
                       bool counted, i64 rs, i64 re, Chunk c0, float gkey) {
    const int lane = threadIdx.x & 31;
    int o = 0;
    if (c0.valid) o = __reduce_max_sync(FULL_MASK, lane == (s & 31) ? ORD_NEG_INF : ord(gkey));
    __syncwarp();
    if (lane == 0) {
        st.id[s] = u | MEMBER_BIT;
        st.key[s] = NEG_INF;
        st.mem[U.nm] = (HT)s;
        if (c0.valid) st.gmax[s >> 5] = o;
        if (counted) g_wcnt[threadIdx.x >> 5][1] += 1ull;
    }
    __syncwarp();
    U.nm++;
    U.K += 2 * d;
    U.V += kd;
    expand(st, a, U, s, +1, true, rs, re, c0);
}

template <class VT, class HT, bool WEIGHTED>
__device__ __forceinline__ void accept_slot(const State<VT, HT, WEIGHTED> &st, const GrowArgs &a, Unit &U, int s,
                                            bool counted) {
    const i32 u = node_of(st.id[s]);
    Chunk none;
    none.valid = false;
    accept(st, a, U, s, u, (i64)st.din[s], st.gk[u], counted, -1, -1, none, NEG_INF);
}

// Smallest-id member (not the seed, id > last) whose removal raises f; -1 if none.
template <class S>
__device__ int first_removable(const S &st, Unit &U, i32 last) {
    const int lane = threadIdx.x & 31;
    i32 bid = INT32_MAX;
    int bslot = -1;
    for (int j = lane; j < U.nm; j += 32) {
        const int i = st.mem[j];
        const i32 u = node_of(st.id[i]);
        if (u == U.seed || u <= last || u >= bid) continue;
        const i64 d = st.din[i], kd = st.gk[u];
        if (!exact::remove_possible(U.K, U.V, d, kd, U.alpha32)) continue;
        if (!exact::remove_test(U.K, U.V, d, kd, U.alpha, U.alpha32, U.xflags)) continue;
        bid = u;
        bslot = i;
    }
    const i32 m = __reduce_min_sync(FULL_MASK, bid);
    const u32 who = __ballot_sync(FULL_MASK, bid == m && bslot >= 0);
    if (!who) return -1;
    return __shfl_sync(FULL_MASK, bslot, __ffs(who) - 1);
}

template <class VT, class HT, bool WEIGHTED>
__device__ void remove_node(const State<VT, HT, WEIGHTED> &st, const GrowArgs &a, Unit &U, int s) {
    const int lane = threadIdx.x & 31;
    const i32 x = st.id[s];
    const i64 d = st.din[s], kd = st.gk[node_of(x)];
    // drop s from the member list in place, keeping the others' order: a
    // lane writes at or below the entry it read, and each chunk is read in
    // full before it is written
    int w = 0;
    for (int b = 0; b < U.nm; b += 32) {
        const int j = b + lane;
        const int e = j < U.nm ? (int)st.mem[j] : -1;
        const bool keep = j < U.nm && e != s;
        const u32 ball = __ballot_sync(FULL_MASK, keep);
        __syncwarp();
        if (keep) st.mem[w + __popc(ball & lanemask_lt())] = (HT)e;
        w += __popc(ball);
    }
    __syncwarp();
    if (lane == 0) {
        st.id[s] = node_of(x);
        g_wcnt[threadIdx.x >> 5][2] += 1ull;
    }
    __syncwarp();
    U.nm = w;
    U.K -= 2 * d;
    U.V -= kd;
    Chunk none;
    none.valid = false;
    expand(st, a, U, s, -1, false, -1, -1, none);
}

// Empty the hash table for the next unit (only its first U.H buckets were
// used; the table is sized to the unit, so a plain sweep is short).
template <class S>
__device__ void clear_hash(const S &st, const Unit &U) {
    __syncwarp();
    zero_table(st.hsh, U.err ? st.Hmax : U.H);
    __syncwarp();
}

// Sort the members ascending into scratch (the key array viewed as int32[C]),
// hash the list and write it out.  Returns false if the output buffer is full.
template <class S>
__device__ bool emit(const S &st, const GrowArgs &a, Unit &U, i64 unit, int status) {
    const int lane = threadIdx.x & 31;
    i32 *scr = (i32 *)st.key;
    const int m = U.nm;
    __syncwarp();
    for (int j = lane; j < m; j += 32) scr[j] = node_of(st.id[st.mem[j]]);
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
    h &= ~a.hash_clear;
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
            f = exp(log((double)U.K) - U.alpha * log((double)U.V) + (1.0 - U.alpha) * (double)a.G.unit_exp * LN2);
        }
        a.uf[unit] = f;
        i64 *stt = a.ustat + unit * MSCD_NSTATS;
        const unsigned long long *wc = g_wcnt[threadIdx.x >> 5];
        stt[MSCD_STAT_EDGES] = (i64)wc[0];
        stt[MSCD_STAT_ADDS] = (i64)wc[1];
        stt[MSCD_STAT_REMOVES] = (i64)wc[2];
        stt[MSCD_STAT_ROUNDS] = U.rounds;
        stt[MSCD_STAT_K] = U.K;
        stt[MSCD_STAT_V] = U.V;
        stt[MSCD_STAT_SLOW] = (U.xflags & EXACT_SLOW) ? 1 : 0;
        stt[MSCD_STAT_UNDECIDED] = (U.xflags & EXACT_UNDECIDED) ? 1 : 0;
        a.ustatus[unit] = status;
    }
    return true;
}

template <class VT, class HT, bool WEIGHTED>
__device__ void grow_unit(const State<VT, HT, WEIGHTED> &st, const GrowArgs &a, i64 unit) {
    const int lane = threadIdx.x & 31;
    const DevGraph &G = a.G;
    Unit U;
    const i64 si = a.unit_alpha ? unit : unit % a.n_seeds;
    U.alpha = a.unit_alpha ? a.unit_alpha[unit] : a.alphas[unit / a.n_seeds];
    U.alpha32 = (float)U.alpha;
    U.seed = a.seeds ? a.seeds[si] : (i32)si;
    U.E2 = 2.0f * 0x1p-20f * (1.0f + U.alpha32) * (1.0f + a.log_kmax);
    U.kmaxf = (float)G.kmax;
    U.K = 0;
    U.V = G.k[U.seed];
    U.ns = 0;
    U.nm = 0;
    U.H = min(HASH_MIN, st.Hmax);
    U.rounds = 0;
    U.xflags = 0;
    U.ovf = U.err = false;
    if (lane < 3) g_wcnt[threadIdx.x >> 5][lane] = 0ull;
    __syncwarp();
    int status = MSCD_OK;
    if (a.big_seed) {
        // this seed's unit outgrew the class at the previous, finer scale: the
        // coarser scale's will too (almost always), so hand it on unopened
        const i64 sc = unit / a.n_seeds;
        if (sc > 0 && a.alphas[sc - 1] > U.alpha && a.big_seed[si]) {
            if (lane == 0) a.retry_state[atomicAdd(a.n_retry_state, 1ull)] = unit;
            return;
        }
    }

    lookup_insert(st, G, U, U.seed, lane == 0);  // slot 0
    if (lane == 0) {
        st.id[0] = U.seed | MEMBER_BIT;
        st.mem[0] = 0;
    }
    U.nm = 1;
    __syncwarp();
    {
        Chunk none;
        none.valid = false;
        expand(st, a, U, 0, +1, false, -1, -1, none);
    }
    if (a.init_ptr) {
        // initial members (Alg. 2 may start from given communities); repeats
        // and the seed itself are skipped
        for (i64 j = a.init_ptr[si]; j < a.init_ptr[si + 1] && !U.ovf && !U.err; ++j) {
            int s = lookup_insert(st, G, U, a.init_nodes[j], lane == 0);
            if (U.ovf || U.err) break;
            s = __shfl_sync(FULL_MASK, s, 0);
            if (st.id[s] < 0) continue;  // already a member
            accept_slot(st, a, U, s, false);
        }
    }

    while (!U.ovf && !U.err) {
        if (U.rounds >= a.max_rounds) {
            status = MSCD_ETIMEOUT;
            break;
        }
        U.rounds++;
        build_queue(st, U);
        i64 added = 0;
        for (;;) {
            const int top = queue_top(st, U);
            if (top < 0) break;
            const i32 utop = node_of(st.id[top]);
            const i64 dtop = (i64)st.din[top];
            const i64 rs = G.rp[utop], re = G.rp[utop + 1];
            const i64 ktop = st.gk[utop];
            // loaded during the test, for the likely addition: the first entries
            // of its row and the keys of its group
            const int gi = (top & ~31) + lane;
            const float gkey = gi < U.ns ? st.key[gi] : NEG_INF;
            const Chunk c0 = load_chunk<WEIGHTED>(G, rs, re);
            if (exact::add_test(U.K, U.V, dtop, ktop, U.alpha, U.alpha32, U.xflags)) {
                accept(st, a, U, top, utop, dtop, ktop, true, rs, re, c0, gkey);
            } else {
                const int s = best_passing(st, U);
                // none passes: every queued node is popped and rejected, the grow
                // pass ends (the next round rebuilds every key)
                if (s < 0) break;
                drop_before(st, s, U);
                accept_slot(st, a, U, s, true);
            }
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
                last = node_of(st.id[s]);
                remove_node(st, a, U, s);
                removed++;
                if (U.ovf || U.err) break;
            }
            if (removed == 0 || U.ovf || U.err) break;
        }
        if (a.single_round) break;
    }
    U.xflags = __reduce_or_sync(FULL_MASK, U.xflags);
    if (U.err) {
        if (lane == 0) atomicOr(a.error_flags, 1u);
    } else if (U.ovf) {
        if (lane == 0) {
            a.retry_state[atomicAdd(a.n_retry_state, 1ull)] = unit;
            if (a.big_seed) a.big_seed[si] = 1;
        }
    } else {
        if (status == MSCD_OK && (U.xflags & EXACT_UNDECIDED)) status = MSCD_EUNDECIDED;
        if (!emit(st, a, U, unit, status)) {
            if (lane == 0) a.retry_out[atomicAdd(a.n_retry_out, 1ull)] = unit;
        }
    }
    clear_hash(st, U);
}

// One unit per warp, persistent: units are taken from a global counter until
// the work list is exhausted (or, in the plain form, one statically mapped
// unit per warp).  State: dynamic shared memory (warp w of the
// CTA at w * state_bytes) or the global arena (warp at its global index).
template <class VT, class HT, bool WEIGHTED, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) grow_kernel(GrowArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const i64 gw = (i64)blockIdx.x * (blockDim.x >> 5) + wib;
    unsigned char *base = a.use_smem ? smem + (size_t)wib * a.state_bytes : a.gstate + (size_t)gw * a.state_bytes;
    // global-arena classes: group bounds and hash table of the warp in shared memory if asked
    unsigned char *wsm = smem + (size_t)wib * a.smem_per_warp;
    int *bounds = a.bounds_smem ? (int *)wsm : nullptr;
    HT *hsh = a.hash_smem ? (HT *)(wsm + (a.bounds_smem ? 8 * (size_t)(a.cap / 32) : 0)) : nullptr;
    const State<VT, HT, WEIGHTED> st = carve<VT, HT, WEIGHTED>(base, a.cap, bounds, hsh, a.G.k);
    zero_table(st.hsh, st.Hmax);
    __syncwarp();
    // one call site of grow_unit, and nothing of the plain form live across it
    // (a second inlined copy, or a flag, costs registers)
    for (;;) {
        unsigned long long t = 0;
        if (a.plain) {
            t = (unsigned long long)(a.work_base + (i64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
        } else {
            if (lane == 0) t = atomicAdd(a.work_counter, 1ull);
            t = __shfl_sync(FULL_MASK, t, 0);
        }
        if ((i64)t >= a.n_work) break;
        const i64 unit = a.work_list ? a.work_list[t] : a.unit_base + (i64)t;
        grow_unit(st, a, unit);
        if (a.plain) break;
    }
}

template <class VT, class HT, bool WEIGHTED, int MAXT, int MINB>
int launch_k(const GrowArgs &a, int blocks, int threads, size_t smem, cudaStream_t st, int *occ) {
    auto k = grow_kernel<VT, HT, WEIGHTED, MAXT, MINB>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_status(e);
    }
    if (occ) return cuda_status(cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, threads, smem));
    k<<<blocks, threads, smem, st>>>(a);
    note_launch();
    return cuda_status(cudaGetLastError());
}

// Shared-memory classes: CTAs of up to 16 one-warp units (shared memory
// bounds the count).  Global-arena classes: CTAs of GLOBAL_CTA_THREADS with
// registers capped so that GLOBAL_MIN_BLOCKS of them fit an SM.
#ifndef GLOBAL_MIN_BLOCKS
#define GLOBAL_MIN_BLOCKS 2
#endif
template <class VT, class HT, bool WEIGHTED>
int launch_t(const GrowArgs &a, int blocks, int threads, size_t smem, cudaStream_t st, int *occ) {
    if (a.use_smem || a.hash_smem) return launch_k<VT, HT, WEIGHTED, GROW_MAX_THREADS, 1>(a, blocks, threads, smem, st, occ);
    return launch_k<VT, HT, WEIGHTED, GLOBAL_CTA_THREADS, GLOBAL_MIN_BLOCKS>(a, blocks, threads, smem, st, occ);
}

typedef unsigned short u16;

// Dispatch on the slot value type (16-bit when every degree fits, else 32 /
// 64-bit) and the bucket type (16-bit up to 32768 slots).
int dispatch(const GrowArgs &a, int blocks, int threads, size_t smem, cudaStream_t st, int *occ) {
    const bool w = a.G.wfx != nullptr;
    const bool small_deg = !w && a.G.kmax < 65536;
    const bool h16 = a.cap <= 32768;
    if (w) return h16 ? launch_t<i64, u16, true>(a, blocks, threads, smem, st, occ)
                      : launch_t<i64, u32, true>(a, blocks, threads, smem, st, occ);
    if (small_deg) return h16 ? launch_t<u16, u16, false>(a, blocks, threads, smem, st, occ)
                              : launch_t<u16, u32, false>(a, blocks, threads, smem, st, occ);
    return h16 ? launch_t<i32, u16, false>(a, blocks, threads, smem, st, occ)
               : launch_t<i32, u32, false>(a, blocks, threads, smem, st, occ);
}

}  // namespace

size_t grow_state_bytes(const DevGraph &G, int cap) {
    const bool w = G.wfx != nullptr;
    const bool h16 = cap <= 32768;
    if (w) return h16 ? state_bytes_t<i64, u16, true>(cap) : state_bytes_t<i64, u32, true>(cap);
    if (G.kmax < 65536)
        return h16 ? state_bytes_t<u16, u16, false>(cap) : state_bytes_t<u16, u32, false>(cap);
    return h16 ? state_bytes_t<i32, u16, false>(cap) : state_bytes_t<i32, u32, false>(cap);
}

int grow_launch(const GrowArgs &a, int blocks, int threads, size_t smem, cudaStream_t st) {
    return dispatch(a, blocks, threads, smem, st, nullptr);
}

int grow_occupancy(const GrowArgs &a, int threads, size_t smem, int *blocks_per_sm) {
    return dispatch(a, 0, threads, smem, nullptr, blocks_per_sm);
}
