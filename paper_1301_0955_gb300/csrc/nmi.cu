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
// Shortcut: when X_k has an identical partner Y_l (equal sorted lists), the
// candidate of that pair is exactly 0 (H(X_k, Y_l) = H(Y_l)), and no
// candidate is negative, so H(X_k|Y) = 0 without counting; likewise for Y_l.
// Successive scales share most communities, so most of the work goes.
//
// For the other communities, only two kinds of partner can be admitted:
//   * partners that share a node;
//   * disjoint partners with |A| + |B| > n/2.  For a disjoint pair with
//     s = (|A| + |B|)/n <= 1/2: h(P00) = h(1-s) <= h(s) (h(1-s) <= h(s)
//     on [0, 1/2]) <= h(P10) + h(P01) (h concave with h(0) = 0 is
//     subadditive), and h(P11) = 0, so the admission test fails.
//     Either side of such a pair may be the small one, so the partners
//     listed for this test are the B communities with 2(|B| + a) > n, a the
//     largest active A community of the part; each A community walks its
//     part's list in descending size and stops at the first B too small.
// The intersections of the sharing pairs are counted by a warp per community:
// it walks its members' lists of partner communities (the lanes spread over
// one list at a time, whose entries are distinct) and counts in a
// shared-memory hash; a community that meets too many partners is redone by
// a whole CTA with a larger shared-memory table, and beyond that with a
// global-memory table of its own.  Minima are kept as the bits of
// non-negative doubles; the per-community terms are summed exactly (each
// rounded once to a multiple of 2^-62, added in 128-bit integers), so the
// value does not depend on the order of the additions.
//
// A graph that is a disjoint union of parts (independent graphs batched as
// one) gets one NMI per part: a community lies inside one part (growth never
// leaves the seed's component), n above is its part's node count, partners
// are only ever taken from the same part, and the means run over each part's
// communities.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "dedup.cuh"

int ctx_device_of(mscd_ctx *c);

namespace {

constexpr int NMI_WARPS = 8;
constexpr int NMI_TABLE = 512;  // shared-memory hash entries per warp (6 CTAs of 8 warps per SM)

__device__ __forceinline__ double hterm(i64 c, double inv_n) {
    if (c <= 0) return 0.0;
    const double p = (double)c * inv_n;
    return -p * log2(p);
}

// Candidate H(A|B) for two communities of sizes sa, sb sharing n11 nodes, if
// admitted; else +inf.
__device__ __forceinline__ double cond_candidate(i64 n11, i64 sa, i64 sb, i64 n, double inv_n) {
    const i64 n10 = sa - n11, n01 = sb - n11, n00 = n - n11 - n10 - n01;
    const i64 lo1 = min(n11, n00), hi1 = max(n11, n00), lo2 = min(n01, n10), hi2 = max(n01, n10);
    if (lo1 == lo2 && hi1 == hi2) return __builtin_huge_val();
    const double h11 = hterm(n11, inv_n), h00 = hterm(n00, inv_n), h01 = hterm(n01, inv_n), h10 = hterm(n10, inv_n);
    if (!(h11 + h00 > h01 + h10)) return __builtin_huge_val();
    return (h11 + h10 + h01 + h00) - (hterm(sb, inv_n) + hterm(n - sb, inv_n));
}

__device__ __forceinline__ double entropy(i64 s, i64 n, double inv_n) { return hterm(s, inv_n) + hterm(n - s, inv_n); }

__device__ __forceinline__ unsigned long long min_bits(double v) {
    return (unsigned long long)__double_as_longlong(v > 0.0 ? v : 0.0);
}

__global__ void count_memberships(const i32 *nodes, i64 m, i32 *cnt) {
    for (i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (i64)gridDim.x * blockDim.x)
        atomicAdd(&cnt[nodes[e]], 1);
}

__global__ void widen_i32(const i32 *a, i64 n, i64 *b) {
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) b[i] = a[i];
}

// Warp per community l: append l to the list of each member.
__global__ void fill_memberships(const i64 *cptr, const i32 *nodes, i64 C, const i64 *mptr, i32 *cursor, i32 *mlist) {
    const int lane = threadIdx.x & 31;
    const i64 warps = (i64)gridDim.x * (blockDim.x >> 5);
    for (i64 l = (i64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); l < C; l += warps)
        for (i64 e = cptr[l] + lane; e < cptr[l + 1]; e += 32) {
            const i32 u = nodes[e];
            mlist[mptr[u] + atomicAdd(&cursor[u], 1)] = (i32)l;
        }
}

// Hash table of community list hashes (0 = empty bucket; list hashes are never 0).
__global__ void hash_insert(const u64 *chash, i64 C, u64 *tkey, i32 *tval, i64 tmask) {
    for (i64 l = (i64)blockIdx.x * blockDim.x + threadIdx.x; l < C; l += (i64)gridDim.x * blockDim.x) {
        i64 h = (i64)(chash[l] & (u64)tmask);
        for (i64 p = 0; p <= tmask; ++p) {
            if (atomicCAS((unsigned long long *)&tkey[h], 0ull, (unsigned long long)chash[l]) == 0ull) {
                tval[h] = (i32)l;
                break;
            }
            h = (h + 1) & tmask;
        }
    }
}

// Warp per X_k: an identical Y_l (same hash, same list) zeroes both.
__global__ void match_identical(const i64 *xptr, const i32 *xnodes, const u64 *xhash, i64 CX, const i64 *yptr,
                                const i32 *ynodes, const u64 *tkey, const i32 *tval, i64 tmask,
                                unsigned char *zeroX, unsigned char *zeroY) {
    const int lane = threadIdx.x & 31;
    const i64 warps = (i64)gridDim.x * (blockDim.x >> 5);
    for (i64 k = (i64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); k < CX; k += warps) {
        const u64 key = xhash[k];
        const i64 sx = xptr[k + 1] - xptr[k];
        i64 h = (i64)(key & (u64)tmask);
        for (i64 p = 0; p <= tmask; ++p) {
            const u64 tk = tkey[h];
            if (tk == 0ull) break;
            if (tk == key) {
                const i32 l = tval[h];
                bool eq = yptr[l + 1] - yptr[l] == sx;
                if (eq) {
                    const i32 *a = xnodes + xptr[k], *b = ynodes + yptr[l];
                    bool diff = false;
                    for (i64 i = lane; i < sx; i += 32) diff |= a[i] != b[i];
                    eq = !__any_sync(FULL_MASK, diff);
                }
                if (eq) {
                    if (lane == 0) {
                        zeroX[k] = 1;
                        zeroY[l] = 1;
                    }
                    break;
                }
            }
            h = (h + 1) & tmask;
        }
    }
}

// Part of every community (that of its first member; a community never spans
// parts) and that part's node count.  No offsets: one part of n nodes.
__global__ void comm_parts(const i64 *ptr, const i32 *nodes, i64 C, const i64 *off, i32 n_parts, i64 n, i32 *cp,
                           i64 *cn) {
    for (i64 l = (i64)blockIdx.x * blockDim.x + threadIdx.x; l < C; l += (i64)gridDim.x * blockDim.x) {
        if (!off) {
            cp[l] = 0;
            cn[l] = n;
            continue;
        }
        const i64 u = nodes[ptr[l]];
        i32 lo = 0, hi = n_parts - 1;  // last part with off[p] <= u
        while (lo < hi) {
            const i32 mid = (lo + hi + 1) >> 1;
            if (off[mid] <= u) lo = mid;
            else hi = mid - 1;
        }
        cp[l] = lo;
        cn[l] = off[lo + 1] - off[lo];
    }
}

// Initial minima: 0 for communities with an identical partner, else H(C)
// (the value when no partner is admitted); list the others.
__global__ void init_best(const i64 *ptr, i64 C, const i64 *cn, const unsigned char *zero, unsigned long long *best,
                          i32 *active, unsigned long long *n_active) {
    for (i64 l = (i64)blockIdx.x * blockDim.x + threadIdx.x; l < C; l += (i64)gridDim.x * blockDim.x) {
        if (zero[l]) {
            best[l] = 0ull;
        } else {
            best[l] = min_bits(entropy(ptr[l + 1] - ptr[l], cn[l], 1.0 / (double)cn[l]));
            active[atomicAdd(n_active, 1ull)] = (i32)l;
        }
    }
}

__device__ __forceinline__ u32 hash_comm(i32 l) { return (u32)l * 0x9E3779B1u; }

struct DirArgs {
    const i64 *aptr;
    const i32 *anodes;
    const i32 *active;  // communities of A to process
    i64 n_active;
    const i64 *bptr;
    const i64 *mptr;    // node -> communities of B
    const i32 *mlist;
    const i64 *acn;            // per A community: node count of its part
    unsigned long long *best;  // per A community (bits of doubles)
    i64 *spill;                // positions in `active` redone with global tables
    unsigned long long *n_spill;
    const i64 *toff;
    i32 *tkey, *tcnt;
    i32 *tused;           // buckets each global table claimed, at the table's offset
    unsigned int *tfill;  // per community of a chunk: buckets claimed
    // work counter of the launch (zeroed before it): communities are taken
    // one at a time as warps or CTAs free up, since their costs differ by
    // orders of magnitude
    unsigned long long *next;
};

// Warp per active A community: intersections with every B community it meets
// (shared-memory hash), minimum admitted candidate.
// The buckets a community fills are listed as they are claimed, so the scan
// and the reset after it touch only those (the table is cleared once).
__global__ void __launch_bounds__(NMI_WARPS * 32) pairs_smem(DirArgs a) {
    __shared__ i32 skey[NMI_WARPS][NMI_TABLE];
    __shared__ i32 scnt[NMI_WARPS][NMI_TABLE];
    __shared__ unsigned short sused[NMI_WARPS][NMI_TABLE / 2];
    __shared__ int sfill[NMI_WARPS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    i32 *keys = skey[w];
    i32 *cnts = scnt[w];
    unsigned short *used = sused[w];
    for (int t = lane; t < NMI_TABLE; t += 32) {
        keys[t] = -1;
        cnts[t] = 0;
    }
    __syncwarp();
    for (;;) {
        unsigned long long qq = 0;
        if (lane == 0) qq = atomicAdd(a.next, 1ull);
        const i64 q = (i64)__shfl_sync(FULL_MASK, qq, 0);
        if (q >= a.n_active) break;
        const i32 k = a.active[q];
        if (lane == 0) sfill[w] = 0;
        __syncwarp();
        bool over = false;
        for (i64 e = a.aptr[k]; e < a.aptr[k + 1] && !over; ++e) {
            const i32 u = a.anodes[e];
            for (i64 j = a.mptr[u] + lane; j < a.mptr[u + 1]; j += 32) {
                const i32 l = a.mlist[j];
                u32 h = hash_comm(l) & (NMI_TABLE - 1);
                for (int p = 0; p < NMI_TABLE; ++p) {
                    i32 cur = keys[h];
                    if (cur == -1) {
                        cur = atomicCAS(&keys[h], -1, l);
                        if (cur == -1) {
                            const int f = atomicAdd(&sfill[w], 1);
                            if (f >= NMI_TABLE / 2) over = true;
                            else used[f] = (unsigned short)h;
                            cur = l;
                        }
                    }
                    if (cur == l) {
                        atomicAdd(&cnts[h], 1);
                        break;
                    }
                    h = (h + 1u) & (NMI_TABLE - 1);
                }
            }
            over = __any_sync(FULL_MASK, over);
        }
        __syncwarp();
        if (over) {
            if (lane == 0) a.spill[atomicAdd(a.n_spill, 1ull)] = q;
            for (int t = lane; t < NMI_TABLE; t += 32) {  // more buckets than listed: clear all
                keys[t] = -1;
                cnts[t] = 0;
            }
            __syncwarp();
            continue;
        }
        const int nf = sfill[w];
        const i64 sa = a.aptr[k + 1] - a.aptr[k], n = a.acn[k];
        const double inv_n = 1.0 / (double)n;
        double bx = __longlong_as_double((long long)a.best[k]);
        for (int t = lane; t < nf; t += 32) {
            const int h = used[t];
            const i32 l = keys[h];
            bx = min(bx, cond_candidate(cnts[h], sa, a.bptr[l + 1] - a.bptr[l], n, inv_n));
            keys[h] = -1;
            cnts[h] = 0;
        }
        for (int o = 16; o; o >>= 1) bx = min(bx, __shfl_xor_sync(FULL_MASK, bx, o));
        if (lane == 0) a.best[k] = min_bits(bx);
        __syncwarp();
    }
}

// CTA per listed community (positions in `active`): the same with a global
// table of its own, the community's members spread over the CTA's warps (these
// communities meet thousands of partners through millions of incidences).
constexpr int GLB_WARPS = 16;

__global__ void __launch_bounds__(GLB_WARPS * 32) pairs_global(DirArgs a, const i64 *list, i64 nk) {
    __shared__ double wmin[GLB_WARPS];
    __shared__ i64 rnext;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) rnext = (i64)atomicAdd(a.next, 1ull);
        __syncthreads();
        const i64 r = rnext;
        if (r >= nk) break;
        const i32 k = a.active[list[r]];
        i32 *keys = a.tkey + a.toff[r];
        i32 *cnts = a.tcnt + a.toff[r];
        i32 *used = a.tused + a.toff[r];
        unsigned int *fill = a.tfill + r;
        const u32 tm = (u32)(a.toff[r + 1] - a.toff[r] - 1);
        for (i64 e = a.aptr[k] + w; e < a.aptr[k + 1]; e += GLB_WARPS) {
            const i32 u = a.anodes[e];
            for (i64 j = a.mptr[u] + lane; j < a.mptr[u + 1]; j += 32) {
                const i32 l = a.mlist[j];
                u32 h = hash_comm(l) & tm;
                for (u32 p = 0; p <= tm; ++p) {
                    i32 cur = keys[h];
                    if (cur == -1) {
                        cur = atomicCAS(&keys[h], -1, l);
                        if (cur == -1) {
                            used[atomicAdd(fill, 1u)] = (i32)h;
                            cur = l;
                        }
                    }
                    if (cur == l) {
                        atomicAdd(&cnts[h], 1);
                        break;
                    }
                    h = (h + 1u) & tm;
                }
            }
        }
        __syncthreads();
        const i64 sa = a.aptr[k + 1] - a.aptr[k], n = a.acn[k];
        const double inv_n = 1.0 / (double)n;
        double bx = __builtin_huge_val();
        // only the claimed buckets, emptied again for the table's next user
        const u32 nf = *(volatile unsigned int *)fill;
        for (u32 t = threadIdx.x; t < nf; t += GLB_WARPS * 32) {
            const i32 hh = used[t];
            const i32 l = keys[hh];
            bx = min(bx, cond_candidate(cnts[hh], sa, a.bptr[l + 1] - a.bptr[l], n, inv_n));
            keys[hh] = -1;
            cnts[hh] = 0;
        }
        for (int o = 16; o; o >>= 1) bx = min(bx, __shfl_xor_sync(FULL_MASK, bx, o));
        if (lane == 0) wmin[w] = bx;
        __syncthreads();
        if (threadIdx.x == 0) {
            double m = __longlong_as_double((long long)a.best[k]);
            for (int q = 0; q < GLB_WARPS; ++q) m = min(m, wmin[q]);
            a.best[k] = min_bits(m);
        }
        __syncthreads();
    }
}

constexpr int BLK_WARPS = 16;
constexpr int BLK_TABLE = 8192;  // shared-memory hash entries of one CTA (72 KB: 3 CTAs per SM)

// CTA per community spilled by pairs_smem: its members are spread over the
// warps, an 8192-entry shared-memory table counts the intersections; a
// community meeting more than half of that is listed for pairs_global.
__global__ void __launch_bounds__(BLK_WARPS * 32) pairs_block(DirArgs a, const i64 *list, i64 nk, i64 *spill2,
                                                              unsigned long long *n_spill2) {
    extern __shared__ i32 tab[];
    i32 *keys = tab, *cnts = tab + BLK_TABLE;
    unsigned short *used = (unsigned short *)(tab + 2 * BLK_TABLE);  // [BLK_TABLE / 2]
    __shared__ int fill, over;
    __shared__ double wmin[BLK_WARPS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __shared__ i64 rnext;
    for (int t = threadIdx.x; t < BLK_TABLE; t += BLK_WARPS * 32) {
        keys[t] = -1;
        cnts[t] = 0;
    }
    for (;;) {
        if (threadIdx.x == 0) rnext = (i64)atomicAdd(a.next, 1ull);
        __syncthreads();
        const i64 r = rnext;
        if (r >= nk) break;
        const i64 q = list[r];
        const i32 k = a.active[q];
        if (threadIdx.x == 0) {
            fill = 0;
            over = 0;
        }
        __syncthreads();
        for (i64 e = a.aptr[k] + w; e < a.aptr[k + 1]; e += BLK_WARPS) {
            if (*(volatile int *)&over) break;
            const i32 u = a.anodes[e];
            for (i64 j = a.mptr[u] + lane; j < a.mptr[u + 1]; j += 32) {
                const i32 l = a.mlist[j];
                u32 h = hash_comm(l) & (BLK_TABLE - 1);
                for (int p = 0; p < BLK_TABLE; ++p) {
                    i32 cur = keys[h];
                    if (cur == -1) {
                        cur = atomicCAS(&keys[h], -1, l);
                        if (cur == -1) {
                            const int f = atomicAdd(&fill, 1);
                            if (f >= BLK_TABLE / 2) over = 1;
                            else used[f] = (unsigned short)h;
                            cur = l;
                        }
                    }
                    if (cur == l) {
                        atomicAdd(&cnts[h], 1);
                        break;
                    }
                    h = (h + 1u) & (BLK_TABLE - 1);
                }
            }
        }
        __syncthreads();
        if (over) {
            if (threadIdx.x == 0) spill2[atomicAdd(n_spill2, 1ull)] = q;
            for (int t = threadIdx.x; t < BLK_TABLE; t += BLK_WARPS * 32) {  // clear all
                keys[t] = -1;
                cnts[t] = 0;
            }
            __syncthreads();
            continue;
        }
        const int nf = fill;
        const i64 sa = a.aptr[k + 1] - a.aptr[k], n = a.acn[k];
        const double inv_n = 1.0 / (double)n;
        double bx = __builtin_huge_val();
        for (int t = threadIdx.x; t < nf; t += BLK_WARPS * 32) {
            const int h = used[t];
            const i32 l = keys[h];
            bx = min(bx, cond_candidate(cnts[h], sa, a.bptr[l + 1] - a.bptr[l], n, inv_n));
            keys[h] = -1;
            cnts[h] = 0;
        }
        for (int o = 16; o; o >>= 1) bx = min(bx, __shfl_xor_sync(FULL_MASK, bx, o));
        if (lane == 0) wmin[w] = bx;
        __syncthreads();
        if (threadIdx.x == 0) {
            double m = __longlong_as_double((long long)a.best[k]);
            for (int i = 0; i < BLK_WARPS; ++i) m = min(m, wmin[i]);
            a.best[k] = min_bits(m);
        }
        __syncthreads();
    }
}

// Table size of each spilled community: 2 * min(incidences, |B|) rounded up
// to a power of two.
__global__ void spill_sizes(const i64 *list, i64 nk, const i32 *active, const i64 *aptr, const i32 *anodes,
                            const i32 *bcnt, i64 CB, i64 *tsz) {
    const int lane = threadIdx.x & 31;
    const i64 warps = (i64)gridDim.x * (blockDim.x >> 5);
    for (i64 r = (i64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < nk; r += warps) {
        const i32 k = active[list[r]];
        i64 s = 0;
        for (i64 e = aptr[k] + lane; e < aptr[k + 1]; e += 32) s += bcnt[anodes[e]];
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(FULL_MASK, s, o);
        s = min(s, CB);
        i64 t = 2;
        while (t < 2 * s) t <<= 1;
        if (lane == 0) tsz[r] = t;
    }
}

// Disjoint pairs that can be admitted (|A| + |B| > n/2).
// The candidate B communities grouped by part (boff: offsets per part) and
// in descending size inside a part, so that an A community meets only those
// of its own part and stops at the first one with 2(|A| + |B|) <= n: warp
// per active A, lanes over its part's list.
__global__ void disjoint_pairs(const i64 *aptr, const i32 *anodes, const i32 *active, i64 n_active,
                               const i64 *bptr, const i32 *bnodes, const i32 *big, const i64 *boff,
                               const i32 *acp, const i64 *acn, unsigned long long *best) {
    const int lane = threadIdx.x & 31;
    const i64 warps = (i64)gridDim.x * (blockDim.x >> 5);
    for (i64 q = (i64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < n_active; q += warps) {
        const i32 k = active[q];
        const i32 p = acp[k];
        const i64 sa = aptr[k + 1] - aptr[k], n = acn[k];
        double bx = __builtin_huge_val();
        for (i64 j = boff[p] + lane; j < boff[p + 1]; j += 32) {
            const i32 l = big[j];
            const i64 sb = bptr[l + 1] - bptr[l];
            if (2 * (sa + sb) <= n) break;  // every later entry of this lane is smaller
            const i32 *x = anodes + aptr[k], *y = bnodes + bptr[l];
            i64 i = 0, jj = 0;
            bool meet = false;
            while (i < sa && jj < sb) {
                if (x[i] < y[jj]) ++i;
                else if (x[i] > y[jj]) ++jj;
                else {
                    meet = true;
                    break;
                }
            }
            if (!meet) bx = min(bx, cond_candidate(0, sa, sb, n, 1.0 / (double)n));
        }
        for (int o = 16; o; o >>= 1) bx = min(bx, __shfl_xor_sync(FULL_MASK, bx, o));
        if (lane == 0 && bx < __builtin_huge_val()) atomicMin(&best[k], min_bits(bx));
    }
}

__global__ void gather_parts(const i32 *big, i64 nbig, const i32 *cp, const i64 *ptr, i32 *out, i64 *size) {
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < nbig; i += (i64)gridDim.x * blockDim.x) {
        out[i] = cp[big[i]];
        size[i] = ptr[big[i] + 1] - ptr[big[i]];
    }
}

// Largest active A community of every part.
__global__ void active_max_size(const i64 *aptr, const i32 *active, i64 n_active, const i32 *acp,
                                unsigned long long *amax) {
    for (i64 q = (i64)blockIdx.x * blockDim.x + threadIdx.x; q < n_active; q += (i64)gridDim.x * blockDim.x) {
        const i32 k = active[q];
        atomicMax(&amax[acp[k]], (unsigned long long)(aptr[k + 1] - aptr[k]));
    }
}

// B communities with 2(|B| + a) > n (n of B's part, a the largest active A
// community of that part): the only ones that can meet an active A community
// of their part in an admitted disjoint pair.
__global__ void list_big(const i64 *ptr, i64 C, const i32 *cp, const i64 *cn, const unsigned long long *amax,
                         i32 *big, unsigned long long *nbig) {
    for (i64 l = (i64)blockIdx.x * blockDim.x + threadIdx.x; l < C; l += (i64)gridDim.x * blockDim.x) {
        const i64 a = (i64)amax[cp[l]];
        if (a > 0 && 2 * (ptr[l + 1] - ptr[l] + a) > cn[l]) big[atomicAdd(nbig, 1ull)] = (i32)l;
    }
}

// Normalised term H(A_k|B) / H(A_k) in [0, 1] (the minimum never exceeds its
// initial value H(A_k), computed the same way), added to its part's total as
// an integer multiple of 2^-62 in 128 bits: acc[2p] low word, acc[2p+1] carries.
__global__ void normalise_sum(const i64 *ptr, i64 C, const i64 *cn, const i32 *cp,
                              const unsigned long long *best, unsigned long long *acc,
                              unsigned long long *count) {
    for (i64 k = (i64)blockIdx.x * blockDim.x + threadIdx.x; k < C; k += (i64)gridDim.x * blockDim.x) {
        const i64 n = cn[k];
        const double H = entropy(ptr[k + 1] - ptr[k], n, 1.0 / (double)n);
        const double t = H > 0.0 ? __longlong_as_double((long long)best[k]) / H : 0.0;
        const unsigned long long q = (unsigned long long)__double2ll_rn(fmin(fmax(t, 0.0), 1.0) * 0x1p62);
        const i32 p = cp[k];
        const unsigned long long old = atomicAdd(&acc[2 * p], q);
        if (old + q < old) atomicAdd(&acc[2 * p + 1], 1ull);
        atomicAdd(&count[p], 1ull);
    }
}

template <class T>
int dev_alloc(T **p, i64 count, cudaStream_t st) {
    return cuda_status(cudaMallocAsync((void **)p, (size_t)std::max<i64>(count, 1) * sizeof(T), st));
}

const unsigned GB = 152 * 16;

// node -> communities map of B.
struct Memberships {
    i32 *cnt = nullptr, *list = nullptr;
    i64 *ptr = nullptr;
};

int build_memberships(const ScaleResult &B, i64 n, Memberships *M, cudaStream_t st) {
    i32 *cursor = nullptr;
    i64 *tmp = nullptr;
    int rc = MSCD_OK;
    do {
        if ((rc = dev_alloc(&M->cnt, n, st))) break;
        if ((rc = dev_alloc(&M->ptr, n + 1, st))) break;
        if ((rc = dev_alloc(&M->list, B.n_nodes, st))) break;
        if ((rc = dev_alloc(&cursor, n, st))) break;
        if ((rc = dev_alloc(&tmp, n + 1, st))) break;
        if ((rc = cuda_status(cudaMemsetAsync(M->cnt, 0, n * sizeof(i32), st)))) break;
        if ((rc = cuda_status(cudaMemsetAsync(cursor, 0, n * sizeof(i32), st)))) break;
        count_memberships<<<GB, 256, 0, st>>>(B.comm_nodes, B.n_nodes, M->cnt); note_launch();
        widen_i32<<<GB, 256, 0, st>>>(M->cnt, n, tmp); note_launch();
        if ((rc = scan_exclusive_i64(tmp, M->ptr, n, M->ptr + n, st))) break;
        fill_memberships<<<GB, 256, 0, st>>>(B.comm_ptr, B.comm_nodes, B.n_comms, M->ptr, cursor, M->list); note_launch();
    } while (0);
    cudaFreeAsync(cursor, st);
    cudaFreeAsync(tmp, st);
    return rc;
}

void free_memberships(Memberships *M, cudaStream_t st) {
    cudaFreeAsync(M->cnt, st);
    cudaFreeAsync(M->ptr, st);
    cudaFreeAsync(M->list, st);
}

// Minimum admitted H(A_k|B) for every active A_k into best[] (one direction).
// Per-community part data of one scale's communities.
struct CommParts {
    i32 *cp = nullptr;  // part index
    i64 *cn = nullptr;  // node count of that part
};

int one_direction(const ScaleResult &A, const ScaleResult &B, const Memberships &MB, const CommParts &PA,
                  const CommParts &PB, int32_t P, const i32 *active, i64 n_active, unsigned long long *best,
                  cudaStream_t st) {
    i64 *spill = nullptr, *spill2 = nullptr, *tsz = nullptr, *toff = nullptr, *dboff = nullptr, *bsize = nullptr;
    i32 *bpart = nullptr;
    i32 *tkey = nullptr, *tcnt = nullptr, *tused = nullptr, *big = nullptr;
    unsigned int *tfill = nullptr;
    unsigned long long *cnt = nullptr, *amax = nullptr;
    int rc = MSCD_OK;
    do {
        if (n_active == 0) break;
        if ((rc = dev_alloc(&spill, n_active, st))) break;
        // spills, big-B count, spills of the block tier, then the launches' work counters
        if ((rc = dev_alloc(&cnt, 6, st))) break;
        if ((rc = dev_alloc(&big, B.n_comms, st))) break;
        if ((rc = dev_alloc(&amax, P, st))) break;
        if ((rc = cuda_status(cudaMemsetAsync(cnt, 0, 6 * sizeof(unsigned long long), st)))) break;
        if ((rc = cuda_status(cudaMemsetAsync(amax, 0, (size_t)P * sizeof(unsigned long long), st)))) break;
        DirArgs a{};
        a.aptr = A.comm_ptr;
        a.anodes = A.comm_nodes;
        a.active = active;
        a.n_active = n_active;
        a.bptr = B.comm_ptr;
        a.mptr = MB.ptr;
        a.mlist = MB.list;
        a.acn = PA.cn;
        a.best = best;
        a.spill = spill;
        a.n_spill = cnt;
        a.next = cnt + 3;
        pairs_smem<<<(unsigned)std::min<i64>((n_active + NMI_WARPS - 1) / NMI_WARPS, 152 * 6), NMI_WARPS * 32, 0,
                     st>>>(a); note_launch();
        active_max_size<<<GB, 256, 0, st>>>(A.comm_ptr, active, n_active, PA.cp, amax); note_launch();
        list_big<<<GB, 256, 0, st>>>(B.comm_ptr, B.n_comms, PB.cp, PB.cn, amax, big, cnt + 1); note_launch();
        unsigned long long h[2] = {0, 0};
        if ((rc = cuda_status(cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, st)))) break;
        if ((rc = cuda_status(cudaStreamSynchronize(st)))) break;
        i64 nk = (i64)h[0];
        const i64 *list = spill;
        if (nk > 0) {
            // middle tier: one community per CTA with a large shared-memory table
            if ((rc = dev_alloc(&spill2, nk, st))) break;
            const size_t bsm = 2 * sizeof(i32) * BLK_TABLE + sizeof(unsigned short) * (BLK_TABLE / 2);
            if ((rc = cuda_status(cudaFuncSetAttribute(pairs_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       (int)bsm))))
                break;
            a.next = cnt + 4;
            // as many CTAs as fit the SMs' shared memory
            const i64 per_sm = std::max<i64>(1, (i64)(216 * 1024) / (i64)bsm);
            pairs_block<<<(unsigned)std::min<i64>(nk, 152 * per_sm), BLK_WARPS * 32, bsm, st>>>(a, spill, nk, spill2,
                                                                                           cnt + 2);
            note_launch();
            unsigned long long h2 = 0;
            if ((rc = cuda_status(cudaMemcpyAsync(&h2, cnt + 2, sizeof(h2), cudaMemcpyDeviceToHost, st)))) break;
            if ((rc = cuda_status(cudaStreamSynchronize(st)))) break;
            nk = (i64)h2;
            list = spill2;
        }
        if (nk > 0) {
            // last tier: a global table per community, 2 min(incidences, |B|)
            // entries; communities go in chunks whose tables fit a bounded
            // scratch (a single table is at most 2^(1+ceil log2 |B|) entries)
            if ((rc = dev_alloc(&tsz, nk + 1, st))) break;
            if ((rc = dev_alloc(&toff, nk + 1, st))) break;
            spill_sizes<<<GB, 256, 0, st>>>(list, nk, active, A.comm_ptr, A.comm_nodes, MB.cnt, B.n_comms, tsz); note_launch();
            std::vector<i64> hs(nk);
            if ((rc = cuda_status(cudaMemcpyAsync(hs.data(), tsz, nk * sizeof(i64), cudaMemcpyDeviceToHost, st)))) break;
            if ((rc = cuda_status(cudaStreamSynchronize(st)))) break;
            i64 largest = 0;
            for (i64 v : hs) largest = std::max(largest, v);
            size_t fr = 0, tot = 0;
            cudaMemGetInfo(&fr, &tot);
            const i64 budget = std::max<i64>(largest, std::min<i64>((i64)1 << 28, (i64)(fr / 8 / (3 * sizeof(i32)))));
            if ((rc = dev_alloc(&tkey, budget, st))) break;
            if ((rc = dev_alloc(&tcnt, budget, st))) break;
            if ((rc = dev_alloc(&tused, budget, st))) break;
            if ((rc = dev_alloc(&tfill, nk, st))) break;
            // emptied once; each community empties the buckets it claimed
            if ((rc = cuda_status(cudaMemsetAsync(tkey, 0xff, budget * sizeof(i32), st)))) break;
            if ((rc = cuda_status(cudaMemsetAsync(tcnt, 0, budget * sizeof(i32), st)))) break;
            a.tkey = tkey;
            a.tcnt = tcnt;
            a.tused = tused;
            a.tfill = tfill;
            a.toff = toff;
            std::vector<i64> ho;
            for (i64 r0 = 0; r0 < nk && rc == MSCD_OK;) {
                ho.assign(1, 0);
                i64 r1 = r0;
                while (r1 < nk && ho.back() + hs[r1] <= budget) {
                    ho.push_back(ho.back() + hs[r1]);
                    ++r1;
                }
                if ((rc = cuda_status(cudaMemcpyAsync(toff, ho.data(), ho.size() * sizeof(i64), cudaMemcpyHostToDevice,
                                                      st))))
                    break;
                if ((rc = cuda_status(cudaMemsetAsync(tfill, 0, (r1 - r0) * sizeof(unsigned int), st)))) break;
                if ((rc = cuda_status(cudaMemsetAsync(cnt + 5, 0, sizeof(unsigned long long), st)))) break;
                a.next = cnt + 5;
                pairs_global<<<(unsigned)std::min<i64>(r1 - r0, 152 * 4), GLB_WARPS * 32, 0, st>>>(a, list + r0,
                                                                                              r1 - r0);
                note_launch();
                // the host offsets are read by the copy before the next chunk rewrites them
                if ((rc = cuda_status(cudaStreamSynchronize(st)))) break;
                r0 = r1;
            }
        }
        if (h[1] > 0) {
            // group the candidate B communities by part, in descending size
            // inside a part (host sort: they are few)
            const i64 nb = (i64)h[1];
            std::vector<i32> hb(nb), hp(nb), sorted(nb);
            std::vector<i64> hsz(nb), order(nb);
            std::vector<i64> boff(P + 1, 0);
            if ((rc = dev_alloc(&bpart, nb, st))) break;
            if ((rc = dev_alloc(&bsize, nb, st))) break;
            if ((rc = dev_alloc(&dboff, P + 1, st))) break;
            gather_parts<<<GB, 256, 0, st>>>(big, nb, PB.cp, B.comm_ptr, bpart, bsize); note_launch();
            if ((rc = cuda_status(cudaMemcpyAsync(hb.data(), big, nb * sizeof(i32), cudaMemcpyDeviceToHost, st))))
                break;
            if ((rc = cuda_status(cudaMemcpyAsync(hp.data(), bpart, nb * sizeof(i32), cudaMemcpyDeviceToHost, st))))
                break;
            if ((rc = cuda_status(cudaMemcpyAsync(hsz.data(), bsize, nb * sizeof(i64), cudaMemcpyDeviceToHost, st))))
                break;
            if ((rc = cuda_status(cudaStreamSynchronize(st)))) break;
            for (i64 i = 0; i < nb; ++i) order[i] = i;
            std::sort(order.begin(), order.end(), [&](i64 x, i64 y) {
                if (hp[x] != hp[y]) return hp[x] < hp[y];
                if (hsz[x] != hsz[y]) return hsz[x] > hsz[y];
                return hb[x] < hb[y];
            });
            for (i64 i = 0; i < nb; ++i) {
                sorted[i] = hb[order[i]];
                boff[hp[i] + 1]++;
            }
            for (int32_t q = 0; q < P; ++q) boff[q + 1] += boff[q];
            if ((rc = cuda_status(cudaMemcpyAsync(big, sorted.data(), nb * sizeof(i32), cudaMemcpyHostToDevice, st))))
                break;
            if ((rc = cuda_status(cudaMemcpyAsync(dboff, boff.data(), (P + 1) * sizeof(i64), cudaMemcpyHostToDevice,
                                                  st))))
                break;
            disjoint_pairs<<<GB, 256, 0, st>>>(A.comm_ptr, A.comm_nodes, active, n_active, B.comm_ptr, B.comm_nodes,
                                               big, dboff, PA.cp, PA.cn, best); note_launch();
            if ((rc = cuda_status(cudaStreamSynchronize(st)))) break;  // host vectors outlive the copies
        }
    } while (0);
    cudaFreeAsync(spill, st);
    if (spill2) cudaFreeAsync(spill2, st);
    cudaFreeAsync(cnt, st);
    cudaFreeAsync(big, st);
    if (tsz) cudaFreeAsync(tsz, st);
    if (toff) cudaFreeAsync(toff, st);
    if (tkey) cudaFreeAsync(tkey, st);
    if (tcnt) cudaFreeAsync(tcnt, st);
    if (tused) cudaFreeAsync(tused, st);
    if (tfill) cudaFreeAsync(tfill, st);
    if (bpart) cudaFreeAsync(bpart, st);
    if (bsize) cudaFreeAsync(bsize, st);
    if (dboff) cudaFreeAsync(dboff, st);
    if (amax) cudaFreeAsync(amax, st);
    return rc;
}

}  // namespace

int nmi_between(const ScaleResult &X, const ScaleResult &Y, i64 n, const i64 *part_off, int32_t n_parts, double *nmi,
                cudaStream_t st) {
    const i64 CX = X.n_comms, CY = Y.n_comms;
    const int32_t P = part_off ? n_parts : 1;
    for (int32_t p = 0; p < P; ++p) nmi[p] = __builtin_nan("");
    if (CX <= 0 || CY <= 0 || n <= 0) return MSCD_OK;
    u64 *tkey = nullptr;
    i32 *tval = nullptr, *actX = nullptr, *actY = nullptr;
    unsigned char *zeroX = nullptr, *zeroY = nullptr;
    unsigned long long *bestX = nullptr, *bestY = nullptr, *cnt = nullptr, *acc = nullptr;
    CommParts PX, PY;
    Memberships MX, MY;
    int rc = MSCD_OK;
    i64 T = 2;
    while (T < 2 * CY) T <<= 1;
    // acc: per part, X's 128-bit sum, Y's 128-bit sum, X's count, Y's count
    const i64 acc_words = 6 * (i64)P;
    do {
        if ((rc = dev_alloc(&tkey, T, st))) break;
        if ((rc = dev_alloc(&tval, T, st))) break;
        if ((rc = dev_alloc(&zeroX, CX, st))) break;
        if ((rc = dev_alloc(&zeroY, CY, st))) break;
        if ((rc = dev_alloc(&bestX, CX, st))) break;
        if ((rc = dev_alloc(&bestY, CY, st))) break;
        if ((rc = dev_alloc(&actX, CX, st))) break;
        if ((rc = dev_alloc(&actY, CY, st))) break;
        if ((rc = dev_alloc(&PX.cp, CX, st))) break;
        if ((rc = dev_alloc(&PX.cn, CX, st))) break;
        if ((rc = dev_alloc(&PY.cp, CY, st))) break;
        if ((rc = dev_alloc(&PY.cn, CY, st))) break;
        if ((rc = dev_alloc(&cnt, 2, st))) break;
        if ((rc = dev_alloc(&acc, acc_words, st))) break;
        if ((rc = cuda_status(cudaMemsetAsync(tkey, 0, T * sizeof(u64), st)))) break;
        if ((rc = cuda_status(cudaMemsetAsync(zeroX, 0, CX, st)))) break;
        if ((rc = cuda_status(cudaMemsetAsync(zeroY, 0, CY, st)))) break;
        if ((rc = cuda_status(cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), st)))) break;
        if ((rc = cuda_status(cudaMemsetAsync(acc, 0, acc_words * sizeof(unsigned long long), st)))) break;
        comm_parts<<<GB, 256, 0, st>>>(X.comm_ptr, X.comm_nodes, CX, part_off, P, n, PX.cp, PX.cn); note_launch();
        comm_parts<<<GB, 256, 0, st>>>(Y.comm_ptr, Y.comm_nodes, CY, part_off, P, n, PY.cp, PY.cn); note_launch();
        // identical communities
        hash_insert<<<GB, 256, 0, st>>>(Y.comm_hash, CY, tkey, tval, T - 1); note_launch();
        match_identical<<<GB, 256, 0, st>>>(X.comm_ptr, X.comm_nodes, X.comm_hash, CX, Y.comm_ptr, Y.comm_nodes, tkey,
                                            tval, T - 1, zeroX, zeroY); note_launch();
        init_best<<<GB, 256, 0, st>>>(X.comm_ptr, CX, PX.cn, zeroX, bestX, actX, cnt); note_launch();
        init_best<<<GB, 256, 0, st>>>(Y.comm_ptr, CY, PY.cn, zeroY, bestY, actY, cnt + 1); note_launch();
        unsigned long long na[2] = {0, 0};
        if ((rc = cuda_status(cudaMemcpyAsync(na, cnt, sizeof(na), cudaMemcpyDeviceToHost, st)))) break;
        if ((rc = cuda_status(cudaStreamSynchronize(st)))) break;
        // H(X_k|Y) for the X communities without an identical partner
        if (na[0] > 0) {
            if ((rc = build_memberships(Y, n, &MY, st))) break;
            if ((rc = one_direction(X, Y, MY, PX, PY, P, actX, (i64)na[0], bestX, st))) break;
        }
        // H(Y_l|X) likewise
        if (na[1] > 0) {
            if ((rc = build_memberships(X, n, &MX, st))) break;
            if ((rc = one_direction(Y, X, MX, PY, PX, P, actY, (i64)na[1], bestY, st))) break;
        }
        normalise_sum<<<GB, 256, 0, st>>>(X.comm_ptr, CX, PX.cn, PX.cp, bestX, acc, acc + 4 * P); note_launch();
        normalise_sum<<<GB, 256, 0, st>>>(Y.comm_ptr, CY, PY.cn, PY.cp, bestY, acc + 2 * P, acc + 5 * P);
        note_launch();
        std::vector<unsigned long long> h(acc_words);
        if ((rc = cuda_status(cudaMemcpyAsync(h.data(), acc, acc_words * sizeof(unsigned long long),
                                              cudaMemcpyDeviceToHost, st))))
            break;
        if ((rc = cuda_status(cudaStreamSynchronize(st)))) break;
        for (int32_t p = 0; p < P; ++p) {
            const unsigned long long cx = h[4 * P + p], cy = h[5 * P + p];
            if (!cx || !cy) continue;  // a part without communities at one of the scales
            const double sx = (double)h[2 * p + 1] * 4.0 + (double)h[2 * p] * 0x1p-62;
            const double sy = (double)h[2 * P + 2 * p + 1] * 4.0 + (double)h[2 * P + 2 * p] * 0x1p-62;
            nmi[p] = 1.0 - 0.5 * (sx / (double)cx + sy / (double)cy);
        }
    } while (0);
    free_memberships(&MX, st);
    free_memberships(&MY, st);
    cudaFreeAsync(tkey, st);
    cudaFreeAsync(tval, st);
    cudaFreeAsync(zeroX, st);
    cudaFreeAsync(zeroY, st);
    cudaFreeAsync(bestX, st);
    cudaFreeAsync(bestY, st);
    cudaFreeAsync(actX, st);
    cudaFreeAsync(actY, st);
    cudaFreeAsync(PX.cp, st);
    cudaFreeAsync(PX.cn, st);
    cudaFreeAsync(PY.cp, st);
    cudaFreeAsync(PY.cn, st);
    cudaFreeAsync(cnt, st);
    cudaFreeAsync(acc, st);
    return rc != MSCD_OK ? rc : cuda_status(cudaGetLastError());
}

// ---- NMI between two covers given by the caller -------------------------

namespace {

__device__ __forceinline__ u64 mix_list(u64 x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
}

// Warp per community: a hash of its sorted list (equal lists, equal hashes).
__global__ void list_hashes(const i64 *ptr, const i32 *nodes, i64 C, u64 *hash) {
    const int lane = threadIdx.x & 31;
    const i64 warps = (i64)gridDim.x * (blockDim.x >> 5);
    for (i64 c = (i64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < C; c += warps) {
        const i64 n = ptr[c + 1] - ptr[c];
        u64 h = 0;
        for (i64 i = lane; i < n; i += 32) h += mix_list((u64)(u32)nodes[ptr[c] + i] + 0x9E3779B97F4A7C15ull * (u64)(i + 1));
        for (int o = 16; o; o >>= 1) h += __shfl_xor_sync(FULL_MASK, h, o);
        if (lane == 0) {
            h ^= mix_list((u64)n);
            hash[c] = h ? h : 1;
        }
    }
}

// Copy a host cover (each list sorted, no repeats, ids in [0, n)) to the device.
int cover_to_device(const int64_t *ptr, const int32_t *nodes, int64_t C, i64 n, ScaleResult *R, cudaStream_t st) {
    R->n_comms = C;
    R->n_nodes = ptr[C];
    for (int64_t c = 0; c < C; ++c) {
        if (ptr[c + 1] <= ptr[c]) return MSCD_EINVAL;
        for (int64_t e = ptr[c]; e < ptr[c + 1]; ++e)
            if (nodes[e] < 0 || nodes[e] >= n || (e > ptr[c] && nodes[e] <= nodes[e - 1])) return MSCD_EINVAL;
    }
    MSCD_CUDA(cudaMalloc((void **)&R->comm_ptr, (C + 1) * sizeof(i64)));
    MSCD_CUDA(cudaMalloc((void **)&R->comm_nodes, std::max<i64>(R->n_nodes, 1) * sizeof(i32)));
    MSCD_CUDA(cudaMalloc((void **)&R->comm_hash, std::max<i64>(C, 1) * sizeof(u64)));
    MSCD_CUDA(cudaMemcpyAsync(R->comm_ptr, ptr, (C + 1) * sizeof(i64), cudaMemcpyHostToDevice, st));
    if (R->n_nodes > 0)
        MSCD_CUDA(cudaMemcpyAsync(R->comm_nodes, nodes, R->n_nodes * sizeof(i32), cudaMemcpyHostToDevice, st));
    if (C > 0) { list_hashes<<<GB, 256, 0, st>>>(R->comm_ptr, R->comm_nodes, C, R->comm_hash); note_launch(); }
    return cuda_status(cudaGetLastError());
}

}  // namespace

extern "C" int mscd_nmi_covers(mscd_ctx *ctx, int64_t n, const int64_t *ptr_a, const int32_t *nodes_a, int64_t n_a,
                               const int64_t *ptr_b, const int32_t *nodes_b, int64_t n_b, double *nmi) {
    if (!ctx || n < 1 || !ptr_a || !ptr_b || !nmi || n_a < 0 || n_b < 0) return MSCD_EINVAL;
    if ((ptr_a[n_a] > 0 && !nodes_a) || (ptr_b[n_b] > 0 && !nodes_b)) return MSCD_EINVAL;
    MSCD_CUDA(cudaSetDevice(ctx_device_of(ctx)));
    cudaStream_t st = nullptr;
    ScaleResult A, B;
    int rc = cover_to_device(ptr_a, nodes_a, n_a, n, &A, st);
    if (!rc) rc = cover_to_device(ptr_b, nodes_b, n_b, n, &B, st);
    if (!rc) rc = nmi_between(A, B, n, nullptr, 1, nmi, st);
    if (!rc) rc = cuda_status(cudaStreamSynchronize(st));
    scale_result_free(&A);
    scale_result_free(&B);
    return rc;
}
