// The full method of Alg. 2: seeds by rule 1 or 2, then for every scale,
// while changes can be made, growth of every community by one call of Alg. 1
// behind the overlap pre-test of Alg. 3, a check for communities to merge and
// merge rounds; the communities of a scale start the next one.
//
// Everything is deterministic and follows one fixed order (the same as the
// oracle's):
//   * seeds: candidates (nodes with at least two neighbours) in increasing
//     (prio, id); a candidate still available becomes a seed and removes its
//     neighbours (rule 1) or every node within two hops (rule 2).  On the GPU
//     this greedy choice is computed in rounds: an undecided candidate whose
//     (prio, id) is smallest among the undecided candidates within the rule's
//     distance is a seed; candidates within that distance of a new seed are
//     removed; repeat.  The seeds of the rounds are exactly the greedy ones.
//   * pre-test and check: community c scans its members in ascending id and,
//     for each, the communities containing it; the first other community o
//     whose shared-node count reaches eta * min(|c|, |o|) is c's partner.  On
//     the GPU the shared counts come from a per-warp hash table; for each o
//     that reaches the threshold t(o), the scan position where it does is the
//     index in c of their t(o)-th common node, and the partner is the smallest
//     (position, o).
//   * growth: one grow call (grow pass, prune passes if it added) from the
//     current members, the community's seed kept; communities the pre-test
//     flags are not grown.
//   * merge rounds (bookkeeping of a few pairs, on the host): pairs in order
//     of the checked community; a pair joins the round if neither community
//     is in it yet; (c, o) merges o into c; later pairs rename o to c and
//     drop (c, c).
// The merge criterion is that of Sec. 3: max(|A n B|/|A|, |A n B|/|B|) >= eta.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "dedup.cuh"
#include "grow.cuh"
#include "ladder.cuh"

namespace {

constexpr int REACH_WARPS = 8;
constexpr int REACH_TABLE = 1024;  // shared-memory hash entries per warp
const unsigned GB = 152 * 16;

template <class T>
int dalloc(T **p, i64 count, cudaStream_t st) {
    return cuda_status(cudaMallocAsync((void **)p, (size_t)std::max<i64>(count, 1) * sizeof(T), st));
}

// ---- seeds -------------------------------------------------------------

enum : unsigned char { S_UNDECIDED = 0, S_SEED = 1, S_REMOVED = 2, S_NONCAND = 3 };

__global__ void seed_init(const i64 *rp, i64 n, unsigned char *state) {
    for (i64 u = (i64)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (i64)gridDim.x * blockDim.x)
        state[u] = rp[u + 1] - rp[u] >= 2 ? S_UNDECIDED : S_NONCAND;
}

__device__ __forceinline__ bool before(const i32 *prio, i32 a, i32 b) {
    return prio[a] < prio[b] || (prio[a] == prio[b] && a < b);
}

// Thread per node: an undecided node with no undecided node ranked before it
// within distance `rule` becomes a seed (written to `pick`).
__global__ void seed_pick(const i64 *rp, const i32 *col, i64 n, int rule, const i32 *prio,
                          const unsigned char *state, unsigned char *pick, unsigned long long *n_left) {
    for (i64 u = (i64)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (i64)gridDim.x * blockDim.x) {
        pick[u] = 0;
        if (state[u] != S_UNDECIDED) continue;
        atomicAdd(n_left, 1ull);
        bool best = true;
        for (i64 e = rp[u]; e < rp[u + 1] && best; ++e) {
            const i32 v = col[e];
            if (v != u && state[v] == S_UNDECIDED && before(prio, v, (i32)u)) best = false;
            if (rule == 2)
                for (i64 f = rp[v]; f < rp[v + 1] && best; ++f) {
                    const i32 x = col[f];
                    if (x != u && state[x] == S_UNDECIDED && before(prio, x, (i32)u)) best = false;
                }
        }
        if (best) pick[u] = 1;
    }
}

// Thread per node: new seeds take their state; undecided nodes within
// distance `rule` of a new seed are removed.
__global__ void seed_apply(const i64 *rp, const i32 *col, i64 n, int rule, const unsigned char *pick,
                           unsigned char *state) {
    for (i64 u = (i64)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (i64)gridDim.x * blockDim.x) {
        if (pick[u]) {
            state[u] = S_SEED;
            continue;
        }
        if (state[u] != S_UNDECIDED) continue;
        bool near = false;
        for (i64 e = rp[u]; e < rp[u + 1] && !near; ++e) {
            const i32 v = col[e];
            if (pick[v]) near = true;
            if (rule == 2)
                for (i64 f = rp[v]; f < rp[v + 1] && !near; ++f)
                    if (pick[col[f]]) near = true;
        }
        if (near) state[u] = S_REMOVED;
    }
}

// ---- membership sets -----------------------------------------------------

__global__ void memset_count(const i64 *cptr, const i32 *cnodes, i64 C, i32 *cnt) {
    const int lane = threadIdx.x & 31;
    const i64 warps = (i64)gridDim.x * (blockDim.x >> 5);
    for (i64 c = (i64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < C; c += warps)
        for (i64 e = cptr[c] + lane; e < cptr[c + 1]; e += 32) atomicAdd(&cnt[cnodes[e]], 1);
}

__global__ void widen(const i32 *a, i64 n, i64 *b) {
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) b[i] = a[i];
}

__global__ void memset_fill(const i64 *cptr, const i32 *cnodes, i64 C, const i64 *mptr, i32 *cursor, i32 *mlist) {
    const int lane = threadIdx.x & 31;
    const i64 warps = (i64)gridDim.x * (blockDim.x >> 5);
    for (i64 c = (i64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < C; c += warps)
        for (i64 e = cptr[c] + lane; e < cptr[c + 1]; e += 32) {
            const i32 u = cnodes[e];
            mlist[mptr[u] + atomicAdd(&cursor[u], 1)] = (i32)c;
        }
}

// ---- first community reaching the merge threshold ------------------------

__device__ __forceinline__ i64 threshold(i64 a, i64 b, double eta) {
    // smallest count k with k >= eta * min(a, b)
    const double t = eta * (double)min(a, b);
    i64 k = (i64)ceil(t);
    if ((double)(k - 1) >= t) --k;
    return k < 1 ? 1 : k;
}

// Index in A (sorted) of the t-th node A shares with B (sorted); -1 if fewer.
__device__ i64 tth_common(const i32 *A, i64 na, const i32 *B, i64 nb, i64 t) {
    i64 i = 0, j = 0, k = 0;
    while (i < na && j < nb) {
        if (A[i] < B[j]) ++i;
        else if (A[i] > B[j]) ++j;
        else {
            if (++k == t) return i;
            ++i;
            ++j;
        }
    }
    return -1;
}

__device__ __forceinline__ u32 hash_c(i32 l) { return (u32)l * 0x9E3779B1u; }

// Warp per listed community c: partner[c] = the first community reaching the
// threshold in c's scan order, or -1; communities meeting more partners than
// the shared-memory table holds are listed in `spill` for reach_global.
__global__ void __launch_bounds__(REACH_WARPS * 32) reach_smem(const i64 *cptr, const i32 *cnodes, const i64 *mptr,
                                                               const i32 *mlist, const i32 *list, i64 nl, double eta,
                                                               i32 *partner, i32 *spill, unsigned long long *n_spill) {
    __shared__ i32 skey[REACH_WARPS][REACH_TABLE];
    __shared__ i32 scnt[REACH_WARPS][REACH_TABLE];
    __shared__ unsigned short sused[REACH_WARPS][REACH_TABLE / 2];  // buckets claimed, in order
    __shared__ int sfill[REACH_WARPS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    i32 *keys = skey[w], *cnts = scnt[w];
    unsigned short *used = sused[w];
    for (int t = lane; t < REACH_TABLE; t += 32) {  // cleared once; afterwards only what was used
        keys[t] = -1;
        cnts[t] = 0;
    }
    __syncwarp();
    for (i64 q = (i64)blockIdx.x * REACH_WARPS + w; q < nl; q += (i64)gridDim.x * REACH_WARPS) {
        const i32 c = list[q];
        if (lane == 0) sfill[w] = 0;
        __syncwarp();
        bool over = false;
        for (i64 e = cptr[c]; e < cptr[c + 1] && !over; ++e) {
            const i32 u = cnodes[e];
            for (i64 j = mptr[u] + lane; j < mptr[u + 1]; j += 32) {
                const i32 o = mlist[j];
                if (o == c) continue;
                u32 h = hash_c(o) & (REACH_TABLE - 1);
                for (int p = 0; p < REACH_TABLE; ++p) {
                    i32 cur = keys[h];
                    if (cur == -1) {
                        cur = atomicCAS(&keys[h], -1, o);
                        if (cur == -1) {
                            const int f = atomicAdd(&sfill[w], 1);
                            if (f >= REACH_TABLE / 2) over = true;
                            else used[f] = (unsigned short)h;
                            cur = o;
                        }
                    }
                    if (cur == o) {
                        atomicAdd(&cnts[h], 1);
                        break;
                    }
                    h = (h + 1u) & (REACH_TABLE - 1);
                }
            }
            over = __any_sync(FULL_MASK, over);
        }
        __syncwarp();
        if (over) {
            if (lane == 0) spill[atomicAdd(n_spill, 1ull)] = c;
            for (int t = lane; t < REACH_TABLE; t += 32) {
                keys[t] = -1;
                cnts[t] = 0;
            }
            __syncwarp();
            continue;
        }
        const int nf = sfill[w];
        const i64 na = cptr[c + 1] - cptr[c];
        unsigned long long best = ~0ull;  // (position << 32) | partner
        for (int t = lane; t < nf; t += 32) {
            const int h = used[t];
            const i32 o = keys[h];
            const i32 cnt = cnts[h];
            keys[h] = -1;
            cnts[h] = 0;
            const i64 nb = cptr[o + 1] - cptr[o];
            const i64 th = threshold(na, nb, eta);
            if (cnt < th) continue;
            const i64 pos = tth_common(cnodes + cptr[c], na, cnodes + cptr[o], nb, th);
            const unsigned long long key = ((unsigned long long)pos << 32) | (u32)o;
            best = min(best, key);
        }
        for (int off = 16; off; off >>= 1) best = min(best, __shfl_xor_sync(FULL_MASK, best, off));
        if (lane == 0) partner[c] = best == ~0ull ? -1 : (i32)(best & 0xffffffffu);
        __syncwarp();
    }
}

// The same with a global table per listed community (toff: its slice).
__global__ void reach_global(const i64 *cptr, const i32 *cnodes, const i64 *mptr, const i32 *mlist, const i32 *list,
                             i64 nl, const i64 *toff, i32 *tkey, i32 *tcnt, double eta, i32 *partner) {
    const int lane = threadIdx.x & 31;
    const i64 warps = (i64)gridDim.x * (blockDim.x >> 5);
    for (i64 r = (i64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < nl; r += warps) {
        const i32 c = list[r];
        i32 *keys = tkey + toff[r], *cnts = tcnt + toff[r];
        const u32 tm = (u32)(toff[r + 1] - toff[r] - 1);
        for (i64 e = cptr[c]; e < cptr[c + 1]; ++e) {
            const i32 u = cnodes[e];
            for (i64 j = mptr[u] + lane; j < mptr[u + 1]; j += 32) {
                const i32 o = mlist[j];
                if (o == c) continue;
                u32 h = hash_c(o) & tm;
                for (u32 p = 0; p <= tm; ++p) {
                    i32 cur = keys[h];
                    if (cur == -1) {
                        cur = atomicCAS(&keys[h], -1, o);
                        if (cur == -1) cur = o;
                    }
                    if (cur == o) {
                        atomicAdd(&cnts[h], 1);
                        break;
                    }
                    h = (h + 1u) & tm;
                }
            }
        }
        __syncwarp();
        const i64 na = cptr[c + 1] - cptr[c];
        unsigned long long best = ~0ull;
        for (u32 t = lane; t <= tm; t += 32) {
            const i32 o = keys[t];
            if (o < 0) continue;
            const i64 nb = cptr[o + 1] - cptr[o];
            const i64 th = threshold(na, nb, eta);
            if (cnts[t] < th) continue;
            const i64 pos = tth_common(cnodes + cptr[c], na, cnodes + cptr[o], nb, th);
            best = min(best, ((unsigned long long)pos << 32) | (u32)o);
        }
        for (int off = 16; off; off >>= 1) best = min(best, __shfl_xor_sync(FULL_MASK, best, off));
        if (lane == 0) partner[c] = best == ~0ull ? -1 : (i32)(best & 0xffffffffu);
    }
}

// Table size of a spilled community: 2 * (its membership incidences) rounded
// up to a power of two.
__global__ void reach_sizes(const i64 *cptr, const i32 *cnodes, const i64 *mptr, const i32 *list, i64 nl, i64 *tsz) {
    const int lane = threadIdx.x & 31;
    const i64 warps = (i64)gridDim.x * (blockDim.x >> 5);
    for (i64 r = (i64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < nl; r += warps) {
        const i32 c = list[r];
        i64 s = 0;
        for (i64 e = cptr[c] + lane; e < cptr[c + 1]; e += 32) s += mptr[cnodes[e] + 1] - mptr[cnodes[e]];
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(FULL_MASK, s, o);
        i64 t = 2;
        while (t < 2 * s) t <<= 1;
        if (lane == 0) tsz[r] = t;
    }
}

// ---- growth bookkeeping -------------------------------------------------

__global__ void gather_lens(const i64 *cptr, const i32 *list, i64 m, i64 *len) {
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (i64)gridDim.x * blockDim.x)
        len[i] = cptr[list[i] + 1] - cptr[list[i]];
}

// Warp per listed community: copy its list (src offsets sptr by list entry, or
// the community's own) to dst at dptr[i].
__global__ void gather_lists(const i64 *cptr, const i32 *cnodes, const i32 *list, i64 m, const i64 *dptr, i32 *dst) {
    const int lane = threadIdx.x & 31;
    const i64 warps = (i64)gridDim.x * (blockDim.x >> 5);
    for (i64 i = (i64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < m; i += warps) {
        const i32 c = list[i];
        const i64 n = cptr[c + 1] - cptr[c];
        for (i64 k = lane; k < n; k += 32) dst[dptr[i] + k] = cnodes[cptr[c] + k];
    }
}

// Warp per grown unit i (community list[i]): changed[i] = its new list differs.
__global__ void compare_lists(const i64 *cptr, const i32 *cnodes, const i32 *list, i64 m, const i64 *uoff,
                              const i32 *ulen, const i32 *out, unsigned char *changed) {
    const int lane = threadIdx.x & 31;
    const i64 warps = (i64)gridDim.x * (blockDim.x >> 5);
    for (i64 i = (i64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < m; i += warps) {
        const i32 c = list[i];
        const i64 n = cptr[c + 1] - cptr[c];
        bool diff = n != (i64)ulen[i];
        for (i64 k = lane; k < n && !diff; k += 32) diff = cnodes[cptr[c] + k] != out[uoff[i] + k];
        diff = __any_sync(FULL_MASK, diff);
        if (lane == 0) changed[i] = diff ? 1 : 0;
    }
}

// New lengths: a grown and changed community takes its grown list.
__global__ void new_lens(const i64 *cptr, i64 C, const i32 *unit_of, const unsigned char *changed, const i32 *ulen,
                         i64 *len) {
    for (i64 c = (i64)blockIdx.x * blockDim.x + threadIdx.x; c < C; c += (i64)gridDim.x * blockDim.x) {
        const i32 u = unit_of[c];
        len[c] = (u >= 0 && changed[u]) ? (i64)ulen[u] : cptr[c + 1] - cptr[c];
    }
}

__global__ void new_lists(const i64 *cptr, const i32 *cnodes, i64 C, const i32 *unit_of, const unsigned char *changed,
                          const i64 *uoff, const i32 *out, const i64 *nptr, i32 *nnodes) {
    const int lane = threadIdx.x & 31;
    const i64 warps = (i64)gridDim.x * (blockDim.x >> 5);
    for (i64 c = (i64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < C; c += warps) {
        const i32 u = unit_of[c];
        const bool g = u >= 0 && changed[u];
        const i32 *src = g ? out + uoff[u] : cnodes + cptr[c];
        const i64 n = nptr[c + 1] - nptr[c];
        for (i64 k = lane; k < n; k += 32) nnodes[nptr[c] + k] = src[k];
    }
}

// ---- per-community fitness and list hash -----------------------------------

__device__ __forceinline__ bool in_sorted(const i32 *a, i64 n, i32 v) {
    i64 lo = 0, hi = n;
    while (lo < hi) {
        const i64 mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo < n && a[lo] == v;
}

__device__ __forceinline__ u64 mix(u64 x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
}

// Warp per community: K (internal degree sum), V, f = K / V^alpha in real
// weight units (Eq. 1), and a hash of the sorted list.
__global__ void comm_fitness(const DevGraph G, const i64 *cptr, const i32 *cnodes, i64 C, double alpha, double *f,
                             u64 *hash) {
    const int lane = threadIdx.x & 31;
    const i64 warps = (i64)gridDim.x * (blockDim.x >> 5);
    for (i64 c = (i64)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < C; c += warps) {
        const i32 *L = cnodes + cptr[c];
        const i64 n = cptr[c + 1] - cptr[c];
        i64 K = 0, V = 0;
        u64 h = 0;
        for (i64 i = 0; i < n; ++i) {
            const i32 u = L[i];
            if (lane == 0) V += G.k[u];
            for (i64 e = G.rp[u] + lane; e < G.rp[u + 1]; e += 32)
                if (in_sorted(L, n, G.col[e])) K += G.wfx ? G.wfx[e] : 1;
        }
        for (i64 i = lane; i < n; i += 32) h += mix((u64)(u32)L[i] + 0x9E3779B97F4A7C15ull * (u64)(i + 1));
        for (int o = 16; o; o >>= 1) {
            K += __shfl_xor_sync(FULL_MASK, K, o);
            h += __shfl_xor_sync(FULL_MASK, h, o);
        }
        if (lane == 0) {
            double fv = 0.0;
            if (K > 0) {
                const double LN2 = 0.6931471805599453;
                fv = exp(log((double)K) - alpha * log((double)V) + (1.0 - alpha) * (double)G.unit_exp * LN2);
            }
            f[c] = fv;
            h ^= mix((u64)n);
            hash[c] = h ? h : 1;
        }
    }
}

}  // namespace

// Device CSR of communities with their seeds.
struct FullComms {
    i64 C = 0, m = 0;
    i64 *ptr = nullptr;
    i32 *nodes = nullptr;
    std::vector<i32> seed;  // host copy
    void free(cudaStream_t st) {
        if (ptr) cudaFreeAsync(ptr, st);
        if (nodes) cudaFreeAsync(nodes, st);
        ptr = nullptr;
        nodes = nullptr;
    }
};

struct FullState {
    std::vector<i32> initial_seeds;
    std::vector<ScaleResult> scales;  // comm_ptr, comm_nodes, comm_f, comm_hash
    std::vector<std::vector<i32>> seeds;
    std::vector<i64> iterations, merges, grown;
    std::vector<double> nmi;
    int status = MSCD_OK;
};

void full_state_free(FullState *f) {
    if (!f) return;
    for (auto &s : f->scales) scale_result_free(&s);
    delete f;
}

namespace {

// Membership sets of C communities over n nodes.
int build_memsets(const FullComms &X, i64 n, i64 **mptr, i32 **mlist, cudaStream_t st) {
    i32 *cnt = nullptr, *cursor = nullptr;
    i64 *tmp = nullptr;
    int rc = MSCD_OK;
    do {
        if ((rc = dalloc(&cnt, n, st))) break;
        if ((rc = dalloc(&cursor, n, st))) break;
        if ((rc = dalloc(&tmp, n + 1, st))) break;
        if ((rc = dalloc(mptr, n + 1, st))) break;
        if ((rc = dalloc(mlist, X.m, st))) break;
        if ((rc = cuda_status(cudaMemsetAsync(cnt, 0, n * sizeof(i32), st)))) break;
        if ((rc = cuda_status(cudaMemsetAsync(cursor, 0, n * sizeof(i32), st)))) break;
        if (X.C > 0) { memset_count<<<GB, 256, 0, st>>>(X.ptr, X.nodes, X.C, cnt); note_launch(); }
        widen<<<GB, 256, 0, st>>>(cnt, n, tmp); note_launch();
        if ((rc = scan_exclusive_i64(tmp, *mptr, n, *mptr + n, st))) break;
        if (X.C > 0) { memset_fill<<<GB, 256, 0, st>>>(X.ptr, X.nodes, X.C, *mptr, cursor, *mlist); note_launch(); }
    } while (0);
    cudaFreeAsync(cnt, st);
    cudaFreeAsync(cursor, st);
    cudaFreeAsync(tmp, st);
    return rc;
}

// partner[c] for the communities in list (host), -1 where none reaches.
int find_partners(const FullComms &X, i64 n, const std::vector<i32> &list, double eta, std::vector<i32> *partner,
                  cudaStream_t st) {
    partner->assign(X.C, -1);
    if (list.empty() || X.C == 0) return MSCD_OK;
    i64 *mptr = nullptr;
    i32 *mlist = nullptr, *dlist = nullptr, *dpart = nullptr, *spill = nullptr, *tkey = nullptr, *tcnt = nullptr;
    i64 *tsz = nullptr, *toff = nullptr;
    unsigned long long *cnt = nullptr;
    const i64 nl = (i64)list.size();
    int rc = MSCD_OK;
    do {
        if ((rc = build_memsets(X, n, &mptr, &mlist, st))) break;
        if ((rc = dalloc(&dlist, nl, st))) break;
        if ((rc = dalloc(&dpart, X.C, st))) break;
        if ((rc = dalloc(&spill, nl, st))) break;
        if ((rc = dalloc(&cnt, 1, st))) break;
        if ((rc = cuda_status(cudaMemcpyAsync(dlist, list.data(), nl * sizeof(i32), cudaMemcpyHostToDevice, st))))
            break;
        if ((rc = cuda_status(cudaMemsetAsync(dpart, 0xff, X.C * sizeof(i32), st)))) break;
        if ((rc = cuda_status(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st)))) break;
        reach_smem<<<(unsigned)std::min<i64>((nl + REACH_WARPS - 1) / REACH_WARPS, 152 * 4), REACH_WARPS * 32, 0,
                     st>>>(X.ptr, X.nodes, mptr, mlist, dlist, nl, eta, dpart, spill, cnt); note_launch();
        unsigned long long ns = 0;
        if ((rc = cuda_status(cudaMemcpyAsync(&ns, cnt, sizeof(ns), cudaMemcpyDeviceToHost, st)))) break;
        if ((rc = cuda_status(cudaStreamSynchronize(st)))) break;
        if (ns > 0) {
            if ((rc = dalloc(&tsz, (i64)ns + 1, st))) break;
            if ((rc = dalloc(&toff, (i64)ns + 1, st))) break;
            reach_sizes<<<GB, 256, 0, st>>>(X.ptr, X.nodes, mptr, spill, (i64)ns, tsz); note_launch();
            if ((rc = scan_exclusive_i64(tsz, toff, (i64)ns, toff + ns, st))) break;
            i64 TT = 0;
            if ((rc = cuda_status(cudaMemcpyAsync(&TT, toff + ns, sizeof(i64), cudaMemcpyDeviceToHost, st)))) break;
            if ((rc = cuda_status(cudaStreamSynchronize(st)))) break;
            if ((rc = dalloc(&tkey, TT, st))) break;
            if ((rc = dalloc(&tcnt, TT, st))) break;
            if ((rc = cuda_status(cudaMemsetAsync(tkey, 0xff, TT * sizeof(i32), st)))) break;
            if ((rc = cuda_status(cudaMemsetAsync(tcnt, 0, TT * sizeof(i32), st)))) break;
            reach_global<<<GB, 256, 0, st>>>(X.ptr, X.nodes, mptr, mlist, spill, (i64)ns, toff, tkey, tcnt, eta,
                                             dpart); note_launch();
        }
        if ((rc = cuda_status(cudaMemcpyAsync(partner->data(), dpart, X.C * sizeof(i32), cudaMemcpyDeviceToHost, st))))
            break;
        rc = cuda_status(cudaStreamSynchronize(st));
    } while (0);
    cudaFreeAsync(mptr, st);
    cudaFreeAsync(mlist, st);
    cudaFreeAsync(dlist, st);
    cudaFreeAsync(dpart, st);
    cudaFreeAsync(spill, st);
    cudaFreeAsync(cnt, st);
    if (tsz) cudaFreeAsync(tsz, st);
    if (toff) cudaFreeAsync(toff, st);
    if (tkey) cudaFreeAsync(tkey, st);
    if (tcnt) cudaFreeAsync(tcnt, st);
    return rc;
}

int download(const FullComms &X, std::vector<i64> *ptr, std::vector<i32> *nodes, cudaStream_t st) {
    ptr->resize(X.C + 1);
    nodes->resize(X.m);
    MSCD_CUDA(cudaMemcpyAsync(ptr->data(), X.ptr, (X.C + 1) * sizeof(i64), cudaMemcpyDeviceToHost, st));
    if (X.m > 0) MSCD_CUDA(cudaMemcpyAsync(nodes->data(), X.nodes, X.m * sizeof(i32), cudaMemcpyDeviceToHost, st));
    return cuda_status(cudaStreamSynchronize(st));
}

int upload(FullComms *X, const std::vector<i64> &ptr, const std::vector<i32> &nodes, cudaStream_t st) {
    X->free(st);
    X->C = (i64)ptr.size() - 1;
    X->m = (i64)nodes.size();
    int rc = dalloc(&X->ptr, X->C + 1, st);
    if (!rc) rc = dalloc(&X->nodes, X->m, st);
    if (!rc)
        rc = cuda_status(cudaMemcpyAsync(X->ptr, ptr.data(), (X->C + 1) * sizeof(i64), cudaMemcpyHostToDevice, st));
    if (!rc && X->m > 0)
        rc = cuda_status(cudaMemcpyAsync(X->nodes, nodes.data(), X->m * sizeof(i32), cudaMemcpyHostToDevice, st));
    if (!rc) rc = cuda_status(cudaStreamSynchronize(st));
    return rc;
}

}  // namespace

// The whole method (see the file header).  pipe: the context's growth pipeline.
int full_run(const DevGraph &G, i64 max_part_n, const double *alphas, int32_t n_scales, int seed_rule,
             const i32 *prio_host, const i64 *init_ptr, const i32 *init_nodes, i64 n_init, double eta,
             i64 max_iters, GrowPipe &pipe, FullState *out, cudaStream_t st) {
    const i64 n = G.n;
    FullComms X;
    int rc = MSCD_OK;
    std::vector<int> ladder;
    std::vector<bool> in_smem;
    if ((rc = make_ladder(G, max_part_n, pipe.p, &ladder, &in_smem))) return rc;
    // ---- initial communities ----
    if (init_ptr) {
        std::vector<i64> ptr(1, 0);
        std::vector<i32> nodes;
        for (i64 i = 0; i < n_init; ++i) {
            std::vector<i32> m(init_nodes + init_ptr[i], init_nodes + init_ptr[i + 1]);
            if (m.empty()) return MSCD_EINVAL;
            for (i32 v : m)
                if (v < 0 || (i64)v >= n) return MSCD_EINVAL;
            X.seed.push_back(m[0]);
            std::sort(m.begin(), m.end());
            m.erase(std::unique(m.begin(), m.end()), m.end());
            nodes.insert(nodes.end(), m.begin(), m.end());
            ptr.push_back((i64)nodes.size());
        }
        if ((rc = upload(&X, ptr, nodes, st))) return rc;
    } else {
        if (seed_rule != 1 && seed_rule != 2) return MSCD_EINVAL;
        unsigned char *state = nullptr, *pick = nullptr;
        i32 *dprio = nullptr;
        unsigned long long *left = nullptr;
        std::vector<unsigned char> hs;
        do {
            if ((rc = dalloc(&state, n, st))) break;
            if ((rc = dalloc(&pick, n, st))) break;
            if ((rc = dalloc(&dprio, n, st))) break;
            if ((rc = dalloc(&left, 1, st))) break;
            if ((rc = cuda_status(cudaMemcpyAsync(dprio, prio_host, n * sizeof(i32), cudaMemcpyHostToDevice, st))))
                break;
            if (n > 0) { seed_init<<<GB, 256, 0, st>>>(G.rp, n, state); note_launch(); }
            for (i64 round = 0; round <= n && rc == MSCD_OK; ++round) {
                unsigned long long hl = 0;
                if ((rc = cuda_status(cudaMemsetAsync(left, 0, sizeof(hl), st)))) break;
                seed_pick<<<GB, 256, 0, st>>>(G.rp, G.col, n, seed_rule, dprio, state, pick, left); note_launch();
                if ((rc = cuda_status(cudaMemcpyAsync(&hl, left, sizeof(hl), cudaMemcpyDeviceToHost, st)))) break;
                if ((rc = cuda_status(cudaStreamSynchronize(st)))) break;
                if (hl == 0) break;
                seed_apply<<<GB, 256, 0, st>>>(G.rp, G.col, n, seed_rule, pick, state); note_launch();
            }
            if (rc) break;
            hs.resize(n);
            if ((rc = cuda_status(cudaMemcpyAsync(hs.data(), state, n * sizeof(unsigned char), cudaMemcpyDeviceToHost,
                                                  st))))
                break;
            rc = cuda_status(cudaStreamSynchronize(st));
        } while (0);
        cudaFreeAsync(state, st);
        cudaFreeAsync(pick, st);
        cudaFreeAsync(dprio, st);
        cudaFreeAsync(left, st);
        if (rc) return rc;
        for (i64 u = 0; u < n; ++u)
            if (hs[u] == S_SEED) X.seed.push_back((i32)u);
        std::sort(X.seed.begin(), X.seed.end(), [&](i32 a, i32 b) {
            return prio_host[a] < prio_host[b] || (prio_host[a] == prio_host[b] && a < b);
        });
        std::vector<i64> ptr(X.seed.size() + 1);
        for (size_t i = 0; i <= X.seed.size(); ++i) ptr[i] = (i64)i;
        if ((rc = upload(&X, ptr, X.seed, st))) return rc;
    }
    out->initial_seeds = X.seed;
    // ---- scales ----
    double *dalpha = nullptr;
    if ((rc = dalloc(&dalpha, 1, st))) return rc;
    for (int32_t sc = 0; sc < n_scales && rc == MSCD_OK; ++sc) {
        const double alpha = alphas[sc];
        if ((rc = cuda_status(cudaMemcpyAsync(dalpha, &alpha, sizeof(double), cudaMemcpyHostToDevice, st)))) break;
        i64 it = 0, merges = 0, grown = 0;
        for (;; ++it) {
            if (it >= max_iters) {
                out->status = MSCD_ETIMEOUT;
                break;
            }
            // pre-test of every community against the current sets
            std::vector<i32 > all(X.C);
            for (i64 c = 0; c < X.C; ++c) all[c] = (i32)c;
            std::vector<i32> pre;
            if ((rc = find_partners(X, n, all, eta, &pre, st))) break;
            std::vector<i32> grow_list, unit_of(X.C, -1);
            for (i64 c = 0; c < X.C; ++c)
                if (pre[c] < 0) {
                    unit_of[c] = (i32)grow_list.size();
                    grow_list.push_back((i32)c);
                }
            const i64 m = (i64)grow_list.size();
            bool changes = false;
            std::vector<unsigned char> changed(std::max<i64>(m, 1), 0);
            if (m > 0) {
                // one grow call from the current members of each unflagged community
                i32 *dlist = nullptr, *dseeds = nullptr, *dunit = nullptr, *ulen = nullptr,
                    *ustatus = nullptr;
                i64 *ilen = nullptr, *iptr = nullptr, *uoff = nullptr, *ustat = nullptr, *nlen = nullptr,
                    *nptr = nullptr;
                i32 *inodes = nullptr, *nnodes = nullptr;
                u64 *uhash = nullptr;
                double *uf = nullptr;
                unsigned char *dchanged = nullptr;
                std::vector<i32> hseeds(m);
                for (i64 i = 0; i < m; ++i) hseeds[i] = X.seed[grow_list[i]];
                do {
                    if ((rc = dalloc(&dlist, m, st))) break;
                    if ((rc = dalloc(&dseeds, m, st))) break;
                    if ((rc = dalloc(&ilen, m + 1, st))) break;
                    if ((rc = dalloc(&iptr, m + 1, st))) break;
                    if ((rc = cuda_status(cudaMemcpyAsync(dlist, grow_list.data(), m * sizeof(i32),
                                                          cudaMemcpyHostToDevice, st))))
                        break;
                    if ((rc = cuda_status(cudaMemcpyAsync(dseeds, hseeds.data(), m * sizeof(i32),
                                                          cudaMemcpyHostToDevice, st))))
                        break;
                    gather_lens<<<GB, 256, 0, st>>>(X.ptr, dlist, m, ilen); note_launch();
                    if ((rc = scan_exclusive_i64(ilen, iptr, m, iptr + m, st))) break;
                    i64 mi = 0;
                    if ((rc = cuda_status(cudaMemcpyAsync(&mi, iptr + m, sizeof(i64), cudaMemcpyDeviceToHost, st))))
                        break;
                    if ((rc = cuda_status(cudaStreamSynchronize(st)))) break;
                    if ((rc = dalloc(&inodes, mi, st))) break;
                    gather_lists<<<GB, 256, 0, st>>>(X.ptr, X.nodes, dlist, m, iptr, inodes); note_launch();
                    if ((rc = dalloc(&uoff, m, st))) break;
                    if ((rc = dalloc(&ulen, m, st))) break;
                    if ((rc = dalloc(&uhash, m, st))) break;
                    if ((rc = dalloc(&uf, m, st))) break;
                    if ((rc = dalloc(&ustat, m * MSCD_NSTATS, st))) break;
                    if ((rc = dalloc(&ustatus, m, st))) break;
                    GrowArgs proto{};
                    proto.G = G;
                    proto.alphas = dalpha;
                    proto.seeds = dseeds;
                    proto.n_seeds = m;
                    proto.init_ptr = iptr;
                    proto.init_nodes = inodes;
                    proto.single_round = 1;
                    proto.max_rounds = 2;
                    proto.uoff = uoff;
                    proto.ulen = ulen;
                    proto.uhash = uhash;
                    proto.uf = uf;
                    proto.ustat = ustat;
                    proto.ustatus = ustatus;
                    proto.log_kmax = G.kmax > 1 ? (float)std::log((double)G.kmax) : 0.0f;
                    unsigned long long cursor = 0;
                    size_t fr = 0, tot = 0;
                    cudaMemGetInfo(&fr, &tot);
                    if ((rc = grow_units(pipe, proto, m, ladder, in_smem, false, (i64)(fr / 10 / sizeof(i32)),
                                         max_part_n, &cursor)))
                        break;
                    grown += m;
                    std::vector<i32> hst(m);
                    if ((rc = cuda_status(cudaMemcpyAsync(hst.data(), ustatus, m * sizeof(i32), cudaMemcpyDeviceToHost,
                                                          st))))
                        break;
                    if ((rc = dalloc(&dchanged, m, st))) break;
                    compare_lists<<<GB, 256, 0, st>>>(X.ptr, X.nodes, dlist, m, uoff, ulen, pipe.out_nodes, dchanged);
                    note_launch();
                    if ((rc = cuda_status(cudaMemcpyAsync(changed.data(), dchanged, m, cudaMemcpyDeviceToHost, st))))
                        break;
                    if ((rc = cuda_status(cudaStreamSynchronize(st)))) break;
                    for (i32 s : hst)
                        if (s == MSCD_EUNDECIDED) out->status = MSCD_EUNDECIDED;
                    for (i64 i = 0; i < m; ++i) changes = changes || changed[i];
                    if (changes) {
                        if ((rc = dalloc(&dunit, X.C, st))) break;
                        if ((rc = dalloc(&nlen, X.C + 1, st))) break;
                        if ((rc = dalloc(&nptr, X.C + 1, st))) break;
                        if ((rc = cuda_status(cudaMemcpyAsync(dunit, unit_of.data(), X.C * sizeof(i32),
                                                              cudaMemcpyHostToDevice, st))))
                            break;
                        new_lens<<<GB, 256, 0, st>>>(X.ptr, X.C, dunit, dchanged, ulen, nlen); note_launch();
                        if ((rc = scan_exclusive_i64(nlen, nptr, X.C, nptr + X.C, st))) break;
                        i64 nm = 0;
                        if ((rc = cuda_status(cudaMemcpyAsync(&nm, nptr + X.C, sizeof(i64), cudaMemcpyDeviceToHost,
                                                              st))))
                            break;
                        if ((rc = cuda_status(cudaStreamSynchronize(st)))) break;
                        if ((rc = dalloc(&nnodes, nm, st))) break;
                        new_lists<<<GB, 256, 0, st>>>(X.ptr, X.nodes, X.C, dunit, dchanged, uoff, pipe.out_nodes, nptr,
                                                      nnodes); note_launch();
                        X.free(st);
                        X.ptr = nptr;
                        X.nodes = nnodes;
                        X.m = nm;
                        nptr = nullptr;
                        nnodes = nullptr;
                    }
                } while (0);
                cudaFreeAsync(dlist, st);
                cudaFreeAsync(dseeds, st);
                cudaFreeAsync(ilen, st);
                cudaFreeAsync(iptr, st);
                cudaFreeAsync(inodes, st);
                cudaFreeAsync(uoff, st);
                cudaFreeAsync(ulen, st);
                cudaFreeAsync(uhash, st);
                cudaFreeAsync(uf, st);
                cudaFreeAsync(ustat, st);
                cudaFreeAsync(ustatus, st);
                cudaFreeAsync(dchanged, st);
                cudaFreeAsync(dunit, st);
                cudaFreeAsync(nlen, st);
                if (nptr) cudaFreeAsync(nptr, st);
                if (nnodes) cudaFreeAsync(nnodes, st);
                if (rc) break;
            }
            // check list: flagged or changed, in index order
            std::vector<i32> check;
            for (i64 c = 0; c < X.C; ++c)
                if (pre[c] >= 0 || (unit_of[c] >= 0 && changed[unit_of[c]])) check.push_back((i32)c);
            std::vector<i32> partner;
            if ((rc = find_partners(X, n, check, eta, &partner, st))) break;
            std::vector<std::pair<i64, i64>> pairs;
            for (i32 c : check)
                if (partner[c] >= 0) pairs.push_back({c, partner[c]});
            if (!pairs.empty()) {
                // merge rounds on the host lists
                std::vector<i64> hp;
                std::vector<i32> hn;
                if ((rc = download(X, &hp, &hn, st))) break;
                std::vector<std::vector<i32>> L(X.C);
                for (i64 c = 0; c < X.C; ++c) L[c].assign(hn.begin() + hp[c], hn.begin() + hp[c + 1]);
                std::vector<char> alive(X.C, 1);
                while (!pairs.empty()) {
                    std::vector<char> used(X.C, 0);
                    std::vector<std::pair<i64, i64>> round, rest;
                    for (auto &pq : pairs) {
                        if (pq.first != pq.second && !used[pq.first] && !used[pq.second]) {
                            used[pq.first] = used[pq.second] = 1;
                            round.push_back(pq);
                        } else {
                            rest.push_back(pq);
                        }
                    }
                    std::vector<i64> into(X.C);
                    for (i64 c = 0; c < X.C; ++c) into[c] = c;
                    for (auto &pq : round) {
                        std::vector<i32> u;
                        std::set_union(L[pq.first].begin(), L[pq.first].end(), L[pq.second].begin(),
                                       L[pq.second].end(), std::back_inserter(u));
                        L[pq.first].swap(u);
                        L[pq.second].clear();
                        alive[pq.second] = 0;
                        into[pq.second] = pq.first;
                        ++merges;
                    }
                    pairs.clear();
                    for (auto &pq : rest) {
                        const i64 a = into[pq.first], b = into[pq.second];
                        if (a != b) pairs.push_back({a, b});
                    }
                }
                changes = true;
                std::vector<i64> np(1, 0);
                std::vector<i32> nn, ns;
                for (i64 c = 0; c < X.C; ++c)
                    if (alive[c]) {
                        nn.insert(nn.end(), L[c].begin(), L[c].end());
                        np.push_back((i64)nn.size());
                        ns.push_back(X.seed[c]);
                    }
                X.seed.swap(ns);
                if ((rc = upload(&X, np, nn, st))) break;
            }
            if (!changes) break;
        }
        if (rc) break;
        // the scale's result: its communities, their fitness and hashes
        ScaleResult R;
        R.n_comms = X.C;
        R.n_nodes = X.m;
        do {
            if ((rc = cuda_status(cudaMalloc((void **)&R.comm_ptr, (X.C + 1) * sizeof(i64))))) break;
            if ((rc = cuda_status(cudaMalloc((void **)&R.comm_nodes, std::max<i64>(X.m, 1) * sizeof(i32))))) break;
            if ((rc = cuda_status(cudaMalloc((void **)&R.comm_f, std::max<i64>(X.C, 1) * sizeof(double))))) break;
            if ((rc = cuda_status(cudaMalloc((void **)&R.comm_hash, std::max<i64>(X.C, 1) * sizeof(u64))))) break;
            if ((rc = cuda_status(cudaMemcpyAsync(R.comm_ptr, X.ptr, (X.C + 1) * sizeof(i64), cudaMemcpyDeviceToDevice,
                                                  st))))
                break;
            if (X.m > 0 && (rc = cuda_status(cudaMemcpyAsync(R.comm_nodes, X.nodes, X.m * sizeof(i32),
                                                             cudaMemcpyDeviceToDevice, st))))
                break;
            if (X.C > 0) {
                comm_fitness<<<GB, 256, 0, st>>>(G, X.ptr, X.nodes, X.C, alpha, R.comm_f, R.comm_hash); note_launch();
            }
            rc = cuda_status(cudaStreamSynchronize(st));
        } while (0);
        out->scales.push_back(R);
        out->seeds.push_back(X.seed);
        out->iterations.push_back(it);
        out->merges.push_back(merges);
        out->grown.push_back(grown);
        if (out->status == MSCD_ETIMEOUT) break;
    }
    cudaFreeAsync(dalpha, st);
    X.free(st);
    if (rc) return rc;
    // stability between successive scales
    out->nmi.assign(std::max<size_t>(out->scales.size(), 1) - 1, NAN);
    for (size_t s = 0; s + 1 < out->scales.size() && rc == MSCD_OK; ++s)
        rc = nmi_between(out->scales[s], out->scales[s + 1], n, nullptr, 1, &out->nmi[s], st);
    if (rc) return rc;
    return out->status;
}

// ---- C ABI ---------------------------------------------------------------

FullState **ctx_full(mscd_ctx *c);
bool ctx_graph_part(mscd_ctx *c, int32_t id, DevGraph *g, i64 *max_part_n);
int ctx_device_of(mscd_ctx *c);
GrowPipe *ctx_pipe(mscd_ctx *c, cudaStream_t st);

extern "C" {

int mscd_full_run(mscd_ctx *c, int32_t graph_id, const double *alphas, int32_t n_scales, const int32_t *prio,
                  const int64_t *init_ptr, const int32_t *init_nodes, int64_t n_init, const mscd_full_params *params,
                  void *cuda_stream) {
    if (!c || !alphas || n_scales < 1) return MSCD_EINVAL;
    mscd_full_params p{};
    p.struct_size = (int32_t)sizeof(mscd_full_params);
    p.seed_rule = 1;
    p.eta = 0.5;
    p.max_iters = 1000;
    if (params) {
        if (params->struct_size != (int32_t)sizeof(mscd_full_params)) return MSCD_EINVAL;
        p = *params;
        if (p.eta == 0.0) p.eta = 0.5;
        if (p.max_iters <= 0) p.max_iters = 1000;
        if (p.seed_rule == 0) p.seed_rule = 1;
    }
    if (!(p.eta > 0.0) || p.eta > 1.0) return MSCD_EINVAL;
    for (int32_t s = 0; s < n_scales; ++s)
        if (!(alphas[s] > 0.0) || !std::isfinite(alphas[s])) return MSCD_EINVAL;
    DevGraph G;
    i64 max_part_n = 0;
    if (!ctx_graph_part(c, graph_id, &G, &max_part_n)) return MSCD_EINVAL;
    if (init_ptr ? (n_init < 0 || (n_init > 0 && !init_nodes) || init_ptr[0] != 0) : !prio) return MSCD_EINVAL;
    if (init_ptr)
        for (i64 i = 0; i < n_init; ++i)
            if (init_ptr[i + 1] <= init_ptr[i]) return MSCD_EINVAL;
    MSCD_CUDA(cudaSetDevice(ctx_device_of(c)));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    GrowPipe *pipe = ctx_pipe(c, st);
    FullState **slot = ctx_full(c);
    full_state_free(*slot);
    *slot = nullptr;
    FullState *f = new (std::nothrow) FullState();
    if (!f) return MSCD_ENOMEM;
    int rc = full_run(G, max_part_n, alphas, n_scales, p.seed_rule, prio, init_ptr, init_nodes, n_init, p.eta,
                      p.max_iters, *pipe, f, st);
    if (rc != MSCD_OK && rc != MSCD_ETIMEOUT && rc != MSCD_EUNDECIDED) {
        full_state_free(f);
        return rc;
    }
    *slot = f;
    return rc;
}

int mscd_full_get_seeds(mscd_ctx *c, int32_t *seeds, int64_t cap, int64_t *n) {
    if (!c || !n) return MSCD_EINVAL;
    FullState *f = *ctx_full(c);
    if (!f) return MSCD_ENORESULT;
    *n = (int64_t)f->initial_seeds.size();
    if (cap < *n || (*n > 0 && !seeds)) return MSCD_ESMALL;
    std::copy(f->initial_seeds.begin(), f->initial_seeds.end(), seeds);
    return MSCD_OK;
}

int mscd_full_get_scale(mscd_ctx *c, int32_t scale, int64_t *ptr, int64_t ptr_cap, int32_t *nodes,
                        int64_t nodes_cap, int32_t *seeds, double *fitness, int64_t *n_comms, int64_t *n_nodes) {
    if (!c || !n_comms || !n_nodes) return MSCD_EINVAL;
    FullState *f = *ctx_full(c);
    if (!f) return MSCD_ENORESULT;
    if (scale < 0 || scale >= (int32_t)f->scales.size()) return MSCD_EINVAL;
    const ScaleResult &R = f->scales[scale];
    *n_comms = R.n_comms;
    *n_nodes = R.n_nodes;
    if (ptr_cap < R.n_comms + 1 || nodes_cap < R.n_nodes || !ptr || (R.n_nodes > 0 && !nodes)) return MSCD_ESMALL;
    MSCD_CUDA(cudaSetDevice(ctx_device_of(c)));
    MSCD_CUDA(cudaMemcpy(ptr, R.comm_ptr, (R.n_comms + 1) * sizeof(i64), cudaMemcpyDeviceToHost));
    if (R.n_nodes > 0) MSCD_CUDA(cudaMemcpy(nodes, R.comm_nodes, R.n_nodes * sizeof(i32), cudaMemcpyDeviceToHost));
    if (fitness && R.n_comms > 0)
        MSCD_CUDA(cudaMemcpy(fitness, R.comm_f, R.n_comms * sizeof(double), cudaMemcpyDeviceToHost));
    if (seeds) std::copy(f->seeds[scale].begin(), f->seeds[scale].end(), seeds);
    return MSCD_OK;
}

int mscd_full_get_info(mscd_ctx *c, int32_t scale, int64_t *iterations, int64_t *merges, int64_t *grown,
                       double *nmi_next) {
    if (!c) return MSCD_EINVAL;
    FullState *f = *ctx_full(c);
    if (!f) return MSCD_ENORESULT;
    if (scale < 0 || scale >= (int32_t)f->scales.size()) return MSCD_EINVAL;
    if (iterations) *iterations = f->iterations[scale];
    if (merges) *merges = f->merges[scale];
    if (grown) *grown = f->grown[scale];
    if (nmi_next) *nmi_next = scale + 1 < (int32_t)f->scales.size() ? f->nmi[scale] : NAN;
    return MSCD_OK;
}

}  // extern "C"
