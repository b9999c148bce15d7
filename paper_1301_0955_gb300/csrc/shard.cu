// Merge of per-GPU shards of one scale's deduplicated communities.
//
// Every unit grows from its own seed alone (Alg. 1), so a job's seeds can be
// split across GPUs and each GPU deduplicates its own units.  Joining the
// shards is the one exchange step of that split: a list found in several
// shards is one community, and the whole job numbers its communities in order
// of their smallest generating seed index.  Each shard community's smallest
// seed index in the whole job is found from the shard's seed map; the shard
// communities are then visited in ascending order of it, so the first visit
// of a list is the one that holds its smallest seed, and numbering lists at
// their first visit gives the whole job's order.  Lists are matched by a
// 64-bit hash and then compared element by element, so a hash collision can
// only cost a comparison.
//
// Host code: the shards arrive in host memory after the exchange and the
// merge is a linear pass over them, so no device is involved.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace {

u64 list_hash(const i32 *a, i64 len) {
    u64 h = 0x243f6a8885a308d3ull ^ (u64)len;
    for (i64 i = 0; i < len; ++i) {
        h ^= (u64)(u32)a[i];
        h *= 0x100000001b3ull;
        h ^= h >> 29;
    }
    return h;
}

struct Ref {  // one community of one shard
    i64 first;    // its smallest seed index in the whole job
    int32_t shard;
    i64 comm;
};

}  // namespace

extern "C" int mscd_merge_shards(const mscd_cover_shard *shards, int32_t n_shards, int64_t n_seeds_total,
                                 int64_t *ptr, int64_t ptr_cap, int32_t *nodes, int64_t nodes_cap, double *fitness,
                                 int32_t *seed2comm, int64_t *n_comms, int64_t *n_nodes) {
    if (!n_comms || !n_nodes || n_shards < 0 || n_seeds_total < 0 || (n_shards > 0 && !shards)) return MSCD_EINVAL;
    // every seed index of the job exactly once
    std::vector<unsigned char> seen((size_t)n_seeds_total, 0);
    i64 total_seeds = 0;
    for (int32_t p = 0; p < n_shards; ++p) {
        const mscd_cover_shard &s = shards[p];
        if (s.n_seeds < 0 || s.n_comms < 0) return MSCD_EINVAL;
        if (s.n_seeds > 0 && (!s.seed_index || !s.seed2comm)) return MSCD_EINVAL;
        if (!s.ptr && s.n_comms > 0) return MSCD_EINVAL;
        if (fitness && s.n_comms > 0 && !s.fitness) return MSCD_EINVAL;
        if (s.ptr && s.ptr[0] != 0) return MSCD_EINVAL;
        const i64 nn = s.n_comms > 0 ? s.ptr[s.n_comms] : 0;
        if (nn > 0 && !s.nodes) return MSCD_EINVAL;
        for (i64 c = 0; c < s.n_comms; ++c) {
            const i64 b = s.ptr[c], e = s.ptr[c + 1];
            if (e <= b || e > nn) return MSCD_EINVAL;  // empty or out of order
            if (s.nodes[b] < 0) return MSCD_EINVAL;
            for (i64 i = b + 1; i < e; ++i)
                if (s.nodes[i] <= s.nodes[i - 1]) return MSCD_EINVAL;
        }
        for (i64 j = 0; j < s.n_seeds; ++j) {
            const i64 g = s.seed_index[j];
            if (g < 0 || g >= n_seeds_total || seen[(size_t)g]) return MSCD_EINVAL;
            seen[(size_t)g] = 1;
            if (s.seed2comm[j] < 0 || (i64)s.seed2comm[j] >= s.n_comms) return MSCD_EINVAL;
        }
        total_seeds += s.n_seeds;
    }
    if (total_seeds != n_seeds_total) return MSCD_EINVAL;

    // smallest seed index of every shard community
    std::vector<Ref> refs;
    std::vector<i64> base(n_shards + 1, 0);
    for (int32_t p = 0; p < n_shards; ++p) base[p + 1] = base[p] + shards[p].n_comms;
    refs.resize((size_t)base[n_shards]);
    for (int32_t p = 0; p < n_shards; ++p) {
        const mscd_cover_shard &s = shards[p];
        for (i64 c = 0; c < s.n_comms; ++c) refs[(size_t)(base[p] + c)] = Ref{n_seeds_total, p, c};
        for (i64 j = 0; j < s.n_seeds; ++j) {
            Ref &r = refs[(size_t)(base[p] + s.seed2comm[j])];
            r.first = std::min<i64>(r.first, s.seed_index[j]);
        }
    }
    for (const Ref &r : refs)
        if (r.first == n_seeds_total) return MSCD_EINVAL;  // a community no seed of its shard grew
    std::vector<i64> order(refs.size());
    std::iota(order.begin(), order.end(), (i64)0);
    std::sort(order.begin(), order.end(), [&](i64 a, i64 b) { return refs[(size_t)a].first < refs[(size_t)b].first; });

    // number the distinct lists at their first visit
    std::vector<i64> gid(refs.size(), -1);
    std::vector<i64> rep;  // global community -> its first shard community (index into refs)
    std::unordered_map<u64, std::vector<i64>> by_hash;
    by_hash.reserve(refs.size() * 2 + 1);
    i64 total_nodes = 0;
    auto list_of = [&](i64 ref, const i32 **a, i64 *len) {
        const mscd_cover_shard &s = shards[refs[(size_t)ref].shard];
        const i64 c = refs[(size_t)ref].comm;
        *a = s.nodes + s.ptr[c];
        *len = s.ptr[c + 1] - s.ptr[c];
    };
    for (i64 ref : order) {
        const i32 *a;
        i64 len;
        list_of(ref, &a, &len);
        std::vector<i64> &cands = by_hash[list_hash(a, len)];
        i64 g = -1;
        for (i64 cand : cands) {
            const i32 *b;
            i64 lb;
            list_of(rep[(size_t)cand], &b, &lb);
            if (lb == len && std::memcmp(a, b, (size_t)len * sizeof(i32)) == 0) {
                g = cand;
                break;
            }
        }
        if (g < 0) {
            g = (i64)rep.size();
            rep.push_back(ref);
            cands.push_back(g);
            total_nodes += len;
        }
        gid[(size_t)ref] = g;
    }

    const i64 C = (i64)rep.size();
    *n_comms = C;
    *n_nodes = total_nodes;
    if (ptr_cap < C + 1 || nodes_cap < total_nodes || !ptr || (total_nodes > 0 && !nodes)) return MSCD_ESMALL;
    ptr[0] = 0;
    for (i64 g = 0; g < C; ++g) {
        const i32 *a;
        i64 len;
        list_of(rep[(size_t)g], &a, &len);
        std::memcpy(nodes + ptr[g], a, (size_t)len * sizeof(i32));
        ptr[g + 1] = ptr[g] + len;
        if (fitness) {
            const Ref &r = refs[(size_t)rep[(size_t)g]];
            fitness[g] = shards[r.shard].fitness[r.comm];
        }
    }
    if (seed2comm)
        for (int32_t p = 0; p < n_shards; ++p) {
            const mscd_cover_shard &s = shards[p];
            for (i64 j = 0; j < s.n_seeds; ++j)
                seed2comm[s.seed_index[j]] = (i32)gid[(size_t)(base[p] + s.seed2comm[j])];
        }
    return MSCD_OK;
}
