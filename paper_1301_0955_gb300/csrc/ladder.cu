// Growth through the node-slot class ladder (see ladder.cuh).
#include <algorithm>
#include <cmath>

#include "ladder.cuh"

namespace {

struct Task {
    int cls;                 // index in the ladder
    std::vector<i64> units;  // the listed work items, unless `all`
    bool all;                // every unit of the call
};

int ensure_arena(GrowPipe &w, size_t bytes) {
    if (w.arena_bytes >= bytes) return MSCD_OK;
    cudaStreamSynchronize(w.st);
    cudaFree(w.arena);
    w.arena = nullptr;
    w.arena_bytes = 0;
    MSCD_CUDA(cudaMalloc((void **)&w.arena, bytes));
    w.arena_bytes = bytes;
    return MSCD_OK;
}

}  // namespace

int pipe_reserve(GrowPipe &w, i64 units) {
    if (!w.ctr) MSCD_CUDA(cudaMalloc((void **)&w.ctr, sizeof(Counters)));
    if (w.retry_cap >= units) return MSCD_OK;
    cudaStreamSynchronize(w.st);
    cudaFree(w.retry_a);
    cudaFree(w.retry_b);
    w.retry_a = w.retry_b = nullptr;
    w.retry_cap = 0;
    const i64 cap = std::max<i64>(units, 1);
    MSCD_CUDA(cudaMalloc((void **)&w.retry_a, cap * sizeof(i64)));
    MSCD_CUDA(cudaMalloc((void **)&w.retry_b, cap * sizeof(i64)));
    w.retry_cap = cap;
    return MSCD_OK;
}

int pipe_output(GrowPipe &w, i64 need, i64 keep) {
    if (need <= w.out_cap) return MSCD_OK;
    const i64 cap = std::max<i64>(need + need / 8, w.out_cap + w.out_cap / 2);
    i32 *nb = nullptr;
    MSCD_CUDA(cudaMalloc((void **)&nb, (size_t)cap * sizeof(i32)));
    if (w.out_nodes && keep > 0)
        MSCD_CUDA(cudaMemcpyAsync(nb, w.out_nodes, (size_t)keep * sizeof(i32), cudaMemcpyDeviceToDevice, w.st));
    cudaStreamSynchronize(w.st);
    cudaFree(w.out_nodes);
    w.out_nodes = nb;
    w.out_cap = cap;
    return MSCD_OK;
}

void pipe_release_output(GrowPipe &w) {
    cudaStreamSynchronize(w.st);
    cudaFree(w.out_nodes);
    w.out_nodes = nullptr;
    w.out_cap = 0;
}

void pipe_free(GrowPipe &w) {
    cudaFree(w.ctr);
    cudaFree(w.retry_a);
    cudaFree(w.retry_b);
    cudaFree(w.arena);
    cudaFree(w.out_nodes);
    const int sm = w.sm_count;
    const mscd_params p = w.p;
    cudaStream_t st = w.st;
    w = GrowPipe{};
    w.sm_count = sm;
    w.p = p;
    w.st = st;
}

int make_ladder(const DevGraph &G, i64 max_part_n, const mscd_params &p, std::vector<int> *ladder,
                std::vector<bool> *in_smem) {
    const size_t smem_budget = 220 * 1024;
    ladder->clear();
    int c0 = p.smem_slots;
    if (c0 == 0) c0 = grow_state_bytes(G, 1024) * 4 <= smem_budget ? 1024 : 512;
    if (grow_state_bytes(G, c0) > smem_budget) return MSCD_EINVAL;  // one unit's slots must fit a CTA
    ladder->push_back(c0);
    if (p.mid_slots > ladder->back() && grow_state_bytes(G, p.mid_slots) <= smem_budget)
        ladder->push_back(p.mid_slots);
    in_smem->assign(ladder->size(), true);
    // a community stays inside its seed's part: the part size bounds it
    i64 full = 32;
    while (full < max_part_n + 1) full <<= 1;
    i64 cg = ladder->back();
    if (p.global_slots > cg && cg < full) {
        cg = std::min<i64>(p.global_slots, full);
        ladder->push_back((int)cg);
        in_smem->push_back(false);
    }
    while (cg < full) {
        cg = std::min<i64>(cg * 8, full);
        ladder->push_back((int)cg);
        in_smem->push_back(false);
    }
    return MSCD_OK;
}

int grow_units(GrowPipe &w, const GrowArgs &proto, i64 n_units, const std::vector<int> &ladder,
               const std::vector<bool> &in_smem, bool plain, i64 out_budget, i64 max_part_n,
               unsigned long long *cursor_out) {
    const DevGraph &G = proto.G;
    cudaStream_t st = w.st;
    int rc = pipe_reserve(w, n_units);
    if (rc) return rc;
    std::vector<Task> tasks;
    if (n_units > 0) tasks.push_back(Task{0, {}, true});
    unsigned long long cursor = 0;
    while (!tasks.empty() && rc == MSCD_OK) {
        Task t = std::move(tasks.front());
        tasks.erase(tasks.begin());
        const int cap = ladder[t.cls];
        const bool sm = in_smem[t.cls];
        const i64 n_work = t.all ? n_units : (i64)t.units.size();
        // room for every list this launch can write (<= min(cap, n) each) when
        // that fits the budget; otherwise units that find it full are retried
        {
            const i64 bound = (i64)cursor + n_work * std::min<i64>(cap, std::max<i64>(max_part_n, 1));
            const i64 want = std::min<i64>(bound, std::max<i64>(out_budget, (i64)cursor + n_work * 64));
            if ((rc = pipe_output(w, want, (i64)cursor))) break;
        }
        if ((rc = cuda_status(cudaMemsetAsync(w.ctr, 0, sizeof(Counters), st)))) break;
        GrowArgs a = proto;
        a.n_work = n_work;
        a.work_counter = &w.ctr->work;
        a.plain = plain ? 1 : 0;
        if (!t.all) a.unit_base = 0;  // listed items are unit indices
        a.cap = cap;
        a.out_nodes = w.out_nodes;
        a.out_cursor = &w.ctr->out_cursor;
        a.out_needed = &w.ctr->out_needed;
        a.out_cap = w.out_cap;
        a.retry_state = w.retry_a;
        a.n_retry_state = &w.ctr->n_retry_state;
        a.retry_out = w.retry_b;
        a.n_retry_out = &w.ctr->n_retry_out;
        a.error_flags = &w.ctr->error_flags;
        a.state_bytes = grow_state_bytes(G, cap);
        a.big_seed = t.cls == 0 ? proto.big_seed : nullptr;
        a.work_list = nullptr;
        i64 *list_dev = nullptr;
        if (!t.all) {
            if ((rc = cuda_status(cudaMallocAsync((void **)&list_dev, n_work * sizeof(i64), st)))) break;
            if ((rc = cuda_status(cudaMemcpyAsync(list_dev, t.units.data(), n_work * sizeof(i64),
                                                  cudaMemcpyHostToDevice, st))))
                break;
            a.work_list = list_dev;
        }
        // unit lists are appended after everything earlier launches wrote
        if ((rc = cuda_status(cudaMemcpyAsync(&w.ctr->out_cursor, &cursor, sizeof(cursor), cudaMemcpyHostToDevice,
                                              st))))
            break;
        int blocks = 0, threads = 32;
        size_t smem = 0;
        i64 chunk = n_work;  // work items per launch (the plain form's arena bounds it)
        if (sm) {
            // as many one-warp units per CTA as fit 220 KiB (<= 16), one CTA per SM
            a.use_smem = 1;
            a.bounds_smem = 0;
            const int wpc = (int)std::max<size_t>(1, std::min<size_t>(16, (220 * 1024) / a.state_bytes));
            threads = 32 * wpc;
            smem = (size_t)wpc * a.state_bytes;
            int per_sm = 0;
            if ((rc = grow_occupancy(a, threads, smem, &per_sm))) break;
            if (t.cls == 0 && w.p.blocks_per_sm > 0) per_sm = std::min(per_sm, w.p.blocks_per_sm);
            if (per_sm < 1) { rc = MSCD_EINVAL; break; }
            blocks = per_sm * w.sm_count;
        } else {
            a.use_smem = 0;
            a.bounds_smem = 0;
            a.hash_smem = 0;
            int wpc = GLOBAL_CTA_THREADS / 32;
            i64 per_sm_warps = w.p.global_warps_per_sm;
            const size_t hash_bytes = 2 * (size_t)cap * (cap <= 32768 ? 2 : 4);
            const size_t bounds_bytes = 8 * (size_t)(cap / 32);
            if (cap <= w.p.hash_smem_slots) {
                // hash table and bounds in shared memory, slot arrays in the arena:
                // as many warps per CTA (one CTA per SM) as their tables fit
                a.bounds_smem = 1;
                a.hash_smem = 1;
                a.smem_per_warp = (bounds_bytes + hash_bytes + 15) & ~(size_t)15;
                wpc = (int)std::max<size_t>(1, std::min<size_t>(16, (220 * 1024) / a.smem_per_warp));
                smem = (size_t)wpc * a.smem_per_warp;
                per_sm_warps = wpc;
            } else if (cap <= 16384) {
                // group bounds (8 bytes per 32 slots and unit) in shared memory when small
                a.bounds_smem = 1;
                a.smem_per_warp = bounds_bytes;
                smem = (size_t)wpc * a.smem_per_warp;
            }
            const size_t budget = (size_t)4 << 30;
            i64 warps = std::max<i64>(1, std::min<i64>((i64)(budget / a.state_bytes), (i64)w.sm_count * per_sm_warps));
            if (plain) warps = (i64)(budget / a.state_bytes);
            warps = std::max<i64>(1, std::min<i64>(warps, std::max<i64>(n_work, 1)));
            if (plain) chunk = warps;
            threads = (int)std::min<i64>(warps, wpc) * 32;
            blocks = (int)((warps + threads / 32 - 1) / (threads / 32));
            if ((rc = ensure_arena(w, (size_t)blocks * (threads / 32) * a.state_bytes))) break;
            a.gstate = w.arena;
        }
        blocks = (int)std::max<i64>(1, std::min<i64>(blocks, (n_work + threads / 32 - 1) / (threads / 32)));
        cudaEvent_t l0, l1;
        cudaEventCreate(&l0);
        cudaEventCreate(&l1);
        cudaEventRecord(l0, st);
        if (!plain) {
            rc = grow_launch(a, blocks, threads, smem, st);
        } else {
            // one statically mapped unit per warp: a grid over the items
            const int wpc = threads / 32;
            for (i64 b = 0; b < n_work && rc == MSCD_OK; b += chunk) {
                a.work_base = b;
                const i64 items = std::min<i64>(chunk, n_work - b);
                rc = grow_launch(a, (int)((items + wpc - 1) / wpc), threads, smem, st);
            }
        }
        if (rc) {
            cudaEventDestroy(l0);
            cudaEventDestroy(l1);
            break;
        }
        cudaEventRecord(l1, st);
        Counters h{};
        if ((rc = cuda_status(cudaMemcpyAsync(&h, w.ctr, sizeof(h), cudaMemcpyDeviceToHost, st)))) break;
        if ((rc = cuda_status(cudaStreamSynchronize(st)))) break;
        if (w.stats) {
            if (w.stats->grow_launches < 8) {
                const int r = (int)w.stats->grow_launches;
                float lms = 0.0f;
                cudaEventElapsedTime(&lms, l0, l1);
                w.stats->launch_cap[r] = cap;
                w.stats->launch_smem[r] = sm ? 1 : 0;
                w.stats->launch_units[r] = n_work;
                w.stats->launch_ms[r] = lms;
            }
            w.stats->grow_launches++;
        }
        cudaEventDestroy(l0);
        cudaEventDestroy(l1);
        if (list_dev) cudaFreeAsync(list_dev, st);
        if (h.error_flags) { rc = MSCD_EDEVICE; break; }
        if (!h.n_retry_out) {
            cursor = h.out_cursor;
        } else {
            // Reservations are taken in increasing order and every list is
            // non-empty, so once one fails all later ones fail: every
            // written list lies below the old capacity.
            std::vector<i64> lst(h.n_retry_out);
            if ((rc = cuda_status(cudaMemcpyAsync(lst.data(), w.retry_b, lst.size() * sizeof(i64),
                                                  cudaMemcpyDeviceToHost, st))))
                break;
            if ((rc = cuda_status(cudaStreamSynchronize(st)))) break;
            cursor = (unsigned long long)w.out_cap;
            if ((rc = pipe_output(w, w.out_cap + (i64)h.out_needed + (1 << 20), (i64)cursor))) break;
            tasks.insert(tasks.begin(), Task{t.cls, std::move(lst), false});
        }
        if (h.n_retry_state) {
            std::vector<i64> lst(h.n_retry_state);
            if ((rc = cuda_status(cudaMemcpyAsync(lst.data(), w.retry_a, lst.size() * sizeof(i64),
                                                  cudaMemcpyDeviceToHost, st))))
                break;
            if ((rc = cuda_status(cudaStreamSynchronize(st)))) break;
            if (w.stats) w.stats->overflow_units += (i64)lst.size();
            if (t.cls + 1 >= (int)ladder.size()) { rc = MSCD_EDEVICE; break; }
            tasks.push_back(Task{t.cls + 1, std::move(lst), false});
        }
    }
    *cursor_out = cursor;
    return rc;
}
