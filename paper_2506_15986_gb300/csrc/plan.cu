// plan.cu -- batching line: one batch of entry selection + search captured in
// a CUDA graph (relaunched without host-side launch work), and an autotuner
// for the knobs that change speed but never results.
#include <cuda_runtime.h>
#include <stdint.h>

#include <new>
#include <vector>

#include "internal.h"

struct ann_plan {
    int device = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

using namespace ann;

extern "C" {

ann_status ann_plan_create(ann_index *idx, const void *d_queries, int64_t nq, int32_t entry_mode, int32_t L_hub,
                           const ann_search_params *p, int32_t *d_entry_buf, int32_t *d_ids, void *d_dists,
                           int32_t *d_stats, ann_plan **out)
{
    if (!idx || !p || !out || nq < 1 || (entry_mode != ANN_ENTRY_MEDOID && !d_entry_buf))
        return ANN_ERR_INVALID_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(idx->device);
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaSetDevice(prev);
        return cuda_status(e);
    }
    ann_plan *plan = new (std::nothrow) ann_plan();
    if (!plan) {
        cudaStreamDestroy(s);
        cudaSetDevice(prev);
        return ANN_ERR_OOM;
    }
    plan->device = idx->device;
    ann_status st = cuda_status(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    ann_status st2 = ANN_OK;
    if (st == ANN_OK) {
        const int32_t *entry = nullptr;
        if (entry_mode != ANN_ENTRY_MEDOID) {
            st2 = ann_select_entries(idx, d_queries, nq, entry_mode, L_hub, p->n_entries > 1 ? p->n_entries : 1,
                                     d_entry_buf, nullptr, s);
            entry = d_entry_buf;
        }
        if (st2 == ANN_OK)
            st2 = ann_search_batch(idx, d_queries, nq, entry, p, d_ids, d_dists, d_stats, s);
        st = cuda_status(cudaStreamEndCapture(s, &plan->graph));
    }
    if (st == ANN_OK && st2 == ANN_OK)
        st = cuda_status(cudaGraphInstantiate(&plan->exec, plan->graph, 0));
    cudaStreamDestroy(s);
    cudaSetDevice(prev);
    if (st2 != ANN_OK)
        st = st2;
    if (st != ANN_OK) {
        if (plan->exec)
            cudaGraphExecDestroy(plan->exec);
        if (plan->graph)
            cudaGraphDestroy(plan->graph);
        delete plan;
        return st;
    }
    *out = plan;
    return ANN_OK;
}

ann_status ann_plan_launch(ann_plan *plan, void *stream)
{
    if (!plan)
        return ANN_ERR_INVALID_ARG;
    return cuda_status(cudaGraphLaunch(plan->exec, static_cast<cudaStream_t>(stream)));
}

ann_status ann_plan_free(ann_plan *plan)
{
    if (!plan)
        return ANN_OK;
    cudaDeviceSynchronize();
    if (plan->exec)
        cudaGraphExecDestroy(plan->exec);
    if (plan->graph)
        cudaGraphDestroy(plan->graph);
    delete plan;
    return ANN_OK;
}

ann_status ann_autotune(ann_index *idx, const void *d_queries, int64_t nq, const int32_t *d_entry,
                        const ann_search_params *p, int32_t *d_ids, void *d_dists, int32_t reps, int32_t lanes,
                        ann_search_params *best, float *best_ms, void *stream)
{
    if (!idx || !p || !best || nq < 1 || reps < 1 || lanes < 1 || lanes > 8 || p->k < 1)
        return ANN_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(idx->device);
    ann_status st = ANN_OK;
    // lane 0 is the caller's stream and buffers; every other lane has its own
    // stream and output buffers from the index's pool
    std::vector<cudaStream_t> ls(lanes, s);
    std::vector<cudaEvent_t> joins(lanes, nullptr);
    std::vector<int32_t *> lids(lanes, d_ids);
    std::vector<void *> ldists(lanes, d_dists);
    cudaEvent_t e0 = nullptr, e1 = nullptr, fork = nullptr;
    void *extra = nullptr;
    const size_t ob = static_cast<size_t>(nq) * p->k * 4;  // ids; distances are 4 bytes for every dtype
    st = cuda_status(cudaEventCreate(&e0));
    if (st == ANN_OK)
        st = cuda_status(cudaEventCreate(&e1));
    if (st == ANN_OK)
        st = cuda_status(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    if (st == ANN_OK && lanes > 1)
        st = scratch_alloc(idx, 2 * ob * (lanes - 1), s, &extra);
    for (int i = 1; i < lanes && st == ANN_OK; ++i) {
        st = cuda_status(cudaStreamCreateWithFlags(&ls[i], cudaStreamNonBlocking));
        if (st == ANN_OK)
            st = cuda_status(cudaEventCreateWithFlags(&joins[i], cudaEventDisableTiming));
        lids[i] = reinterpret_cast<int32_t *>(static_cast<uint8_t *>(extra) + 2 * ob * (i - 1));
        ldists[i] = static_cast<uint8_t *>(extra) + 2 * ob * (i - 1) + ob;
    }
    // the other lanes start after what the caller's stream holds so far
    auto fork_lanes = [&](cudaEvent_t ev) {
        for (int i = 1; i < lanes; ++i)
            cudaStreamWaitEvent(ls[i], ev, 0);
    };
    auto join_lanes = [&]() {
        for (int i = 1; i < lanes; ++i) {
            cudaEventRecord(joins[i], ls[i]);
            cudaStreamWaitEvent(s, joins[i], 0);
        }
    };
    // visited-table sizes around the default, and gather round sizes
    int hb0 = 10;
    while ((1 << hb0) * 3 / 4 < 12 * p->L && hb0 < 13)
        ++hb0;
    std::vector<int> hbs = {-1};  // -1: no shared table
    for (int hb = hb0 - 3; hb <= hb0; ++hb)
        if (hb >= 8 && hb <= 15)
            hbs.push_back(hb);
    const int srs[] = {4, 6, 8, 12, 16};
    float bms = 1e30f;
    ann_search_params bp = *p;
    // times one candidate: reps batches, batch r on lane r mod lanes; false on
    // a hard error (st set)
    auto trial = [&](const ann_search_params &c) -> bool {
        cudaEventRecord(fork, s);
        fork_lanes(fork);
        for (int i = 0; i < lanes && st == ANN_OK; ++i)  // warm-up
            st = ann_search_batch(idx, d_queries, nq, d_entry, &c, lids[i], ldists[i], nullptr, ls[i]);
        join_lanes();
        if (st == ANN_ERR_UNSUPPORTED) {  // does not fit in shared memory
            st = ANN_OK;
            return true;
        }
        if (st != ANN_OK)
            return false;
        cudaEventRecord(e0, s);
        fork_lanes(e0);
        for (int r = 0; r < reps && st == ANN_OK; ++r)
            st = ann_search_batch(idx, d_queries, nq, d_entry, &c, lids[r % lanes], ldists[r % lanes], nullptr,
                                  ls[r % lanes]);
        join_lanes();
        cudaEventRecord(e1, s);
        if (st != ANN_OK)
            return false;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = ANN_ERR_CUDA;
            return false;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        if (ms < bms) {
            bms = ms;
            bp = c;
        }
        return true;
    };
    bool ok = st == ANN_OK;
    // stage 1: visited-table size x gather round size at the given team size
    for (size_t h = 0; ok && h < hbs.size(); ++h) {
        for (int sr : srs) {
            ann_search_params c = *p;
            c.hash_bits = hbs[h];
            c.stage_rows = sr;
            c.team = p->team > 0 ? p->team : ann::default_team(idx->rowbytes);
            if (!(ok = trial(c)))
                break;
        }
    }
    // stage 2: team sizes at the best pair, from 1 to 16 chunks of the row per lane
    const int chunks = idx->rowbytes / 16;
    const ann_search_params b1 = bp;
    for (int g = 2; ok && g <= 32; g <<= 1) {
        if (g > chunks || g * 16 < chunks || g == b1.team)
            continue;
        ann_search_params c = b1;
        c.team = g;
        ok = trial(c);
    }
    // stage 3: first spill tables one and two sizes either side of the
    // default at the best so far (larger: fewer collisions; smaller: less to
    // clear; the second table takes the tail)
    const ann_search_params b2 = bp;
    const int sb0 = b2.spill_bits > 0 ? b2.spill_bits : ann::default_spill_bits(p->L);
    for (int sb = sb0 - 2; ok && sb <= sb0 + 2; ++sb) {
        if (sb < 10 || sb > 16 || sb == sb0)
            continue;
        ann_search_params c = b2;
        c.spill_bits = sb;
        ok = trial(c);
    }
    // stage 4: four-row TMA tensor gathers (when the index's rows allow
    // them) at the best sizes so far, with larger rounds and eight-lane
    // distance teams (the gathered rows are unpadded, so small teams read
    // them with bank conflicts)
    if (idx->has_row_map) {
        const ann_search_params b3 = bp;
        const int teams[2] = {b3.team > 0 ? b3.team : ann::default_team(idx->rowbytes), 8};
        for (int sr : {8, 12, 16}) {
            for (int ti = 0; ti < 2 && ok; ++ti) {
                if (ti == 1 && teams[1] == teams[0])
                    continue;
                ann_search_params c = b3;
                c.gather = 4;
                c.stage_rows = sr;
                c.team = teams[ti];
                ok = trial(c);
            }
        }
    }
    // stage 5: first-level visited tables kept resident in L2 (applied by
    // the launch only when they fit the persisting-L2 capacity), at the best
    // table size so far and one and two sizes smaller; the lines a trial
    // leaves persisting are released before the next trial, so no other
    // candidate is timed with a smaller L2
    {
        const ann_search_params b4 = bp;
        const int sbb = b4.spill_bits > 0 ? b4.spill_bits : ann::default_spill_bits(p->L);
        for (int sb = sbb; ok && sb >= sbb - 2; --sb) {
            if (sb < 10 || sb > 16)
                continue;
            ann_search_params c = b4;
            c.flags |= ANN_SEARCH_VISITED_L2;
            c.spill_bits = sb;
            ok = trial(c);
            if (ann_release_l2(idx) != ANN_OK) {
                st = ANN_ERR_CUDA;
                ok = false;
            }
        }
    }
    // stage 6: with entries given, the work order grouped by first seed at
    // the best so far
    if (ok && d_entry) {
        ann_search_params c = bp;
        c.flags |= ANN_SEARCH_GROUP_ENTRIES;
        ok = trial(c);
        if ((c.flags & ANN_SEARCH_VISITED_L2) && ann_release_l2(idx) != ANN_OK) {
            st = ANN_ERR_CUDA;
            ok = false;
        }
    }
    // the caller's outputs hold the chosen combination's results; lines it
    // leaves persisting are released (the caller's own searches with the
    // chosen flags make them resident again)
    if (ok && bms < 1e30f)
        st = ann_search_batch(idx, d_queries, nq, d_entry, &bp, d_ids, d_dists, nullptr, s);
    if (st == ANN_OK && (bp.flags & ANN_SEARCH_VISITED_L2))
        st = ann_release_l2(idx);
    for (int i = 1; i < lanes; ++i)
        if (ls[i] != s) {
            cudaStreamSynchronize(ls[i]);
            cudaStreamDestroy(ls[i]);
        }
    if (extra)
        scratch_free(idx, extra, s);
    if (st == ANN_OK)
        st = cuda_status(cudaStreamSynchronize(s));
    for (int i = 1; i < lanes; ++i)
        if (joins[i])
            cudaEventDestroy(joins[i]);
    if (fork)
        cudaEventDestroy(fork);
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    cudaSetDevice(prev);
    if (st != ANN_OK)
        return st;
    *best = bp;
    if (best_ms)
        *best_ms = bms;
    return ANN_OK;
}

}  // extern "C"
