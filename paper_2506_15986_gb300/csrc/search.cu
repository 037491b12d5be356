// search.cu -- batched best-first beam search (Sec. 2.1, Algorithm 1) on sm_103a.
//
// One warp (a "team") serves one query at a time; a persistent grid sized to
// the SM count pulls queries from a device work queue (one atomic counter), so
// queries of uneven cost and per-query (k, L) share one launch.  Per team the
// shared memory holds:
//   - the query row;
//   - a staging area the neighbour rows are gathered into by bulk copies
//     (cp.async.bulk, one 16-byte-aligned row per copy, completion counted on
//     an mbarrier);
//   - the candidate pool: L 64-bit (distance, id, expanded) keys kept sorted;
//     new candidates are sorted by a warp-shuffle bitonic network and merged
//     in by rank (merge path);
//   - the visited set: an open-addressing hash table (linear probing, key
//     id+1, 0 = empty).  When it would pass 3/4 load, later inserts go to a
//     per-team table in global scratch, so the set stays exact; when that
//     one would pass 3/4 load the query fails with a capacity status.
// Semantics follow the sorted-pool reading of Algorithm 1: single entry, a
// node is visited when its distance is computed, a step expands the first W
// unexpanded pool entries, the pool is truncated to L, the search stops when
// no unexpanded entry is left.  Results are independent of the order in which
// the lanes of a step insert, because the pool is the L smallest keys of the
// union under a total order.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "device_util.cuh"
#include "internal.h"

namespace ann {

namespace {

constexpr int kSearchWarps = 1;  // warps (teams) per CTA
constexpr int kTimeoutIters = 1 << 22;

struct SearchArgs {
    const uint8_t *base;
    const int32_t *graph;
    int64_t n;
    int dim, R, rowbytes;
    const uint8_t *queries;
    int qbytes;
    int64_t nq;
    int64_t qdiv;  // work item i reads query row and target i / qdiv
    const int32_t *entries;
    int32_t medoid;
    int L, k, W;
    const int32_t *dk, *dL, *dtarget;
    int32_t *out_ids;
    void *out_dists;
    int32_t *out_stats;
    int *status;
    unsigned long long *counter;
    uint32_t *spill;
    int hash_bits, spill_bits;
    // per-warp shared-memory layout (byte offsets)
    int off_sel, off_q, off_stage, off_pool, off_ptmp, off_cbuf, off_cids, off_hash, per_warp;
    int stage_rows, stage_stride;
};

__device__ __forceinline__ uint32_t hash_slot(uint32_t key, int bits)
{
    return (key * 0x9E3779B1u) >> (32 - bits);
}

// Visited test-and-insert.  Returns 1 when `id` was not yet visited (and is
// now), 0 when it was, -1 when the table is full (cannot happen below the
// load limits the caller enforces).
__device__ __forceinline__ int visit(uint32_t *htab, int hbits, bool global_mode, uint32_t *gtab,
                                     int gbits, int32_t id)
{
    const uint32_t key = static_cast<uint32_t>(id) + 1u;
    const uint32_t hmask = (1u << hbits) - 1u;
    uint32_t h = hash_slot(key, hbits);
    if (!global_mode) {
        for (uint32_t p = 0; p <= hmask; ++p) {
            uint32_t old = atomicCAS(&htab[h], 0u, key);
            if (old == 0u)
                return 1;
            if (old == key)
                return 0;
            h = (h + 1u) & hmask;
        }
        return -1;
    }
    // shared table is frozen in global mode: lookup only
    for (uint32_t p = 0; p <= hmask; ++p) {
        uint32_t v = htab[h];
        if (v == key)
            return 0;
        if (v == 0u)
            break;
        h = (h + 1u) & hmask;
    }
    const uint32_t gmask = (1u << gbits) - 1u;
    uint32_t g = hash_slot(key, gbits);
    for (uint32_t p = 0; p <= gmask; ++p) {
        uint32_t old = atomicCAS(&gtab[g], 0u, key);
        if (old == 0u)
            return 1;
        if (old == key)
            return 0;
        g = (g + 1u) & gmask;
    }
    return -1;
}

// distance of one staged row to the query, as order-preserving key bits
template <int DT, int MT>
__device__ __forceinline__ uint32_t row_distance(const uint8_t *row, const uint8_t *q, int dim)
{
    if constexpr (DT == ANN_U8) {
        const uint4 *x4 = reinterpret_cast<const uint4 *>(row);
        const uint4 *q4 = reinterpret_cast<const uint4 *>(q);
        uint32_t acc = 0;
        for (int c = 0; c < dim / 16; ++c) {
            uint4 x = x4[c], y = q4[c];
            uint32_t d;
            d = __vabsdiffu4(x.x, y.x);
            acc = __dp4a(d, d, acc);
            d = __vabsdiffu4(x.y, y.y);
            acc = __dp4a(d, d, acc);
            d = __vabsdiffu4(x.z, y.z);
            acc = __dp4a(d, d, acc);
            d = __vabsdiffu4(x.w, y.w);
            acc = __dp4a(d, d, acc);
        }
        return acc;  // exact non-negative int32, ordered as unsigned
    } else {
        const float4 *q4 = reinterpret_cast<const float4 *>(q);
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        auto acc4 = [&](float x0, float x1, float x2, float x3, float4 y) {
            if constexpr (MT == ANN_L2) {
                float d0 = x0 - y.x, d1 = x1 - y.y, d2 = x2 - y.z, d3 = x3 - y.w;
                a0 = fmaf(d0, d0, a0);
                a1 = fmaf(d1, d1, a1);
                a2 = fmaf(d2, d2, a2);
                a3 = fmaf(d3, d3, a3);
            } else {
                a0 = fmaf(x0, y.x, a0);
                a1 = fmaf(x1, y.y, a1);
                a2 = fmaf(x2, y.z, a2);
                a3 = fmaf(x3, y.w, a3);
            }
        };
        if constexpr (DT == ANN_F32) {
            const float4 *x4 = reinterpret_cast<const float4 *>(row);
            for (int c = 0; c < dim / 4; ++c) {
                float4 x = x4[c];
                acc4(x.x, x.y, x.z, x.w, q4[c]);
            }
        } else {
            const uint4 *x8 = reinterpret_cast<const uint4 *>(row);
            for (int c = 0; c < dim / 8; ++c) {
                uint4 x = x8[c];
                float2 f0, f1, f2, f3;
                if constexpr (DT == ANN_F16) {
                    f0 = __half22float2(*reinterpret_cast<const __half2 *>(&x.x));
                    f1 = __half22float2(*reinterpret_cast<const __half2 *>(&x.y));
                    f2 = __half22float2(*reinterpret_cast<const __half2 *>(&x.z));
                    f3 = __half22float2(*reinterpret_cast<const __half2 *>(&x.w));
                } else {
                    f0 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&x.x));
                    f1 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&x.y));
                    f2 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&x.z));
                    f3 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&x.w));
                }
                acc4(f0.x, f0.y, f1.x, f1.y, q4[2 * c]);
                acc4(f2.x, f2.y, f3.x, f3.y, q4[2 * c + 1]);
            }
        }
        float s = (a0 + a1) + (a2 + a3);
        if constexpr (MT == ANN_IP)
            s = -s;
        return f32_to_ord(s);
    }
}

template <int DT, int MT>
__global__ void __launch_bounds__(32 * kSearchWarps) beam_search_kernel(const SearchArgs a)
{
    extern __shared__ __align__(128) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    uint8_t *my = smem + wid * a.per_warp;
    uint64_t *bar = reinterpret_cast<uint64_t *>(my);
    int32_t *sel = reinterpret_cast<int32_t *>(my + a.off_sel);
    uint8_t *qbuf = my + a.off_q;
    uint8_t *stage = my + a.off_stage;
    uint64_t *pool = reinterpret_cast<uint64_t *>(my + a.off_pool);
    uint64_t *ptmp = reinterpret_cast<uint64_t *>(my + a.off_ptmp);
    uint64_t *cbuf = reinterpret_cast<uint64_t *>(my + a.off_cbuf);
    int32_t *cids = reinterpret_cast<int32_t *>(my + a.off_cids);
    uint32_t *htab = reinterpret_cast<uint32_t *>(my + a.off_hash);
    const int team = blockIdx.x * kSearchWarps + wid;
    uint32_t *gtab = a.spill + (static_cast<size_t>(team) << a.spill_bits);

    if (lane == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint32_t phase = 0;
    const int hcap = 1 << a.hash_bits;
    const int hlimit = hcap * 3 / 4;
    const int glimit = (1 << a.spill_bits) * 3 / 4;

    for (;;) {
        long long qi = 0;
        if (lane == 0)
            qi = static_cast<long long>(atomicAdd(a.counter, 1ull));
        qi = __shfl_sync(kFull, qi, 0);
        if (qi >= a.nq)
            break;

        const int Lq = a.dL ? a.dL[qi] : a.L;
        const int kq = a.dk ? a.dk[qi] : a.k;
        const int64_t qrow = qi / a.qdiv;
        const int32_t target = a.dtarget ? a.dtarget[qrow] : -1;
        const int32_t entry = a.entries ? a.entries[qi] : a.medoid;
        bool failed = false;
        bool timed_out = false;
        if (Lq < 1 || Lq > a.L || kq < 1 || kq > a.k || kq > Lq || entry < 0 || entry >= a.n) {
            failed = true;
            if (lane == 0)
                atomicOr(a.status, kStatusBadInputBit);
        }

        int cnt = 0, cursor = 0, evals = 0, hops = 0, hused = 0, gused = 0;
        bool gmode = false, found = false;
        if (!failed) {
            // query row -> shared memory; clear the visited table
            const uint8_t *qsrc = a.queries + qrow * a.qbytes;
            for (int o = lane * 16; o < a.qbytes; o += 32 * 16)
                *reinterpret_cast<uint4 *>(qbuf + o) = *reinterpret_cast<const uint4 *>(qsrc + o);
            for (int o = lane; o < hcap / 4; o += 32)
                reinterpret_cast<uint4 *>(htab)[o] = make_uint4(0u, 0u, 0u, 0u);
            __syncwarp();
            if (lane == 0) {
                visit(htab, a.hash_bits, false, gtab, a.spill_bits, entry);
                cids[0] = entry;
            }
            hused = 1;
            evals = 1;
            found = (entry == target);
        }
        int nc = failed ? 0 : 1;
        __syncwarp();

        while (!failed) {
            // ---- evaluate the nc candidates in cids[] and merge them into the pool
            if (nc > 0) {
                for (int c0 = 0; c0 < nc; c0 += a.stage_rows) {
                    const int ch = min(a.stage_rows, nc - c0);
                    if (lane == 0)
                        mbar_arrive_expect_tx(bar, static_cast<uint32_t>(ch) * a.rowbytes);
                    __syncwarp();
                    for (int j = lane; j < ch; j += 32)
                        bulk_g2s(stage + j * a.stage_stride,
                                 a.base + static_cast<size_t>(cids[c0 + j]) * a.rowbytes,
                                 a.rowbytes, bar);
                    bool ok = mbar_wait_bounded(bar, phase, kTimeoutIters);
                    if (!__all_sync(kFull, ok)) {
                        // give the copies one more bounded chance, then retire this team
                        mbar_wait_bounded(bar, phase, kTimeoutIters);
                        timed_out = true;
                        failed = true;
                        break;
                    }
                    phase ^= 1u;
                    for (int j = lane; j < ch; j += 32)
                        cbuf[c0 + j] = make_key(
                            row_distance<DT, MT>(stage + j * a.stage_stride, qbuf, a.dim), cids[c0 + j]);
                    __syncwarp();
                    fence_proxy_async_smem();  // stage reads done before the next bulk writes
                }
                if (failed)
                    break;
                uint64_t k0 = lane < nc ? cbuf[lane] : kKeyMax;
                uint64_t k1 = lane + 32 < nc ? cbuf[lane + 32] : kKeyMax;
                const uint64_t worst = (cnt == Lq) ? key_plain(pool[Lq - 1]) : kKeyMax;
                if (k0 >= worst)
                    k0 = kKeyMax;
                if (k1 >= worst)
                    k1 = kKeyMax;
                if (nc > 32)
                    warp_sort64(k0, k1, lane);
                else
                    k0 = warp_sort32(k0, lane);
                const int m = __popc(__ballot_sync(kFull, k0 != kKeyMax)) +
                              __popc(__ballot_sync(kFull, k1 != kKeyMax));
                __syncwarp();
                if (m > 0) {
                    cbuf[lane] = k0;
                    cbuf[lane + 32] = k1;
                    __syncwarp();
                    const int p0 = count_less(pool, cnt, cbuf[0]);
                    const int mv = cnt - p0;
                    for (int i = lane; i < mv; i += 32)
                        ptmp[i] = pool[p0 + i];
                    __syncwarp();
                    for (int i = lane; i < mv; i += 32) {
                        const uint64_t v = ptmp[i];
                        const int np = p0 + i + count_less(cbuf, m, key_plain(v));
                        if (np < Lq)
                            pool[np] = v;
                    }
                    for (int j = lane; j < m; j += 32) {
                        const uint64_t v = cbuf[j];
                        const int np = p0 + j + count_less(ptmp, mv, v);
                        if (np < Lq)
                            pool[np] = v;
                    }
                    __syncwarp();
                    cnt = min(Lq, cnt + m);
                    cursor = min(cursor, p0);
                }
            }
            if (found)
                break;

            // ---- select the first W unexpanded pool entries
            int ns = 0, first = -1;
            for (int i0 = cursor; i0 < cnt && ns < a.W; i0 += 32) {
                const int i = i0 + lane;
                const bool un = i < cnt && !(pool[i] & 1ull);
                const unsigned um = __ballot_sync(kFull, un);
                if (um) {
                    if (first < 0)
                        first = i0 + __ffs(um) - 1;
                    const int rank = __popc(um & lanemask_lt());
                    if (un && ns + rank < a.W) {
                        const uint64_t v = pool[i];
                        pool[i] = v | 1ull;
                        sel[ns + rank] = key_id(v);
                    }
                    ns = min(a.W, ns + __popc(um));
                }
            }
            __syncwarp();
            if (ns == 0)
                break;
            cursor = first;
            hops += ns;

            // ---- neighbours of the selected entries: visited test, compaction
            const int total = ns * a.R;
            if (!gmode && hused + total > hlimit) {
                gmode = true;  // freeze the shared table, continue in global scratch
                for (int o = lane; o < (1 << a.spill_bits) / 4; o += 32)
                    reinterpret_cast<uint4 *>(gtab)[o] = make_uint4(0u, 0u, 0u, 0u);
                __syncwarp();
            }
            if (gmode && gused + total > glimit) {
                failed = true;
                if (lane == 0)
                    atomicOr(a.status, kStatusCapacityBit);
                break;
            }
            nc = 0;
            bool bad = false;
            for (int t0 = 0; t0 < total; t0 += 32) {
                const int t = t0 + lane;
                int32_t id = -1;
                if (t < total) {
                    const int s = t / a.R;
                    id = __ldg(a.graph + static_cast<int64_t>(sel[s]) * a.R + (t - s * a.R));
                }
                int r = 0;
                if (id >= 0 && id < a.n)
                    r = visit(htab, a.hash_bits, gmode, gtab, a.spill_bits, id);
                bad |= (r < 0);
                const unsigned nm = __ballot_sync(kFull, r == 1);
                if (r == 1) {
                    cids[nc + __popc(nm & lanemask_lt())] = id;
                    if (id == target)
                        found = true;
                }
                nc += __popc(nm);
            }
            found = __any_sync(kFull, found);
            if (__any_sync(kFull, bad)) {
                failed = true;
                if (lane == 0)
                    atomicOr(a.status, kStatusCapacityBit);
                break;
            }
            evals += nc;
            if (gmode)
                gused += nc;
            else
                hused += nc;
            __syncwarp();
        }

        if (timed_out && lane == 0)
            atomicOr(a.status, kStatusTimeoutBit);

        // ---- outputs
        for (int j = lane; j < a.k; j += 32) {
            int32_t id = -1;
            uint32_t db = 0;
            if (!failed && j < kq && j < cnt) {
                const uint64_t v = pool[j];
                id = key_id(v);
                db = static_cast<uint32_t>(v >> 32);
            }
            a.out_ids[qi * a.k + j] = id;
            if constexpr (DT == ANN_U8)
                reinterpret_cast<int32_t *>(a.out_dists)[qi * a.k + j] =
                    id >= 0 ? static_cast<int32_t>(db) : INT32_MAX;
            else
                reinterpret_cast<float *>(a.out_dists)[qi * a.k + j] =
                    id >= 0 ? ord_to_f32(db) : __int_as_float(0x7f800000);
        }
        if (a.out_stats && lane == 0) {
            const bool miss = failed || (target >= 0 && !found);
            a.out_stats[2 * qi] = miss && target >= 0 ? INT32_MAX : evals;
            a.out_stats[2 * qi + 1] = miss && target >= 0 ? INT32_MAX : hops;
        }
        __syncwarp();
        if (timed_out)
            return;  // this team's barrier state is unknown: retire it
    }
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

template <int DT, int MT>
ann_status teams_for(ann_index *idx, size_t smem, int *teams)
{
    auto kern = beam_search_kernel<DT, MT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess)
        return cuda_status(e);
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * kSearchWarps, smem);
    if (e != cudaSuccess)
        return cuda_status(e);
    if (per_sm < 1)
        return ANN_ERR_UNSUPPORTED;  // the per-query state does not fit in shared memory
    *teams = per_sm * idx->num_sms * kSearchWarps;
    return ANN_OK;
}

template <int DT, int MT>
ann_status launch_typed(const SearchArgs &a, size_t smem, int teams, cudaStream_t s)
{
    const int grid = (teams + kSearchWarps - 1) / kSearchWarps;
    beam_search_kernel<DT, MT><<<grid, 32 * kSearchWarps, smem, s>>>(a);
    return cuda_status(cudaGetLastError());
}

#define ANN_DISPATCH(FN, ...)                                                        \
    switch (idx->dtype * 2 + idx->metric) {                                          \
    case ANN_U8 * 2 + ANN_L2: st = FN<ANN_U8, ANN_L2>(__VA_ARGS__); break;           \
    case ANN_F32 * 2 + ANN_L2: st = FN<ANN_F32, ANN_L2>(__VA_ARGS__); break;         \
    case ANN_F32 * 2 + ANN_IP: st = FN<ANN_F32, ANN_IP>(__VA_ARGS__); break;         \
    case ANN_F16 * 2 + ANN_L2: st = FN<ANN_F16, ANN_L2>(__VA_ARGS__); break;         \
    case ANN_F16 * 2 + ANN_IP: st = FN<ANN_F16, ANN_IP>(__VA_ARGS__); break;         \
    case ANN_BF16 * 2 + ANN_L2: st = FN<ANN_BF16, ANN_L2>(__VA_ARGS__); break;       \
    case ANN_BF16 * 2 + ANN_IP: st = FN<ANN_BF16, ANN_IP>(__VA_ARGS__); break;       \
    default: st = ANN_ERR_UNSUPPORTED; break;                                        \
    }

}  // namespace

size_t search_scratch_bytes(int teams, int spill_bits)
{
    return 256 + static_cast<size_t>(teams) * (static_cast<size_t>(4) << spill_bits);
}

ann_status launch_search(ann_index *idx, const SearchLaunch &L, cudaStream_t s)
{
    const ann_search_params *p = L.p;
    SearchArgs a{};
    a.base = static_cast<const uint8_t *>(idx->d_base);
    a.graph = idx->d_graph;
    a.n = idx->n;
    a.dim = idx->dim;
    a.R = idx->degree;
    a.rowbytes = idx->rowbytes;
    a.queries = static_cast<const uint8_t *>(L.queries);
    a.qbytes = L.qbytes;
    a.nq = L.nq;
    a.qdiv = L.qdiv > 0 ? L.qdiv : 1;
    a.entries = L.entries;
    a.medoid = idx->medoid;
    a.L = p->L;
    a.k = p->k;
    a.W = p->W;
    a.dk = p->d_k;
    a.dL = p->d_L;
    a.dtarget = p->d_target;
    a.out_ids = L.ids;
    a.out_dists = L.dists;
    a.out_stats = L.stats;
    a.status = idx->d_status;

    int hb = p->hash_bits;
    if (hb == 0) {
        // searches evaluate about 10-16 nodes per pool slot; size the shared
        // table for 16 per slot below its 3/4 load limit (the exact global
        // spill table takes any excess)
        hb = 10;
        while ((1 << hb) * 3 / 4 < 16 * p->L && hb < 13)
            ++hb;
    }
    a.hash_bits = hb;
    a.spill_bits = 15;

    const int maxc = p->W * idx->degree;
    int s16 = idx->rowbytes / 16;
    if ((s16 & 1) == 0)
        s16 += 1;  // odd 16-byte stride: 8-lane phases of 16-byte loads hit distinct banks
    a.stage_stride = s16 * 16;
    // Most steps find far fewer new neighbours than W * R (about 9 of 32 on
    // average), so 16 rows per gather round keep shared memory per team small
    // (more teams per SM); at most 48 KB staged at once, which also keeps one
    // mbarrier phase's byte count far below its 2^20 limit.
    a.stage_rows = std::max(1, std::min({maxc, 16, 49152 / a.stage_stride}));

    size_t off = 16;  // mbarrier
    a.off_sel = static_cast<int>(off);
    off = align_up(off + 4 * ANN_MAX_W, 16);
    a.off_q = static_cast<int>(off);
    off = align_up(off + L.qbytes, 16);
    a.off_stage = static_cast<int>(off);
    off = align_up(off + static_cast<size_t>(a.stage_rows) * a.stage_stride, 16);
    a.off_pool = static_cast<int>(off);
    off = align_up(off + 8 * static_cast<size_t>(p->L), 16);
    a.off_ptmp = static_cast<int>(off);
    off = align_up(off + 8 * static_cast<size_t>(p->L), 16);
    a.off_cbuf = static_cast<int>(off);
    off = align_up(off + 8 * ANN_MAX_STEP_CAND, 16);
    a.off_cids = static_cast<int>(off);
    off = align_up(off + 4 * ANN_MAX_STEP_CAND, 16);
    a.off_hash = static_cast<int>(off);
    off = align_up(off + (static_cast<size_t>(4) << hb), 128);
    a.per_warp = static_cast<int>(off);
    const size_t smem = off * kSearchWarps;

    // persistent grid: occupancy-limited, at most one team per query
    int teams = 0;
    ann_status st = ANN_OK;
    ANN_DISPATCH(teams_for, idx, smem, &teams);
    if (st != ANN_OK)
        return st;
    if (L.max_teams > 0)
        teams = std::min(teams, L.max_teams);
    teams = static_cast<int>(std::min<long long>(teams, L.nq));
    if (teams < 1)
        return ANN_OK;

    // scratch: work counter, then one spill table per team
    const size_t need = search_scratch_bytes(teams, a.spill_bits);
    void *scratch = L.scratch;
    const bool own = scratch == nullptr;
    if (own) {
        st = scratch_alloc(idx, need, s, &scratch);
        if (st != ANN_OK)
            return st;
    } else if (L.scratch_bytes < need) {
        return ANN_ERR_CAPACITY;
    }
    a.counter = static_cast<unsigned long long *>(scratch);
    a.spill = reinterpret_cast<uint32_t *>(static_cast<uint8_t *>(scratch) + 256);
    cudaError_t e = cudaMemsetAsync(scratch, 0, 8, s);
    if (e == cudaSuccess) {
        ANN_DISPATCH(launch_typed, a, smem, teams, s);
    } else {
        st = cuda_status(e);
    }
    if (own)
        scratch_free(idx, scratch, s);
    return st;
}

}  // namespace ann
