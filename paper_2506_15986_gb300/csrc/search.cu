// search.cu -- batched best-first beam search (Sec. 2.1, Algorithm 1) on sm_103a.
//
// One warp (a "team") serves one query at a time; a persistent grid sized to
// the SM count pulls queries from a device work queue (one atomic counter), so
// queries of uneven cost and per-query (k, L) share one launch.  Optionally
// the queue hands the queries out grouped by their first seed (a counting sort
// by a hash of the seed), so that queries that start at the same node run at
// the same time and share the rows of their first steps in L2.  Per team the
// shared memory holds:
//   - the query row;
//   - a staging area the neighbour rows are gathered into by bulk copies
//     (cp.async.bulk, one 16-byte-aligned row per copy, completion counted on
//     an mbarrier);
//   - the candidate pool: L 64-bit (distance, id, expanded) keys kept sorted;
//     new candidates are sorted by a warp-shuffle bitonic network and merged
//     in by rank (merge path);
//   - optionally, the first level of the visited set (hash_bits > 0).
// The visited set is an exact open-addressing hash (linear probing, key id+1,
// 0 = empty) with up to three levels: the optional shared-memory table, a
// per-team table in global scratch (2^spill_bits slots), and one four times
// larger.  A level that would pass 3/4 load hands its keys to the next one,
// which takes every later insert; only past the last does the query fail
// with a capacity status.  Without a shared table (hash_bits = -1, what the
// tuned configurations use) the set starts in the first global table.
// Semantics follow the sorted-pool reading of Algorithm 1: a seed set (one
// entry by default), a node is visited when its distance is computed, a step
// expands the first W unexpanded pool entries, the pool is truncated to L,
// the search stops when no unexpanded entry is left.  Results are
// independent of the order in which the lanes of a step insert, because the
// pool is the L smallest keys of the union under a total order.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "device_util.cuh"
#include "internal.h"

namespace ann {

namespace {

constexpr int kMaxSearchWarps = 2;  // warps (teams) per CTA: 1 or 2, whichever fits more teams
constexpr int kTimeoutIters = 1 << 22;
constexpr int kSlots = ANN_MAX_STEP_CAND / 32;  // neighbour slots per lane in one step

struct SearchArgs {
    CUtensorMap row_map;  // four-row TMA gathers of base rows (gather4 only)
    int gather4;          // 1: a round's rows come in TMA tensor gathers of four
    int nteams;           // teams of the launch (the first-level tables come first in the scratch)
    const uint8_t *base;
    const int32_t *graph;
    int64_t n;
    int dim, R, rowbytes;
    int R_inv;  // ceil(2^16 / R): (t * R_inv) >> 16 == t / R for all t < 128, 1 <= R <= 128
    const uint8_t *queries;
    int qbytes;
    int qpad;  // zero bytes after the query row in shared memory
    int64_t nq;
    int64_t qdiv;          // work item i reads query row and target i / qdiv
    const int32_t *order;  // optional: the w-th item taken from the queue is order[w]
    const int32_t *entries;
    int32_t medoid;
    int L, k, W;
    int n_entries;   // seeds per query in entries[] (1 when entries is null: the medoid)
    int fault_wait;  // fault injection: every bulk-copy wait gives up at once
    const int32_t *dk, *dL, *dtarget;
    int32_t *out_ids;
    void *out_dists;
    int32_t *out_stats;
    int32_t *pool_out;  // optional: the whole final pool (nq x L ids, -1 padded)
    int *status;
    unsigned long long *counter;
    uint32_t *spill;
    int hash_bits, spill_bits;
    // per-warp shared-memory layout (byte offsets)
    int off_sel, off_q, off_stage, off_pool, off_ptop, off_cbuf, off_hash, per_warp;
    int stage_rows, stage_stride;
    int team_lg;  // log2 of the lanes computing one distance
    int cpl;      // 8 when a row is exactly 8 16-byte chunks per lane (unrolled), else 0
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
    if (!global_mode) {
        const uint32_t hmask = (1u << hbits) - 1u;
        uint32_t h = hash_slot(key, hbits);
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
    // global mode: the set lives in a global table (after a spill, or from
    // the start when there is no shared table)
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

// Visited test-and-insert for NS ids per lane (-1 = none) in one table.
// res[s] = 1 when ids[s] was not yet visited (and is now), 0 when it was, -1
// when the table is full.  All first probes go out before any result is
// used, and the collision chains of all slots advance together, so their
// latencies overlap.  Concurrent inserts of the same id (from any lane or
// slot) give exactly one 1: every insert of a key walks the same probe
// sequence and the compare-and-swap decides each slot once.
template <int NS>
__device__ __forceinline__ void visit_slots(uint32_t *tab, int bits, const int32_t (&ids)[NS], int (&res)[NS])
{
    const uint32_t mask = (1u << bits) - 1u;
    uint32_t h[NS], key[NS], old[NS];
    // issue every compare-and-swap before looking at any result
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        key[s] = static_cast<uint32_t>(ids[s]) + 1u;
        h[s] = hash_slot(key[s], bits);
        old[s] = ids[s] >= 0 ? atomicCAS(&tab[h[s]], 0u, key[s]) : 0u;
    }
    bool more = false;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        res[s] = ids[s] < 0 ? 0 : (old[s] == 0u ? 1 : (old[s] == key[s] ? 0 : 2));
        more |= res[s] == 2;
    }
    for (uint32_t p = 1; p <= mask && more; ++p) {
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            if (res[s] == 2) {
                h[s] = (h[s] + 1u) & mask;
                old[s] = atomicCAS(&tab[h[s]], 0u, key[s]);
            }
        }
        more = false;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            if (res[s] == 2)
                res[s] = old[s] == 0u ? 1 : (old[s] == key[s] ? 0 : 2);
            more |= res[s] == 2;
        }
    }
#pragma unroll
    for (int s = 0; s < NS; ++s)
        if (res[s] == 2)
            res[s] = -1;  // every slot probed: the table is full
}

// Moves every key of the table src (2^sbits slots; in global memory when
// src_global) into the global table dst (2^dbits slots), which is cleared
// first.  The whole warp calls it.
__device__ __forceinline__ void migrate_keys(const uint32_t *src, int sbits, bool src_global, uint32_t *dst,
                                             int dbits, int lane)
{
    for (int o = lane; o < (1 << dbits) / 4; o += 32)
        reinterpret_cast<uint4 *>(dst)[o] = make_uint4(0u, 0u, 0u, 0u);
    __syncwarp();
    const uint32_t dmask = (1u << dbits) - 1u;
    for (int o = lane; o < (1 << sbits); o += 32) {
        const uint32_t key = src_global ? __ldcg(src + o) : src[o];
        if (key == 0u)
            continue;
        uint32_t g = hash_slot(key, dbits);
        for (uint32_t pr = 0; pr <= dmask; ++pr) {
            if (atomicCAS(&dst[g], 0u, key) == 0u)
                break;
            g = (g + 1u) & dmask;
        }
    }
    __syncwarp();
}

// Distance of one staged row to the query, computed by a team of G lanes
// (G a power of two <= 32; sub = lane % G takes the row's 16-byte chunks sub,
// sub+G, ...) and combined with log2(G) xor-shuffles inside the team; every
// lane of the team returns the order-preserving key bits.  CPL > 0: the row
// has exactly CPL * G chunks, so the chunk loop is unrolled and its shared-
// memory loads issue back to back (CPL = 0: any chunk count).  The whole warp
// must call it.
template <int DT, int MT, int CPL>
__device__ __forceinline__ uint32_t group_distance(const uint8_t *row, const uint8_t *q, int rowbytes, int sub,
                                                   int G)
{
    const int chunks = CPL > 0 ? CPL * G : rowbytes / 16;
    if constexpr (DT == ANN_U8) {
        const uint4 *x4 = reinterpret_cast<const uint4 *>(row);
        const uint4 *q4 = reinterpret_cast<const uint4 *>(q);
        uint32_t acc = 0;
        auto chunk = [&](int c) {
            const uint4 x = x4[c], y = q4[c];
            uint32_t d;
            d = __vabsdiffu4(x.x, y.x);
            acc = __dp4a(d, d, acc);
            d = __vabsdiffu4(x.y, y.y);
            acc = __dp4a(d, d, acc);
            d = __vabsdiffu4(x.z, y.z);
            acc = __dp4a(d, d, acc);
            d = __vabsdiffu4(x.w, y.w);
            acc = __dp4a(d, d, acc);
        };
        if constexpr (CPL > 0) {
#pragma unroll
            for (int i = 0; i < CPL; ++i)
                chunk(sub + i * G);
        } else {
            for (int c = sub; c < chunks; c += G)
                chunk(c);
        }
        for (int o = G >> 1; o > 0; o >>= 1)
            acc += __shfl_xor_sync(kFull, acc, o);
        return acc;  // exact non-negative int32, ordered as unsigned
    } else if constexpr (DT == ANN_I8S) {
        // x_j = scale * code_j.  L2: sum of (q_j - scale * code_j)^2, each
        // difference from one fused multiply-add; IP: scale * sum q_j code_j.
        // The query buffer is zero beyond dim, where the codes are zero too.
        const float scale = *reinterpret_cast<const float *>(row);
        const uint4 *c4 = reinterpret_cast<const uint4 *>(row + 16);
        const float4 *q4 = reinterpret_cast<const float4 *>(q);
        float a0 = 0.f, a1 = 0.f;
        for (int c = sub; c < chunks - 1; c += G) {
            const uint4 x = c4[c];
            const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float4 y = q4[4 * c + k];
                const float c0 = static_cast<float>(static_cast<int8_t>(w[k] & 0xffu));
                const float c1 = static_cast<float>(static_cast<int8_t>((w[k] >> 8) & 0xffu));
                const float c2 = static_cast<float>(static_cast<int8_t>((w[k] >> 16) & 0xffu));
                const float c3 = static_cast<float>(static_cast<int8_t>(w[k] >> 24));
                if constexpr (MT == ANN_L2) {
                    const float d0 = fmaf(-scale, c0, y.x), d1 = fmaf(-scale, c1, y.y);
                    const float d2 = fmaf(-scale, c2, y.z), d3 = fmaf(-scale, c3, y.w);
                    a0 = fmaf(d0, d0, a0);
                    a1 = fmaf(d1, d1, a1);
                    a0 = fmaf(d2, d2, a0);
                    a1 = fmaf(d3, d3, a1);
                } else {
                    a0 = fmaf(c0, y.x, a0);
                    a1 = fmaf(c1, y.y, a1);
                    a0 = fmaf(c2, y.z, a0);
                    a1 = fmaf(c3, y.w, a1);
                }
            }
        }
        float s = a0 + a1;
        for (int o = G >> 1; o > 0; o >>= 1)
            s += __shfl_xor_sync(kFull, s, o);
        if constexpr (MT == ANN_IP)
            s = -(scale * s);
        return f32_to_ord(s);
    } else {
        const float4 *q4 = reinterpret_cast<const float4 *>(q);
        // four FP32 accumulators (coordinates 4c+0..3) held as two packed
        // pairs: each f32x2 operation rounds both halves exactly as the scalar
        // operations would, at half the instruction count, and the two pairs
        // are independent dependency chains
        uint64_t acc = 0, acc2 = 0;  // (0.f, 0.f)
        auto acc4 = [&](float x0, float x1, float x2, float x3, float4 y) {
            if constexpr (MT == ANN_L2)
                asm("{\n\t.reg .b64 x, y, d;\n\t"
                    "mov.b64 x, {%2, %3};\n\tmov.b64 y, {%6, %7};\n\t"
                    "sub.rn.f32x2 d, x, y;\n\tfma.rn.f32x2 %0, d, d, %0;\n\t"
                    "mov.b64 x, {%4, %5};\n\tmov.b64 y, {%8, %9};\n\t"
                    "sub.rn.f32x2 d, x, y;\n\tfma.rn.f32x2 %1, d, d, %1;\n\t}"
                    : "+l"(acc), "+l"(acc2)
                    : "f"(x0), "f"(x1), "f"(x2), "f"(x3), "f"(y.x), "f"(y.y), "f"(y.z), "f"(y.w));
            else
                asm("{\n\t.reg .b64 x, y;\n\t"
                    "mov.b64 x, {%2, %3};\n\tmov.b64 y, {%6, %7};\n\t"
                    "fma.rn.f32x2 %0, x, y, %0;\n\t"
                    "mov.b64 x, {%4, %5};\n\tmov.b64 y, {%8, %9};\n\t"
                    "fma.rn.f32x2 %1, x, y, %1;\n\t}"
                    : "+l"(acc), "+l"(acc2)
                    : "f"(x0), "f"(x1), "f"(x2), "f"(x3), "f"(y.x), "f"(y.y), "f"(y.z), "f"(y.w));
        };
        auto chunk = [&](int c) {
            if constexpr (DT == ANN_F32) {
                const float4 x = reinterpret_cast<const float4 *>(row)[c];
                acc4(x.x, x.y, x.z, x.w, q4[c]);
            } else {
                const uint4 x = reinterpret_cast<const uint4 *>(row)[c];
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
        };
        if constexpr (CPL > 0) {
#pragma unroll
            for (int i = 0; i < CPL; ++i)
                chunk(sub + i * G);
        } else {
            for (int c = sub; c < chunks; c += G)
                chunk(c);
        }
        float s = (__uint_as_float(static_cast<uint32_t>(acc)) + __uint_as_float(static_cast<uint32_t>(acc >> 32))) +
                  (__uint_as_float(static_cast<uint32_t>(acc2)) + __uint_as_float(static_cast<uint32_t>(acc2 >> 32)));
        for (int o = G >> 1; o > 0; o >>= 1)
            s += __shfl_xor_sync(kFull, s, o);
        if constexpr (MT == ANN_IP)
            s = -s;
        return f32_to_ord(s);
    }
}

// group_distance with the chunk count per lane picked at run time: cpl is
// uniform over the launch (0 = the general loop).
template <int DT, int MT>
__device__ __forceinline__ uint32_t row_distance(const uint8_t *row, const uint8_t *q, int rowbytes, int sub, int G,
                                                 int cpl)
{
    if constexpr (DT != ANN_I8S) {
        if (cpl == 8)
            return group_distance<DT, MT, 8>(row, q, rowbytes, sub, G);
    }
    return group_distance<DT, MT, 0>(row, q, rowbytes, sub, G);
}

// One TMA tensor gather of four whole base rows (row ids r0..r3) into four
// consecutive staging rows at dst, counted on bar.
__device__ __forceinline__ void gather4_rows(void *dst, const CUtensorMap *map, int32_t r0, int32_t r1, int32_t r2,
                                             int32_t r3, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(0), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(smem_addr(bar))
        : "memory");
}

template <int DT, int MT>
__global__ void __launch_bounds__(32 * kMaxSearchWarps, 16) beam_search_kernel(const __grid_constant__ SearchArgs a)
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
    uint64_t *ptop = reinterpret_cast<uint64_t *>(my + a.off_ptop);  // W keys for the prediction
    uint64_t *cbuf = reinterpret_cast<uint64_t *>(my + a.off_cbuf);
    uint32_t *htab = reinterpret_cast<uint32_t *>(my + a.off_hash);
    const int team = blockIdx.x * (blockDim.x >> 5) + wid;
    // two global spill tables per team: 2^spill_bits slots, then one four
    // times larger for the rare query that outgrows the first; the first
    // tables of all teams lie together at the front of the scratch (one
    // range for an L2 access-policy window), the larger ones after them
    uint32_t *gtab1 = a.spill + static_cast<size_t>(team) * (static_cast<size_t>(1) << a.spill_bits);
    uint32_t *gtab2 = a.spill + static_cast<size_t>(a.nteams) * (static_cast<size_t>(1) << a.spill_bits) +
                      static_cast<size_t>(team) * (static_cast<size_t>(4) << a.spill_bits);

    if (lane == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint32_t phase = 0;
    // hash_bits < 0: no shared table, the visited set starts in the global one
    const bool shared_tab = a.hash_bits > 0;
    const int hcap = shared_tab ? 1 << a.hash_bits : 0;
    const int hlimit = hcap * 3 / 4;

    for (;;) {
        long long qi = 0;
        if (lane == 0)
            qi = static_cast<long long>(atomicAdd(a.counter, 1ull));
        qi = __shfl_sync(kFull, qi, 0);
        if (qi >= a.nq)
            break;
        if (a.order)
            qi = a.order[qi];

        const int Lq = a.dL ? a.dL[qi] : a.L;
        const int kq = a.dk ? a.dk[qi] : a.k;
        const int64_t qrow = qi / a.qdiv;
        const int32_t target = a.dtarget ? a.dtarget[qrow] : -1;
        // seed set: lane e < n_entries holds seed e (-1 = unused slot)
        const int32_t seed = a.entries ? (lane < a.n_entries ? a.entries[qi * a.n_entries + lane] : -1)
                                       : (lane == 0 ? a.medoid : -1);
        const bool seeds_ok = !__any_sync(kFull, seed < -1 || seed >= a.n) && __any_sync(kFull, seed >= 0);
        bool failed = false;
        bool timed_out = false, lost = false;
        if (Lq < 1 || Lq > a.L || kq < 1 || kq > a.k || kq > Lq || !seeds_ok) {
            failed = true;
            if (lane == 0)
                atomicOr(a.status, kStatusBadInputBit);
        }

        int cnt = 0, cursor = 0, evals = 0, hops = 0;
        // visited set: level 0 = the shared table, 1 and 2 = the global ones;
        // used = keys in the current table, limit = its 3/4 load
        int level = shared_tab ? 0 : 1, used = 0, gbits = a.spill_bits;
        int limit = shared_tab ? hlimit : (1 << a.spill_bits) * 3 / 4;
        uint32_t *gtab = gtab1;
        int32_t *pred = sel + ANN_MAX_W;  // predicted ids of the next selection
        int npred = 0;
        int32_t nxt[kSlots];  // their adjacency rows, lane-distributed like cur[]
#pragma unroll
        for (int r = 0; r < kSlots; ++r)
            nxt[r] = -1;
        bool found = false;
        if (!failed) {
            // query row -> shared memory; clear the visited table
            const uint8_t *qsrc = a.queries + qrow * a.qbytes;
            for (int o = lane * 16; o < a.qbytes; o += 32 * 16)
                *reinterpret_cast<uint4 *>(qbuf + o) = *reinterpret_cast<const uint4 *>(qsrc + o);
            for (int o = a.qbytes + lane * 4; o < a.qbytes + a.qpad; o += 32 * 4)
                *reinterpret_cast<float *>(qbuf + o) = 0.f;
            for (int o = lane; o < hcap / 4; o += 32)
                reinterpret_cast<uint4 *>(htab)[o] = make_uint4(0u, 0u, 0u, 0u);
            if (!shared_tab)
                for (int o = lane; o < (1 << a.spill_bits) / 4; o += 32)
                    reinterpret_cast<uint4 *>(gtab1)[o] = make_uint4(0u, 0u, 0u, 0u);
            __syncwarp();
            // the initial pool: every distinct seed, evaluated in the first step
            const int r = seed >= 0 ? visit(htab, a.hash_bits, !shared_tab, gtab1, a.spill_bits, seed) : 0;
            const unsigned nm = __ballot_sync(kFull, r == 1);
            if (r == 1)
                cbuf[__popc(nm & lanemask_lt())] = static_cast<uint64_t>(seed) << 1;
            used = evals = __popc(nm);
            found = __any_sync(kFull, r == 1 && seed == target);
        }
        int nc = failed ? 0 : evals;
        __syncwarp();

        while (!failed) {
            // ---- evaluate the nc candidates in cbuf[] (their ids in the key
            // layout, distance bits 0); the survivors end sorted
            // in cbuf[0, m)
            int m = 0;
            if (nc > 0) {
                for (int c0 = 0; c0 < nc; c0 += a.stage_rows) {
                    const int ch = min(a.stage_rows, nc - c0);
                    if (a.gather4) {
                        // groups of four rows, the last group padded by
                        // repeating its last row
                        const int ng = (ch + 3) >> 2;
                        if (lane == 0)
                            mbar_arrive_expect_tx(bar, static_cast<uint32_t>(ng) * 4 * a.rowbytes);
                        __syncwarp();
                        for (int g = lane; g < ng; g += 32) {
                            const int j = c0 + 4 * g, last = c0 + ch - 1;
                            gather4_rows(stage + 4 * g * a.stage_stride, &a.row_map, key_id(cbuf[j]),
                                         key_id(cbuf[min(j + 1, last)]), key_id(cbuf[min(j + 2, last)]),
                                         key_id(cbuf[min(j + 3, last)]), bar);
                        }
                    } else {
                        if (lane == 0)
                            mbar_arrive_expect_tx(bar, static_cast<uint32_t>(ch) * a.rowbytes);
                        __syncwarp();
                        for (int j = lane; j < ch; j += 32)
                            bulk_g2s(stage + j * a.stage_stride,
                                     a.base + static_cast<size_t>(key_id(cbuf[c0 + j])) * a.rowbytes, a.rowbytes,
                                     bar);
                    }
                    const bool ok = !a.fault_wait && mbar_wait_bounded(bar, phase, kTimeoutIters);
                    if (!__all_sync(kFull, ok)) {
                        // the query fails with a timeout; give the copies one
                        // more bounded wait: if they land, the barrier is in a
                        // known state and the team goes on with the next
                        // query, else it retires
                        const bool landed = __all_sync(kFull, mbar_wait_bounded(bar, phase, kTimeoutIters));
                        if (landed)
                            phase ^= 1u;
                        lost = !landed;
                        timed_out = true;
                        failed = true;
                        break;
                    }
                    phase ^= 1u;
                    // a team of G lanes per staged row, 32 / G rows per pass
                    for (int r0 = 0; r0 < ch; r0 += 32 >> a.team_lg) {
                        const int r = r0 + (lane >> a.team_lg);
                        const int sub = lane & ((1 << a.team_lg) - 1);
                        const uint32_t bits = row_distance<DT, MT>(stage + min(r, ch - 1) * a.stage_stride, qbuf,
                                                                   a.rowbytes, sub, 1 << a.team_lg, a.cpl);
                        if (r < ch && sub == 0)
                            cbuf[c0 + r] = make_key(bits, key_id(cbuf[c0 + r]));
                    }
                    __syncwarp();
                    fence_proxy_async_smem();  // stage reads done before the next bulk writes
                }
                if (failed)
                    break;
                // candidates no better than a full pool's last entry cannot
                // enter it; only the survivors are sorted
                const uint64_t worst = (cnt == Lq) ? key_plain(pool[Lq - 1]) : kKeyMax;
                uint64_t kk[kSlots];
                unsigned bm[kSlots];
#pragma unroll
                for (int s = 0; s < kSlots; ++s) {
                    uint64_t v = lane + 32 * s < nc ? cbuf[lane + 32 * s] : kKeyMax;
                    if (v >= worst)
                        v = kKeyMax;
                    kk[s] = v;
                    bm[s] = __ballot_sync(kFull, v != kKeyMax);
                    m += __popc(bm[s]);
                }
                __syncwarp();
                if (m > 0) {
                    if (m <= 32 || (m <= 64 && nc > 64)) {
                        // compact the survivors into cbuf[0, m) (a 64-key
                        // sort of candidates that all sit in slots 0-1 needs
                        // none: the dropped ones sort to the end)
                        int base = 0;
#pragma unroll
                        for (int s = 0; s < kSlots; ++s) {
                            if (kk[s] != kKeyMax)
                                cbuf[base + __popc(bm[s] & lanemask_lt())] = kk[s];
                            base += __popc(bm[s]);
                        }
                        __syncwarp();
                        kk[0] = lane < m ? cbuf[lane] : kKeyMax;
                        kk[1] = lane + 32 < m ? cbuf[lane + 32] : kKeyMax;
                        __syncwarp();
                    }
                    if (m <= 32) {
                        // sort over the next power of two only
                        int width = 1;
                        while (width < m)
                            width <<= 1;
                        kk[0] = warp_sort_lanes(kk[0], lane, width);
                        cbuf[lane] = kk[0];
                    } else if (m <= 64) {
                        warp_sort64(kk[0], kk[1], lane);
                        cbuf[lane] = kk[0];
                        cbuf[lane + 32] = kk[1];
                    } else {
                        warp_sort_n<kSlots>(kk, lane);
#pragma unroll
                        for (int s = 0; s < kSlots; ++s)
                            cbuf[lane + 32 * s] = kk[s];
                    }
                    __syncwarp();
                }
            }

            // ---- predict the next selection: the W smallest unexpanded keys
            // among the pool and the survivors.  Their adjacency rows are
            // loaded now, so the loads overlap the merge.
            {
                int nf = 0;
                for (int i0 = cursor; i0 < cnt && nf < a.W; i0 += 32) {
                    const int i = i0 + lane;
                    const bool un = i < cnt && !(pool[i] & 1ull);
                    const unsigned um = __ballot_sync(kFull, un);
                    const int g = nf + __popc(um & lanemask_lt());
                    if (un && g < a.W)
                        ptop[g] = pool[i];
                    nf = min(a.W, nf + __popc(um));
                }
                __syncwarp();
                const int mw = min(m, a.W);
                int i = 0, j = 0, np = 0;
                for (; np < a.W && (i < nf || j < mw); ++np) {
                    const bool from_pool = j >= mw || (i < nf && ptop[i] < cbuf[j]);
                    const uint64_t v = from_pool ? ptop[i++] : cbuf[j++];
                    if (lane == 0)
                        pred[np] = key_id(v);
                }
                npred = np;
                __syncwarp();
                const int tp = npred * a.R;
#pragma unroll
                for (int r = 0; r < kSlots; ++r) {
                    const int t = lane + 32 * r;
                    const int e = (t * a.R_inv) >> 16;  // t / R
                    nxt[r] = t < tp ? __ldg(a.graph + static_cast<int64_t>(pred[e]) * a.R + (t - e * a.R)) : -1;
                }
            }

            // ---- merge the survivors into the pool by rank, in place: the
            // survivors' ranks come from the unmodified pool; pool entries move
            // right by the number of smaller survivors, 32 at a time from the
            // back, so that none is overwritten before it is read
            if (m > 0) {
                int dst[kSlots];
#pragma unroll
                for (int r = 0; r < kSlots; ++r) {
                    const int j = lane + 32 * r;
                    dst[r] = j < m ? j + count_less(pool, cnt, cbuf[j]) : Lq;
                }
                const int p0 = __shfl_sync(kFull, dst[0], 0);  // rank of the best survivor
                __syncwarp();
                for (int b = cnt > p0 ? p0 + (cnt - 1 - p0) / 32 * 32 : p0 - 32; b >= p0; b -= 32) {
                    const int i = b + lane;
                    uint64_t v = 0;
                    int np = Lq;
                    if (i < cnt) {
                        v = pool[i];
                        np = i + count_less(cbuf, m, key_plain(v));
                    }
                    __syncwarp();
                    if (np < Lq)
                        pool[np] = v;
                    __syncwarp();
                }
#pragma unroll
                for (int r = 0; r < kSlots; ++r)
                    if (dst[r] < Lq)
                        pool[dst[r]] = cbuf[lane + 32 * r];
                __syncwarp();
                cnt = min(Lq, cnt + m);
                cursor = min(cursor, p0);
            }
            if (found)
                break;

            // ---- select the first W unexpanded pool entries; mark them expanded
            int ns = 0, first = -1;
            for (int i0 = cursor; i0 < cnt && ns < a.W; i0 += 32) {
                const int i = i0 + lane;
                const bool un = i < cnt && !(pool[i] & 1ull);
                const unsigned um = __ballot_sync(kFull, un);
                if (um) {
                    if (first < 0)
                        first = i0 + __ffs(um) - 1;
                    const int g = ns + __popc(um & lanemask_lt());
                    if (un && g < a.W) {
                        const uint64_t v = pool[i];
                        pool[i] = v | 1ull;
                        sel[g] = key_id(v);
                    }
                    ns = min(a.W, ns + __popc(um));
                }
            }
            __syncwarp();
            if (ns == 0)
                break;
            cursor = first;
            hops += ns;

            // ---- adjacency rows of the selected entries: the predicted ones,
            // unless truncation to L dropped a predicted entry (then loaded now)
            const int total = ns * a.R;
            bool hit = ns == npred;
            for (int s = 0; s < ns && hit; ++s)
                hit = sel[s] == pred[s];
            int32_t cur[kSlots];
#pragma unroll
            for (int r = 0; r < kSlots; ++r) {
                const int t = lane + 32 * r;
                cur[r] = hit ? nxt[r]
                             : (t < total ? __ldg(a.graph + static_cast<int64_t>(sel[(t * a.R_inv) >> 16]) * a.R +
                                                   (t - ((t * a.R_inv) >> 16) * a.R))
                                          : -1);
            }

            // ---- neighbours of the selected entries: visited test, compaction
            // A table that would pass 3/4 load hands its keys to the next,
            // larger one (shared -> global -> 4x larger global), which takes
            // every later insert, so a lookup probes one table only and the
            // set stays exact.
            while (used + total > limit && level < 2) {
                uint32_t *dst = level == 0 ? gtab1 : gtab2;
                const int dbits = level == 0 ? a.spill_bits : a.spill_bits + 2;
                if (level == 0)
                    migrate_keys(htab, a.hash_bits, false, dst, dbits, lane);
                else
                    migrate_keys(gtab, gbits, true, dst, dbits, lane);
                gtab = dst;
                gbits = dbits;
                limit = (1 << dbits) * 3 / 4;
                ++level;
            }
            if (used + total > limit) {
                failed = true;
                if (lane == 0)
                    atomicOr(a.status, kStatusCapacityBit);
                break;
            }
            // every slot's first probe is issued before any result is used, so
            // their latencies overlap (global atomics in spill mode)
            int32_t vid[kSlots];
            int res[kSlots];
#pragma unroll
            for (int s = 0; s < kSlots; ++s) {
                const int32_t id = lane + 32 * s < total ? cur[s] : -1;
                vid[s] = (id >= 0 && id < a.n) ? id : -1;
            }
            if (level > 0)
                visit_slots<kSlots>(gtab, gbits, vid, res);
            else
                visit_slots<kSlots>(htab, a.hash_bits, vid, res);
            nc = 0;
            bool bad = false;
#pragma unroll
            for (int s = 0; s < kSlots; ++s) {
                if (32 * s >= total)
                    break;
                bad |= (res[s] < 0);
                const unsigned nm = __ballot_sync(kFull, res[s] == 1);
                if (res[s] == 1) {
                    cbuf[nc + __popc(nm & lanemask_lt())] = static_cast<uint64_t>(static_cast<uint32_t>(vid[s])) << 1;
                    if (vid[s] == target)
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
            used += nc;
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
        if (a.pool_out) {
            for (int j = lane; j < a.L; j += 32)
                a.pool_out[qi * a.L + j] = (!failed && j < cnt) ? key_id(pool[j]) : -1;
        }
        if (a.out_stats && lane == 0) {
            const bool miss = failed || (target >= 0 && !found);
            a.out_stats[2 * qi] = miss && target >= 0 ? INT32_MAX : evals;
            a.out_stats[2 * qi + 1] = miss && target >= 0 ? INT32_MAX : hops;
        }
        __syncwarp();
        if (lost)
            return;  // this team's barrier state is unknown: retire it
    }
}

// Work order grouped by first seed: a counting sort of the work items by a
// 12-bit hash of their first seed, in one CTA (the histogram and the scatter
// use shared-memory atomics, so items of one bucket come out in no fixed
// order; the search's results do not depend on the order).  Each thread
// reads its items' seeds eight at a time, so their loads are in flight
// together, and keeps the buckets of the first kGroupCache items in shared
// memory for the scatter pass.
constexpr int kGroupThreads = 1024;
constexpr int kGroupBits = 12;
constexpr int kGroupPer = (1 << kGroupBits) / kGroupThreads;  // buckets per thread
constexpr int kGroupBatch = 8;                                 // seeds loaded together per thread
constexpr int kGroupCache = 12288;                             // items whose bucket is kept

__device__ __forceinline__ uint32_t seed_bucket(int32_t e)
{
    return (static_cast<uint32_t>(e) * 0x9E3779B1u) >> (32 - kGroupBits);
}

__global__ void __launch_bounds__(kGroupThreads)
    group_by_seed_kernel(const int32_t *__restrict__ entries, int n_entries, int64_t nitems,
                         int32_t *__restrict__ order)
{
    __shared__ int cnt[1 << kGroupBits];
    __shared__ int wsum[kGroupThreads / 32];
    __shared__ uint16_t bucket_of[kGroupCache];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    for (int i = t; i < (1 << kGroupBits); i += kGroupThreads)
        cnt[i] = 0;
    __syncthreads();
    // item w = base + j * kGroupThreads + t for j < kGroupBatch
    constexpr int64_t kStride = static_cast<int64_t>(kGroupThreads) * kGroupBatch;
    for (int64_t base = 0; base < nitems; base += kStride) {
        int32_t e[kGroupBatch];
#pragma unroll
        for (int j = 0; j < kGroupBatch; ++j) {
            const int64_t w = base + j * kGroupThreads + t;
            e[j] = w < nitems ? __ldg(entries + w * n_entries) : 0;
        }
#pragma unroll
        for (int j = 0; j < kGroupBatch; ++j) {
            const int64_t w = base + j * kGroupThreads + t;
            if (w < nitems) {
                const uint32_t bk = seed_bucket(e[j]);
                atomicAdd(&cnt[bk], 1);
                if (w < kGroupCache)
                    bucket_of[w] = static_cast<uint16_t>(bk);
            }
        }
    }
    __syncthreads();
    // exclusive scan: thread t owns buckets [kGroupPer t, kGroupPer (t + 1))
    int v[kGroupPer], tot = 0;
#pragma unroll
    for (int j = 0; j < kGroupPer; ++j) {
        v[j] = cnt[kGroupPer * t + j];
        tot += v[j];
    }
    int inc = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o)
            inc += u;
    }
    if (lane == 31)
        wsum[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int x = wsum[lane], xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o)
                xi += u;
        }
        wsum[lane] = xi - x;
    }
    __syncthreads();
    int run = wsum[wid] + inc - tot;
#pragma unroll
    for (int j = 0; j < kGroupPer; ++j) {
        cnt[kGroupPer * t + j] = run;
        run += v[j];
    }
    __syncthreads();
    for (int64_t base = 0; base < nitems; base += kStride) {
        uint32_t bk[kGroupBatch];
#pragma unroll
        for (int j = 0; j < kGroupBatch; ++j) {
            const int64_t w = base + j * kGroupThreads + t;
            bk[j] = w >= nitems ? 0u : w < kGroupCache ? bucket_of[w] : seed_bucket(__ldg(entries + w * n_entries));
        }
#pragma unroll
        for (int j = 0; j < kGroupBatch; ++j) {
            const int64_t w = base + j * kGroupThreads + t;
            if (w < nitems)
                order[atomicAdd(&cnt[bk[j]], 1)] = static_cast<int32_t>(w);
        }
    }
}

// Exact rerank of the final pool (reduced-precision storage): one warp per
// query re-scores every pool id against the fp32 copy of its row (lanes over
// the row, FP32 accumulation), sorts the (distance, id) keys in shared memory
// with a bitonic network and writes the best k.
constexpr int kRerankWarps = 4;

template <int MT>
__global__ void __launch_bounds__(32 * kRerankWarps)
    rerank_kernel(const float *base_f32, int dim, const float *queries, int64_t nq, int64_t qdiv,
                  const int32_t *pool, int L, int P, int k, const int32_t *dk, int32_t *out_ids,
                  float *out_dists)
{
    extern __shared__ __align__(16) uint64_t rkeys[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint64_t *keys = rkeys + static_cast<size_t>(w) * P;
    for (int64_t qi = static_cast<int64_t>(blockIdx.x) * kRerankWarps + w; qi < nq;
         qi += static_cast<int64_t>(gridDim.x) * kRerankWarps) {
        const float *q = queries + (qi / qdiv) * dim;
        for (int c = 0; c < P; ++c) {
            const int32_t id = c < L ? pool[qi * L + c] : -1;
            uint64_t key = kKeyMax;
            if (id >= 0) {
                const float *x = base_f32 + static_cast<int64_t>(id) * dim;
                float s = 0.f;
                for (int j = lane; j < dim; j += 32) {
                    if constexpr (MT == ANN_L2) {
                        const float t = x[j] - q[j];
                        s = fmaf(t, t, s);
                    } else {
                        s = fmaf(x[j], q[j], s);
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
                    s += __shfl_xor_sync(kFull, s, o);
                key = make_key(f32_to_ord(MT == ANN_IP ? -s : s), id);
            }
            if (lane == 0)
                keys[c] = key;
        }
        __syncwarp();
        for (int kk = 2; kk <= P; kk <<= 1) {
            for (int j = kk >> 1; j > 0; j >>= 1) {
                for (int i = lane; i < P; i += 32) {
                    const int p = i ^ j;
                    if (p > i) {
                        const uint64_t a = keys[i], b = keys[p];
                        const bool asc = (i & kk) == 0;
                        if ((a > b) == asc) {
                            keys[i] = b;
                            keys[p] = a;
                        }
                    }
                }
                __syncwarp();
            }
        }
        const int kq = dk ? dk[qi] : k;
        for (int j = lane; j < k; j += 32) {
            const uint64_t v = j < kq ? keys[j] : kKeyMax;
            const bool ok = v != kKeyMax;
            out_ids[qi * k + j] = ok ? key_id(v) : -1;
            out_dists[qi * k + j] = ok ? ord_to_f32(static_cast<uint32_t>(v >> 32)) : __int_as_float(0x7f800000);
        }
        __syncwarp();
    }
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Resident teams for `per_warp` bytes of shared memory per team, with one or
// two teams per CTA, whichever fits more (each CTA also costs the SM a fixed
// reserve of shared memory, which two teams share).
template <int DT, int MT>
ann_status teams_for(ann_index *idx, size_t per_warp, int *teams, int *wpc)
{
    auto kern = beam_search_kernel<DT, MT>;
    int best = 0, best_w = 1;
    for (int w = 1; w <= kMaxSearchWarps; ++w) {
        const size_t smem = per_warp * w;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
            cudaSuccess) {
            cudaGetLastError();  // too large for one CTA: not a candidate
            continue;
        }
        int per_sm = 0;
        const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * w, smem);
        if (e != cudaSuccess)
            return cuda_status(e);
        if (per_sm * w > best) {
            best = per_sm * w;
            best_w = w;
        }
    }
    if (best < 1)
        return ANN_ERR_UNSUPPORTED;  // the per-query state does not fit in shared memory
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               static_cast<int>(per_warp * best_w));
    if (e != cudaSuccess)
        return cuda_status(e);
    *teams = best * idx->num_sms;
    *wpc = best_w;
    return ANN_OK;
}

// window: bytes of the first-level visited tables to keep resident in L2
// (0 = launch without an access-policy window), at the given hit ratio
template <int DT, int MT>
ann_status launch_typed(const SearchArgs &a, size_t smem, int teams, int wpc, cudaStream_t s, size_t window,
                        float hit_ratio)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(teams / wpc);
    cfg.blockDim = dim3(32 * wpc);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeAccessPolicyWindow;
    at[0].val.accessPolicyWindow.base_ptr = a.spill;
    at[0].val.accessPolicyWindow.num_bytes = window;
    at[0].val.accessPolicyWindow.hitRatio = hit_ratio;
    at[0].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    at[0].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    cfg.attrs = at;
    cfg.numAttrs = window > 0 ? 1 : 0;
    return cuda_status(cudaLaunchKernelEx(&cfg, beam_search_kernel<DT, MT>, a));
}

// Bytes of L2 the first-level visited tables may keep resident on the
// current device: the device's persisting-L2 maximum, to which the context's
// set-aside is raised (outside stream capture) when it is lower, for
// ANN_SEARCH_VISITED_L2; ann_release_l2 lowers it again.
size_t persisting_l2_bytes(int dev, cudaStream_t s)
{
    int maxp = 0;
    if (cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, dev) != cudaSuccess || maxp <= 0)
        return 0;
    size_t cur = 0;
    if (cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize) != cudaSuccess)
        return 0;
    if (cur < static_cast<size_t>(maxp)) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone &&
            cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, static_cast<size_t>(maxp)) == cudaSuccess)
            cur = static_cast<size_t>(maxp);
        cudaGetLastError();
    }
    return cur;
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
    case ANN_I8S * 2 + ANN_L2: st = FN<ANN_I8S, ANN_L2>(__VA_ARGS__); break;         \
    case ANN_I8S * 2 + ANN_IP: st = FN<ANN_I8S, ANN_IP>(__VA_ARGS__); break;         \
    default: st = ANN_ERR_UNSUPPORTED; break;                                        \
    }

}  // namespace

int default_team(int rowbytes)
{
    const int chunks = rowbytes / 16;
    int G = 4;
    while (G < 32 && chunks > 4 * G)
        G <<= 1;
    return G;
}

int default_spill_bits(int L)
{
    int sb = 12;
    while ((1 << sb) * 3 / 4 < 40 * L && sb < 15)
        ++sb;
    return sb;
}

size_t search_scratch_bytes(int teams, int spill_bits, int64_t order_items)
{
    return 256 + static_cast<size_t>(teams) * (static_cast<size_t>(20) << spill_bits) +
           4 * static_cast<size_t>(order_items);
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
    a.R_inv = ((1 << 16) + a.R - 1) / a.R;
    a.rowbytes = idx->rowbytes;
    a.queries = static_cast<const uint8_t *>(L.queries);
    a.qbytes = L.qbytes;
    // int8 rows are read in whole 16-code chunks: the query is zero-extended
    // to the padded code count
    a.qpad = idx->dtype == ANN_I8S ? 4 * ((idx->dim + 15) / 16 * 16 - idx->dim) : 0;
    a.nq = L.nq;
    a.qdiv = L.qdiv > 0 ? L.qdiv : 1;
    a.entries = L.entries;
    a.medoid = idx->medoid;
    a.L = p->L;
    a.k = p->k;
    a.W = p->W;
    a.n_entries = L.n_entries > 0 ? L.n_entries : 1;
    a.fault_wait = (p->flags & ANN_SEARCH_FAULT_WAIT) != 0;
    a.dk = p->d_k;
    a.dL = p->d_L;
    a.dtarget = p->d_target;
    a.out_ids = L.ids;
    a.out_dists = L.dists;
    a.out_stats = L.stats;
    a.status = idx->status_sink ? idx->status_sink : idx->d_status;

    int hb = p->hash_bits;  // -1: no shared table
    if (hb == 0) {
        // searches evaluate about 10-16 nodes per pool slot; size the shared
        // table for 12 per slot below its 3/4 load limit (the exact global
        // spill table takes any excess; ann_autotune refines the choice)
        hb = 10;
        while ((1 << hb) * 3 / 4 < 12 * p->L && hb < 13)
            ++hb;
    }
    a.hash_bits = hb;
    // the first spill table holds 40 evaluations per pool slot below 3/4 load
    // (about 3x the typical count), small enough to stay mostly L2-resident
    // and cheap to clear when a query starts spilling; the second holds four
    // times more for the tail
    int sb = default_spill_bits(p->L);
    if (p->spill_bits > 0)
        sb = p->spill_bits;
    a.spill_bits = sb;

    const int maxc = p->W * idx->degree;
    // distance team: the smallest power of two >= 4 that leaves at most four
    // 16-byte chunks of a row to each lane, unless the caller fixed it
    const int chunks = idx->rowbytes / 16;
    const int G = p->team > 0 ? p->team : default_team(idx->rowbytes);
    a.team_lg = 0;
    while ((1 << a.team_lg) < G)
        ++a.team_lg;
    // gather mode: one TMA tensor gather per four rows when the index has a
    // row map and the caller asks for it (or leaves it to the default, one
    // bulk copy per row)
    a.gather4 = (p->gather == 4 && idx->has_row_map) ? 1 : 0;
    if (a.gather4)
        a.row_map = idx->row_map;
    // staging stride in 16-byte units.  A quarter-warp phase of 16-byte loads
    // covers 8 lanes; with G < 8 they read 8 / G rows, whose G-chunk runs hit
    // distinct banks when the stride is G times an odd number.  Tensor
    // gathers write four rows back to back, so their stride is the row size.
    int s16 = chunks;
    if (G < 8 && !a.gather4)
        while (s16 % G != 0 || ((s16 / G) & 1) == 0)
            ++s16;
    a.stage_stride = s16 * 16;
    a.cpl = 0;
    if (idx->dtype != ANN_I8S && chunks % G == 0) {
        const int c = chunks / G;
        a.cpl = c == 8 ? c : 0;
    }
    // Most steps find far fewer new neighbours than W * R (about 30 % of
    // them), so a small staging area filled in rounds keeps shared memory per
    // team small (more teams per SM); at most 48 KB staged at once, which also
    // keeps one mbarrier phase's byte count far below its 2^20 limit.
    a.stage_rows = std::max(1, std::min({maxc, p->stage_rows > 0 ? p->stage_rows : 16, 49152 / a.stage_stride}));
    if (a.gather4)
        a.stage_rows = (a.stage_rows + 3) / 4 * 4;  // whole groups of four

    size_t off = 16;  // mbarrier
    a.off_sel = static_cast<int>(off);
    off = align_up(off + 4 * 2 * ANN_MAX_W, 16);  // selected and predicted ids
    a.off_q = static_cast<int>(off);
    off = align_up(off + L.qbytes + a.qpad, 16);
    if (a.gather4)
        off = align_up(off, 128);  // tensor gathers land on 128-byte boundaries
    a.off_stage = static_cast<int>(off);
    off = align_up(off + static_cast<size_t>(a.stage_rows) * a.stage_stride, 16);
    a.off_pool = static_cast<int>(off);
    off = align_up(off + 8 * static_cast<size_t>(p->L), 16);
    a.off_ptop = static_cast<int>(off);
    off = align_up(off + 8 * ANN_MAX_W, 16);
    a.off_cbuf = static_cast<int>(off);
    off = align_up(off + 8 * ANN_MAX_STEP_CAND, 16);
    a.off_hash = static_cast<int>(off);
    off = align_up(off + (hb > 0 ? static_cast<size_t>(4) << hb : 0), 128);
    a.per_warp = static_cast<int>(off);

    // persistent grid: occupancy-limited, at most one team per query
    int teams = 0, wpc = 1;
    ann_status st = ANN_OK;
    ANN_DISPATCH(teams_for, idx, off, &teams, &wpc);
    if (st != ANN_OK)
        return st;
    if (L.max_teams > 0)
        teams = std::min(teams, L.max_teams);
    teams = static_cast<int>(std::min<long long>(teams, L.nq));
    if (teams < 1)
        return ANN_OK;
    teams = (teams + wpc - 1) / wpc * wpc;  // whole CTAs
    const size_t smem = off * wpc;

    // scratch: work counter, then two spill tables per team, then the grouped
    // work order (when asked for, with seeds given and item indices in int32)
    const bool group = (p->flags & ANN_SEARCH_GROUP_ENTRIES) && L.entries && L.nq <= INT32_MAX;
    const size_t need = search_scratch_bytes(teams, a.spill_bits, group ? L.nq : 0);
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
    a.nteams = teams;
    a.spill = reinterpret_cast<uint32_t *>(static_cast<uint8_t *>(scratch) + 256);
    int32_t *order = nullptr;
    if (group)
        order = reinterpret_cast<int32_t *>(static_cast<uint8_t *>(scratch) +
                                            search_scratch_bytes(teams, a.spill_bits, 0));
    a.order = order;
    // exact rerank: the search hands its whole pool to rerank_kernel
    const bool rerank = (p->flags & ANN_SEARCH_RERANK) != 0;
    void *pool_buf = nullptr;
    if (rerank) {
        st = scratch_alloc(idx, static_cast<size_t>(L.nq) * p->L * 4, s, &pool_buf);
        if (st != ANN_OK) {
            if (own)
                scratch_free(idx, scratch, s);
            return st;
        }
        a.pool_out = static_cast<int32_t *>(pool_buf);
    }
    // L2-resident first-level visited tables, when asked for and they fit
    size_t window = 0;
    float hit_ratio = 1.f;
    if (p->flags & ANN_SEARCH_VISITED_L2) {
        const size_t tbytes = static_cast<size_t>(teams) * (static_cast<size_t>(4) << a.spill_bits);
        int maxwin = 0;
        cudaDeviceGetAttribute(&maxwin, cudaDevAttrMaxAccessPolicyWindowSize, idx->device);
        const size_t setaside = persisting_l2_bytes(idx->device, s);
        if (tbytes <= setaside && tbytes <= static_cast<size_t>(maxwin))
            window = tbytes;
    }
    cudaError_t e = cudaMemsetAsync(scratch, 0, 8, s);
    if (e == cudaSuccess && group) {
        group_by_seed_kernel<<<1, kGroupThreads, 0, s>>>(L.entries, a.n_entries, L.nq, order);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        ANN_DISPATCH(launch_typed, a, smem, teams, wpc, s, window, hit_ratio);
    } else {
        st = cuda_status(e);
    }
    if (st == ANN_OK && rerank) {
        int P = 32;
        while (P < p->L)
            P <<= 1;
        const size_t rs = static_cast<size_t>(P) * 8 * kRerankWarps;
        const unsigned grid = static_cast<unsigned>(std::min<int64_t>((L.nq + kRerankWarps - 1) / kRerankWarps,
                                                                      static_cast<int64_t>(idx->num_sms) * 16));
        auto rk = idx->metric == ANN_IP ? rerank_kernel<ANN_IP> : rerank_kernel<ANN_L2>;
        e = cudaFuncSetAttribute(rk, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(rs));
        if (e == cudaSuccess) {
            rk<<<grid, 32 * kRerankWarps, rs, s>>>(idx->d_base_f32, idx->dim,
                                                    static_cast<const float *>(L.queries), L.nq, a.qdiv,
                                                    a.pool_out, p->L, P, p->k, p->d_k, L.ids,
                                                    static_cast<float *>(L.dists));
            e = cudaGetLastError();
        }
        st = cuda_status(e);
    }
    if (pool_buf)
        scratch_free(idx, pool_buf, s);
    if (own)
        scratch_free(idx, scratch, s);
    return st;
}

}  // namespace ann
