// entry.cu -- learned entry selection (Sec. 4.3) on tcgen05 tensor cores.
//
// Query tower (Module II, "lightweight MLP with ReLU"):
//     q -> Z1 = q W1 + b1 -> A1 = ReLU(Z1) -> Z2 = A1 W2 + b2 -> q_hat = Z2/|Z2|
// fused in one kernel: 128 queries per CTA, GEMM 1 (K = dim, N = 256) and
// GEMM 2 (K = 256, N = 64) on kind::f16 MMAs with BF16 operands and FP32
// accumulators in TMEM; the hidden layer goes TMEM -> registers (bias, ReLU,
// BF16) -> shared memory -> GEMM 2 without leaving the SM.
// Hub side: each hub v has an embedding e_v; e_hat_v = e_v / |e_v| is kept as
// BF16.  The entry of a query is the hub node of argmax_v q_hat . e_hat_v,
// found either exhaustively (entry_exhaustive_kernel: the tower and every
// hub's score in one launch; hub_argmax_kernel: the scores alone, a tcgen05
// GEMM with a fused per-row argmax epilogue) or by the greedy search of
// Algorithm 1 with the inner-product metric over the high-tier hub graph
// (Sec. 4.3: every hub linked to its s most cosine-similar hubs, as directed
// lists or, after ann_build_hub_graph, as undirected edges): hub_nav_kernel
// for pools of up to 64 hubs, the beam-search kernel on a BF16 index of the
// hub embeddings for larger ones.  The walk starts from the entry hub or from
// a caller-drawn sample of hubs (ann_set_hub_seeds).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <new>
#include <utility>
#include <vector>

#include "entry.h"
#include "internal.h"
#include "tc.cuh"

namespace ann {
namespace {

// ---- query tower ------------------------------------------------------------

constexpr int kTowerSmem = 16384 + 32768 + 65536 + 64;

struct TowerArgs {
    Operand X;  // queries: rows = nq, cols = in_dim
    const __nv_bfloat16 *W1t;  // [256][in_dim]
    int in_dim;
    const float *b1;
    const __nv_bfloat16 *W2t;  // [64][256]
    const float *b2;
    int64_t nq;
    float *qhat;                // [nq][64] optional
    __nv_bfloat16 *qhat_bf;     // [nq][64] optional
    float *z1;                  // [nq][256] optional (training)
    __nv_bfloat16 *a1;          // [nq][256] optional (training)
    float *nrm;                 // [nq] optional (training)
    int *status;
};

__device__ __forceinline__ uint4 pack8_bf16(const float *a)
{
    uint4 o;
    __nv_bfloat162 h0 = __floats2bfloat162_rn(a[0], a[1]), h1 = __floats2bfloat162_rn(a[2], a[3]);
    __nv_bfloat162 h2 = __floats2bfloat162_rn(a[4], a[5]), h3 = __floats2bfloat162_rn(a[6], a[7]);
    o.x = *reinterpret_cast<uint32_t *>(&h0);
    o.y = *reinterpret_cast<uint32_t *>(&h1);
    o.z = *reinterpret_cast<uint32_t *>(&h2);
    o.w = *reinterpret_cast<uint32_t *>(&h3);
    return o;
}

__global__ void __launch_bounds__(128) tower_forward_kernel(const TowerArgs t)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sA = smem;            // 128 x 64 canonical (16 KB)
    uint8_t *sB = smem + 16384;    // 256 x 64 or 64 x 256 canonical (32 KB)
    uint8_t *sH = smem + 49152;    // 128 x 256 hidden layer, canonical KG=32 (64 KB)
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 114688);
    uint32_t *slot = reinterpret_cast<uint32_t *>(smem + 114688 + 8);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m = warp * 32 + lane;
    const int64_t r0 = static_cast<int64_t>(blockIdx.x) * 128;
    const int64_t row = r0 + m;
    const bool live = row < t.nq;

    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    if (warp == 0)
        tmem_alloc(slot, 256);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *slot;
    const uint32_t my_lane = tmem + (static_cast<uint32_t>(warp * 32) << 16);
    uint32_t phase = 0;

    // GEMM 1: [128 x in_dim] x [in_dim x 256]
    const Operand W1{t.W1t, OP_BF16, t.in_dim, 1, 256, t.in_dim, nullptr};
    bool ok = tc_gemm_tile<256>(t.X, r0, W1, 0, t.in_dim, sA, sB, bar, phase, tmem);
    if (ok) {
        for (int c0 = 0; c0 < 256; c0 += 32) {
            float v[32];
            tmem_ld32(my_lane + c0, v);
#pragma unroll
            for (int j = 0; j < 32; ++j)
                v[j] += t.b1[c0 + j];
            if (t.z1 && live) {
                float4 *dst = reinterpret_cast<float4 *>(t.z1 + row * 256 + c0);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
            }
#pragma unroll
            for (int j = 0; j < 32; j += 8) {
                float a[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    a[u] = fmaxf(v[j + u], 0.f);
                const uint4 pk = pack8_bf16(a);
                *reinterpret_cast<uint4 *>(sH + canon_off(m, c0 + j, 32)) = pk;
                if (t.a1 && live)
                    *reinterpret_cast<uint4 *>(t.a1 + row * 256 + c0 + j) = pk;
            }
        }
        // GEMM 2: [128 x 256] x [256 x 64]; W2t staged whole (64 rows x 256 k)
        const Operand W2{t.W2t, OP_BF16, 256, 1, 64, 256, nullptr};
        stage_tile<64, 32>(sB, W2, 0, 0);
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc_fence_after();
            constexpr uint32_t ID2 = idesc_bf16_f32(128, 64);
#pragma unroll
            for (int kk = 0; kk < 16; ++kk)
                tc_mma(tmem, smem_desc(sH + kk * 256, 128, 4096), smem_desc(sB + kk * 256, 128, 4096), ID2,
                       kk > 0 ? 1u : 0u);
            tc_commit(bar);
        }
        ok = tc_wait(bar, phase);
    }
    if (ok) {
        float z[64];
        float v[32];
        tmem_ld32(my_lane, v);
#pragma unroll
        for (int j = 0; j < 32; ++j)
            z[j] = v[j] + t.b2[j];
        tmem_ld32(my_lane + 32, v);
#pragma unroll
        for (int j = 0; j < 32; ++j)
            z[32 + j] = v[j] + t.b2[32 + j];
        float ss = 0.f;
#pragma unroll
        for (int j = 0; j < 64; ++j)
            ss = fmaf(z[j], z[j], ss);
        const float nrm = sqrtf(ss);
        const float inv = nrm > 0.f ? 1.0f / nrm : 0.f;
        if (live) {
            if (t.nrm)
                t.nrm[row] = nrm;
#pragma unroll
            for (int j = 0; j < 64; ++j)
                z[j] *= inv;
            if (t.qhat) {
                float4 *dst = reinterpret_cast<float4 *>(t.qhat + row * 64);
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    dst[j] = make_float4(z[4 * j], z[4 * j + 1], z[4 * j + 2], z[4 * j + 3]);
            }
            if (t.qhat_bf) {
                uint4 *dst = reinterpret_cast<uint4 *>(t.qhat_bf + row * 64);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    dst[j] = pack8_bf16(z + 8 * j);
            }
        }
    } else if (threadIdx.x == 0) {
        atomicOr(t.status, kStatusTimeoutBit);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 256);
    }
}

// ---- exhaustive hub scoring with a fused argmax ------------------------------

// 100 KB keeps at most two CTAs (2 x 256 TMEM columns) on an SM
constexpr int kArgmaxSmem = 100 * 1024;

// One thread per query row keeps the M best (score, hub) pairs, ties to the
// smaller hub index; outputs are nq x M, best first (M = 1: the argmax).
template <int M>
__global__ void __launch_bounds__(128)
    hub_argmax_kernel(const Operand Q, const __nv_bfloat16 *Eb, int H, int64_t nq, const int32_t *hub_nodes,
                      int32_t *out_node, int32_t *out_hub, float *out_score, int *status)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sA = smem;
    uint8_t *sB = smem + 16384;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 49152);
    uint32_t *slot = reinterpret_cast<uint32_t *>(smem + 49152 + 8);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r0 = static_cast<int64_t>(blockIdx.x) * 128;
    const int64_t row = r0 + warp * 32 + lane;
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    if (warp == 0)
        tmem_alloc(slot, 256);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *slot;
    const uint32_t my_lane = tmem + (static_cast<uint32_t>(warp * 32) << 16);
    uint32_t phase = 0;
    const Operand E{Eb, OP_BF16, 64, 1, H, 64, nullptr};
    float best[M];
    int bi[M];
#pragma unroll
    for (int j = 0; j < M; ++j) {
        best[j] = -INFINITY;
        bi[j] = -1;
    }
    bool ok = true;
    for (int c0 = 0; c0 < H && ok; c0 += 256) {
        ok = tc_gemm_tile<256>(Q, r0, E, c0, 64, sA, sB, bar, phase, tmem);
        if (!ok)
            break;
        for (int cc = 0; cc < 256 && c0 + cc < H; cc += 32) {
            float v[32];
            tmem_ld32(my_lane + cc, v);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int col = c0 + cc + j;
                if (col < H && v[j] > best[M - 1]) {  // strict: the first of equal scores wins
                    float sv = v[j];
                    int si = col;
#pragma unroll
                    for (int t = 0; t < M; ++t) {
                        if (sv > best[t]) {
                            const float tv = best[t];
                            const int ti = bi[t];
                            best[t] = sv;
                            bi[t] = si;
                            sv = tv;
                            si = ti;
                        }
                    }
                }
            }
        }
        tc_fence_before();
    }
    if (!ok && threadIdx.x == 0)
        atomicOr(status, kStatusTimeoutBit);
    if (row < nq) {
#pragma unroll
        for (int j = 0; j < M; ++j) {
            const bool good = ok && bi[j] >= 0;
            if (out_hub)
                out_hub[row * M + j] = good ? bi[j] : -1;
            if (out_score)
                out_score[row * M + j] = good ? best[j] : -INFINITY;
            if (out_node)
                out_node[row * M + j] = good ? hub_nodes[bi[j]] : -1;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 256);
    }
}

// ---- exhaustive entry selection in one kernel ----------------------------------

// The query tower and the exhaustive hub scores with the top-M epilogue for
// 128 queries per CTA: GEMM 1 and GEMM 2 of the tower as in
// tower_forward_kernel, q_hat written as BF16 straight into the canonical A
// tile of the hub GEMM (never through global memory), then the hubs in tiles
// of 256 with two B buffers and two TMEM accumulators, so that one tile's
// epilogue overlaps the next tile's load and MMA.  Scores, ties and the
// top-M rule are those of hub_argmax_kernel.
// The weight and hub operands arrive as whole 32 KB canonical images
// (packed once per model) by one bulk copy each (cp.async.bulk, completion
// counted on an mbarrier), issued by thread 0 as soon as their buffer is
// free: each W1 chunk when the MMA before it has read sB, W2 into sB when
// GEMM 1 is done (the load overlaps the GEMM 1 epilogue), the first two hub
// tiles into sH when GEMM 2 is done (overlapping the normalisation), each
// later hub tile when the MMA two tiles back has read its buffer.  Only the
// queries are staged by the threads (FP32 to BF16).
//   shared memory: sA 16 KB (GEMM 1 A chunks, then the q_hat tile), sB 32 KB
//   (W1 chunks, then W2), sH 64 KB (the hidden layer, then the two hub
//   tiles), then the barriers: 112 KB, so that the CTA finds room on an SM
//   that search CTAs of another stream still half occupy; it owns all 512
//   TMEM columns, so one runs per SM.
constexpr int kEntrySmem = 114688 + 64;

struct EntryBars {
    uint64_t mma[2];  // MMA commits (accumulator 0 / 1)
    uint64_t w1, w2;  // W1 chunk and W2 image loads
    uint64_t e[2];    // hub tile loads (buffer 0 / 1)
};

template <int M>
__global__ void __launch_bounds__(128)
    entry_exhaustive_kernel(const TowerArgs t, const uint8_t *packed, int H, const int32_t *hub_nodes,
                            int32_t *out_node)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sA = smem;
    uint8_t *sB = smem + 16384;
    uint8_t *sH = smem + 49152;
    uint8_t *sW = sB;  // W2 after GEMM 1
    uint8_t *sE = sH;  // the hub tiles after GEMM 2
    EntryBars *bars = reinterpret_cast<EntryBars *>(smem + 114688);
    uint32_t *slot = reinterpret_cast<uint32_t *>(smem + 114688 + sizeof(EntryBars));
    int *sfail = reinterpret_cast<int *>(smem + 114688 + sizeof(EntryBars) + 4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m = warp * 32 + lane;
    const int64_t r0 = static_cast<int64_t>(blockIdx.x) * 128;
    const int64_t row = r0 + m;
    const bool live = row < t.nq;
    const bool leader = threadIdx.x == 0;
    const int nc1 = (t.in_dim + 63) / 64, ntiles = (H + 255) / 256;
    const uint8_t *pW1 = packed, *pW2 = packed + static_cast<size_t>(nc1) * 32768,
                  *pE = packed + static_cast<size_t>(nc1 + 1) * 32768;
    // loads issued and waited for, per load barrier (thread 0 only): every
    // issued copy is waited for before the CTA exits
    int w1_iss = 0, w1_wt = 0, w2_iss = 0, w2_wt = 0, e_iss[2] = {0, 0}, e_wt[2] = {0, 0};
    auto load = [&](void *dst, const void *src, uint64_t *bar, int &issued) {
        mbar_arrive_expect_tx(bar, 32768);
        bulk_g2s(dst, src, 32768, bar);
        ++issued;
    };
    // thread 0: wait for the next load on `bar`; on a timeout record the
    // failure (the results are then discarded)
    auto wait_load = [&](uint64_t *bar, int &waited) {
        if (!mbar_wait_bounded(bar, static_cast<uint32_t>(waited & 1), kTcWaitIters))
            *sfail = 1;
        ++waited;
    };

    if (leader) {
        mbar_init(&bars->mma[0], 1);
        mbar_init(&bars->mma[1], 1);
        mbar_init(&bars->w1, 1);
        mbar_init(&bars->w2, 1);
        mbar_init(&bars->e[0], 1);
        mbar_init(&bars->e[1], 1);
        *sfail = 0;
        fence_mbar_init();
        load(sB, pW1, &bars->w1, w1_iss);
    }
    if (warp == 0)
        tmem_alloc(slot, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *slot;
    const uint32_t my_lane = tmem + (static_cast<uint32_t>(warp * 32) << 16);
    uint32_t ph[2] = {0u, 0u};
    bool ok = true;

    // ---- GEMM 1: the queries staged chunk by chunk, W1 chunks by bulk copy
    constexpr uint32_t ID1 = idesc_bf16_f32(128, 256);
    for (int c = 0; c < nc1 && ok; ++c) {
        stage_tile<128, 8>(sA, t.X, r0, static_cast<int64_t>(c) * 64);
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        if (leader) {
            wait_load(&bars->w1, w1_wt);
            if (*sfail) {
                mbar_arrive(&bars->mma[0]);  // no MMA: release the waiters
            } else {
                tc_fence_after();
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    tc_mma(tmem, smem_desc(sA + kk * 256, 128, 1024), smem_desc(sB + kk * 256, 128, 1024), ID1,
                           (c > 0 || kk > 0) ? 1u : 0u);
                tc_commit(&bars->mma[0]);
            }
        }
        ok = tc_wait(&bars->mma[0], ph[0]);
        if (ok && leader) {  // sB is free again: the next W1 chunk, or W2 after the last
            if (c + 1 < nc1)
                load(sB, pW1 + static_cast<size_t>(c + 1) * 32768, &bars->w1, w1_iss);
            else
                load(sW, pW2, &bars->w2, w2_iss);
        }
    }
    if (ok) {
        for (int c0 = 0; c0 < 256; c0 += 32) {
            float v[32];
            tmem_ld32(my_lane + c0, v);
#pragma unroll
            for (int j = 0; j < 32; j += 8) {
                float a[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    a[u] = fmaxf(v[j + u] + t.b1[c0 + j + u], 0.f);
                *reinterpret_cast<uint4 *>(sH + canon_off(m, c0 + j, 32)) = pack8_bf16(a);
            }
        }
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        if (leader) {
            wait_load(&bars->w2, w2_wt);
            if (*sfail) {
                mbar_arrive(&bars->mma[0]);
            } else {
                tc_fence_after();
                constexpr uint32_t ID2 = idesc_bf16_f32(128, 64);
#pragma unroll
                for (int kk = 0; kk < 16; ++kk)
                    tc_mma(tmem, smem_desc(sH + kk * 256, 128, 4096), smem_desc(sW + kk * 256, 128, 4096), ID2,
                           kk > 0 ? 1u : 0u);
                tc_commit(&bars->mma[0]);
            }
        }
        ok = tc_wait(&bars->mma[0], ph[0]);
        if (ok && leader)  // the hidden layer is read: the first two hub tiles into sH
            for (int b = 0; b < 2 && b < ntiles; ++b)
                load(sE + b * 32768, pE + static_cast<size_t>(b) * 32768, &bars->e[b], e_iss[b]);
    }
    if (ok) {
        float z[64];
        float v[32];
        tmem_ld32(my_lane, v);
#pragma unroll
        for (int j = 0; j < 32; ++j)
            z[j] = v[j] + t.b2[j];
        tmem_ld32(my_lane + 32, v);
#pragma unroll
        for (int j = 0; j < 32; ++j)
            z[32 + j] = v[j] + t.b2[32 + j];
        float ss = 0.f;
#pragma unroll
        for (int j = 0; j < 64; ++j)
            ss = fmaf(z[j], z[j], ss);
        const float nrm = sqrtf(ss);
        const float inv = nrm > 0.f ? 1.0f / nrm : 0.f;
#pragma unroll
        for (int j = 0; j < 64; ++j)
            z[j] *= inv;
        if (live && t.qhat) {
            float4 *dst = reinterpret_cast<float4 *>(t.qhat + row * 64);
#pragma unroll
            for (int j = 0; j < 16; ++j)
                dst[j] = make_float4(z[4 * j], z[4 * j + 1], z[4 * j + 2], z[4 * j + 3]);
        }
        // q_hat as the A operand of the hub GEMM (rows past nq hold zeros'
        // embeddings and are never written out)
#pragma unroll
        for (int j = 0; j < 64; j += 8)
            *reinterpret_cast<uint4 *>(sA + canon_off(m, j, 8)) = pack8_bf16(z + j);
    }
    // ---- hub scores in tiles of 256, double buffered
    float best[M];
    int bi[M];
#pragma unroll
    for (int j = 0; j < M; ++j) {
        best[j] = -INFINITY;
        bi[j] = -1;
    }
    constexpr uint32_t IDH = idesc_bf16_f32(128, 256);
    auto issue = [&](int tile) {
        // the MMA of hub tile `tile` (buffer and accumulator tile & 1) once
        // its image has landed
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        if (leader) {
            wait_load(&bars->e[tile & 1], e_wt[tile & 1]);
            if (*sfail) {
                mbar_arrive(&bars->mma[tile & 1]);
            } else {
                tc_fence_after();
                const uint8_t *b = sE + (tile & 1) * 32768;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    tc_mma(tmem + (tile & 1) * 256, smem_desc(sA + kk * 256, 128, 1024),
                           smem_desc(b + kk * 256, 128, 1024), IDH, kk > 0 ? 1u : 0u);
                tc_commit(&bars->mma[tile & 1]);
            }
        }
    };
    if (ok)
        issue(0);
    for (int tile = 0; tile < ntiles && ok; ++tile) {
        if (tile + 1 < ntiles)
            issue(tile + 1);  // overlaps this tile's wait and epilogue
        if (!(ok = tc_wait(&bars->mma[tile & 1], ph[tile & 1])))
            break;
        if (leader && tile + 2 < ntiles)  // this tile's buffer is free again
            load(sE + (tile & 1) * 32768, pE + static_cast<size_t>(tile + 2) * 32768, &bars->e[tile & 1],
                 e_iss[tile & 1]);
        const int c0 = tile * 256;
        for (int cc = 0; cc < 256 && c0 + cc < H; cc += 32) {
            float v[32];
            tmem_ld32(my_lane + (tile & 1) * 256 + cc, v);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int col = c0 + cc + j;
                if (col < H && v[j] > best[M - 1]) {  // strict: the first of equal scores wins
                    float sv = v[j];
                    int si = col;
#pragma unroll
                    for (int u = 0; u < M; ++u) {
                        if (sv > best[u]) {
                            const float tv = best[u];
                            const int ti = bi[u];
                            best[u] = sv;
                            bi[u] = si;
                            sv = tv;
                            si = ti;
                        }
                    }
                }
            }
        }
        tc_fence_before();  // these TMEM reads end before the MMA that reuses the accumulator
    }
    const bool failed = __syncthreads_or(leader && *sfail) || !ok;
    if (failed && leader)
        atomicOr(t.status, kStatusTimeoutBit);
    if (live) {
#pragma unroll
        for (int j = 0; j < M; ++j)
            out_node[row * M + j] = (!failed && bi[j] >= 0) ? hub_nodes[bi[j]] : -1;
    }
    if (leader) {
        // every copy issued lands before the CTA's shared memory goes away
        auto drain = [&](uint64_t *bar, int &waited, int issued) {
            for (; waited < issued; ++waited)
                mbar_wait_bounded(bar, static_cast<uint32_t>(waited & 1), kTcWaitIters);
        };
        drain(&bars->w1, w1_wt, w1_iss);
        drain(&bars->w2, w2_wt, w2_iss);
        drain(&bars->e[0], e_wt[0], e_iss[0]);
        drain(&bars->e[1], e_wt[1], e_iss[1]);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// ---- model preparation ------------------------------------------------------

// Canonical K-major images (the layout stage_tile writes: 16-byte chunk c of
// an image holds row (c / (8 KG)) * 8 + c % 8 and k-chunk (c / 8) % KG) of a
// row-major BF16 matrix src [rows][cols], one 16-byte chunk per thread.
// Image (tr, tk), at out + (tr * ntk + tk) * ROWS * KG * 16, holds rows
// [tr * ROWS, +ROWS) x columns [tk * 8 KG, +8 KG), zero outside the matrix.
__global__ void pack_canonical_kernel(const __nv_bfloat16 *src, int64_t rows, int cols, int ROWS, int KG, int ntr,
                                      int ntk, uint8_t *out)
{
    const int64_t per = static_cast<int64_t>(ROWS) * KG;
    const int64_t total = per * ntr * ntk;
    const unsigned short *bits = reinterpret_cast<const unsigned short *>(src);
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t img = i / per;
        const int c = static_cast<int>(i % per);
        const int64_t r = (img / ntk) * ROWS + (c / (8 * KG)) * 8 + (c & 7);
        const int64_t k = (img % ntk) * 8 * KG + ((c >> 3) % KG) * 8;
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t lo = (r < rows && k + 2 * j < cols) ? bits[r * cols + k + 2 * j] : 0u;
            const uint32_t hi = (r < rows && k + 2 * j + 1 < cols) ? bits[r * cols + k + 2 * j + 1] : 0u;
            w[j] = lo | (hi << 16);
        }
        reinterpret_cast<uint4 *>(out)[i] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// BF16 transposed weight copies for K-major B operands, and normalised hub
// embeddings (FP32 and BF16)
__global__ void prepare_model_kernel(const float *W1, const float *W2, const float *E, int in_dim, int H,
                                     __nv_bfloat16 *W1t, __nv_bfloat16 *W2t, float *En, __nv_bfloat16 *Eb)
{
    const int64_t tid = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    const int64_t n1 = static_cast<int64_t>(in_dim) * 256, n2 = 256 * 64;
    if (tid < n1) {
        const int n = static_cast<int>(tid / in_dim), k = static_cast<int>(tid % in_dim);
        W1t[tid] = __float2bfloat16_rn(W1[static_cast<int64_t>(k) * 256 + n]);
    } else if (tid < n1 + n2) {
        const int64_t i = tid - n1;
        const int n = static_cast<int>(i / 256), k = static_cast<int>(i % 256);
        W2t[i] = __float2bfloat16_rn(W2[k * 64 + n]);
    } else if (tid < n1 + n2 + H) {
        const int64_t h = tid - n1 - n2;
        float ss = 0.f;
        for (int j = 0; j < 64; ++j)
            ss = fmaf(E[h * 64 + j], E[h * 64 + j], ss);
        const float inv = ss > 0.f ? rsqrtf(ss) : 0.f;
        for (int j = 0; j < 64; ++j) {
            const float v = E[h * 64 + j] * inv;
            En[h * 64 + j] = v;
            Eb[h * 64 + j] = __float2bfloat16_rn(v);
        }
    }
}

// hub with the largest cosine to the mean raw embedding (first maximum)
__global__ void hub_entry_kernel(const float *E, int H, int32_t *out)
{
    __shared__ float mean[64];
    __shared__ float best_v[256];
    __shared__ int best_i[256];
    const int t = threadIdx.x;
    if (t < 64) {
        float s = 0.f;
        for (int h = 0; h < H; ++h)
            s += E[static_cast<int64_t>(h) * 64 + t];
        mean[t] = s / static_cast<float>(H);
    }
    __syncthreads();
    float mn = 0.f;
    for (int j = 0; j < 64; ++j)
        mn = fmaf(mean[j], mean[j], mn);
    mn = sqrtf(mn);
    float bv = -INFINITY;
    int bidx = 0x7fffffff;
    for (int h = t; h < H; h += blockDim.x) {
        float dot = 0.f, ee = 0.f;
        for (int j = 0; j < 64; ++j) {
            const float e = E[static_cast<int64_t>(h) * 64 + j];
            dot = fmaf(e, mean[j], dot);
            ee = fmaf(e, e, ee);
        }
        const float c = dot / (sqrtf(ee) * mn);
        if (c > bv) {
            bv = c;
            bidx = h;
        }
    }
    best_v[t] = bv;
    best_i[t] = bidx;
    __syncthreads();
    if (t == 0) {
        float v = best_v[0];
        int i = best_i[0];
        for (int u = 1; u < blockDim.x; ++u)
            if (best_v[u] > v || (best_v[u] == v && best_i[u] < i)) {
                v = best_v[u];
                i = best_i[u];
            }
        *out = i;
    }
}

// Seed sets from the hub-graph search: out[i*m + j] = node of the j-th hub
// found for query i; a missing first hub falls back to the medoid, a missing
// later one is an unused slot (-1).
__global__ void map_hub_seeds(const int32_t *hub_ids, int64_t nq, int m, const int32_t *hub_nodes,
                              int32_t medoid, int32_t *out)
{
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i < nq * m) {
        const int32_t h = hub_ids[i];
        out[i] = h >= 0 ? hub_nodes[h] : (i % m == 0 ? medoid : -1);
    }
}

// Every query's seed set is the model's hub sample: out[i] = seeds[i mod n]
// for i < ns (the nq x n seed array of the general search on the hub index).
__global__ void broadcast_hub_seeds(const int32_t *seeds, int n, int64_t ns, int32_t *out)
{
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i < ns)
        out[i] = seeds[i % n];
}

// ---- hub-graph search (Sec. 4.3: Algorithm 1 on the high-tier hub graph) ----
// One warp per query, pools of at most 32 hubs: lane i holds the i-th
// smallest (score, hub) key of the pool (bit 0: expanded), so a step is a
// ballot for the first unexpanded entry, one adjacency row read by lanes
// 0..s-1, a visited test-and-set in a per-warp shared-memory bitmap over the
// hubs, the fresh neighbours scored lane-parallel (-q_hat . e_hat in FP32
// over the BF16 hub rows) and inserted into the pool one by one (rank by
// ballot, shift by shuffle), truncated to L.  The steps and the pool
// follow the sorted-pool reading of Algorithm 1 with W = 1: the pool is the
// L smallest keys of every hub evaluated, a hub is evaluated once, the search
// stops when no unexpanded entry is left.  The m best pool entries become the
// seeds (their hubs' nodes).
constexpr int kNavWarps = 8;
constexpr int kNavMaxPool = 64;

// <q, e> over NC 16-byte chunks (8 coordinates each) of a BF16 hub row, with
// four FP32 accumulators over coordinates j mod 4
template <int NC>
__device__ __forceinline__ float hub_dot(const float *q, const __nv_bfloat16 *row)
{
    const uint4 *r4 = reinterpret_cast<const uint4 *>(row);
    const float4 *q4 = reinterpret_cast<const float4 *>(q);
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll 4
    for (int c = 0; c < NC; ++c) {
        const uint4 x = __ldg(r4 + c);
        const float4 qa = q4[2 * c], qb = q4[2 * c + 1];
        const float2 f0 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&x.x));
        const float2 f1 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&x.y));
        const float2 f2 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&x.z));
        const float2 f3 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&x.w));
        a0 = fmaf(f0.x, qa.x, a0);
        a1 = fmaf(f0.y, qa.y, a1);
        a2 = fmaf(f1.x, qa.z, a2);
        a3 = fmaf(f1.y, qa.w, a3);
        a0 = fmaf(f2.x, qb.x, a0);
        a1 = fmaf(f2.y, qb.y, a1);
        a2 = fmaf(f3.x, qb.z, a2);
        a3 = fmaf(f3.y, qb.w, a3);
    }
    return (a0 + a1) + (a2 + a3);
}

// -<q, e> over the whole 64-coordinate row
__device__ __forceinline__ float hub_score(const float *q, const __nv_bfloat16 *row) { return -hub_dot<8>(q, row); }

// The fresh keys of a warp (cand != kKeyMax on the lanes that hold one) enter
// the pool one at a time: a key's rank is the count of smaller pool keys (one
// ballot per register), the keys from that rank on move up one place and the
// L-th drops out, so the pool stays the L smallest keys evaluated, the set a
// sort and merge of all the new keys would give.  A key not below the pool's
// L-th key when the insertion starts cannot enter (that key only gets
// smaller), so such keys are dropped before the serial loop.
template <int NP>
__device__ __forceinline__ void nav_insert(uint64_t (&pool)[NP], uint64_t cand, int L, int lane)
{
    const int lr = (L - 1) >> 5, ll = (L - 1) & 31;
    uint64_t worst = kKeyMax;  // the L-th smallest key, kKeyMax while the pool has room
#pragma unroll
    for (int r = 0; r < NP; ++r) {
        const uint64_t v = __shfl_sync(kFull, pool[r], ll);
        if (r == lr)
            worst = v;
    }
    unsigned fresh = __ballot_sync(kFull, cand < worst);
    while (fresh) {
        const int src = __ffs(fresh) - 1;
        fresh &= fresh - 1;
        const uint64_t c = __shfl_sync(kFull, cand, src);
        int rank = 0;
#pragma unroll
        for (int r = 0; r < NP; ++r)
            rank += __popc(__ballot_sync(kFull, pool[r] < c));
        if (rank >= L)
            continue;
        uint64_t below = c;  // what lane 0 of the next register takes
#pragma unroll
        for (int r = 0; r < NP; ++r) {
            const uint64_t up = __shfl_up_sync(kFull, pool[r], 1);
            const uint64_t top = __shfl_sync(kFull, pool[r], 31);
            const int idx = r * 32 + lane;
            uint64_t v = pool[r];
            if (idx == rank)
                v = c;
            else if (idx > rank)
                v = lane == 0 ? below : up;
            pool[r] = idx < L ? v : kKeyMax;
            below = top;
        }
    }
}

// <q, e> over the 8 coordinates 8 sub .. 8 sub + 7 of a BF16 hub row, q in
// registers (qr), one FP32 accumulator in coordinate order
__device__ __forceinline__ float hub_dot8(const float (&qr)[8], const __nv_bfloat16 *row, int sub)
{
    const uint4 x = __ldg(reinterpret_cast<const uint4 *>(row) + sub);
    const float2 f0 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&x.x));
    const float2 f1 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&x.y));
    const float2 f2 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&x.z));
    const float2 f3 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&x.w));
    float a = f0.x * qr[0];
    a = fmaf(f0.y, qr[1], a);
    a = fmaf(f1.x, qr[2], a);
    a = fmaf(f1.y, qr[3], a);
    a = fmaf(f2.x, qr[4], a);
    a = fmaf(f2.y, qr[5], a);
    a = fmaf(f3.x, qr[6], a);
    return fmaf(f3.y, qr[7], a);
}

// NP keys per lane: pools of up to 32 * NP hubs (element r * 32 + lane in
// pool[r]).
// A step scores its fresh neighbours four at a time, eight lanes per
// neighbour: lane 8g + sub keeps coordinates 8 sub .. 8 sub + 7 of q_hat in
// registers, reads the matching 16 bytes of the hub row and the group adds
// its eight partial products by three xor-shuffles.  So q_hat is read from
// shared memory once per query instead of once per scored neighbour, and
// only fresh neighbours are scored (their ids are compacted through shared
// memory first).
// Registers are capped at 40 (six 8-warp CTAs per SM; no spills with one or
// two keys per lane): the eight q_hat coordinates per lane do not fit the 32
// that eight CTAs would leave.
template <int NP>
__global__ void __launch_bounds__(32 * kNavWarps, 6)
    hub_nav_kernel(const float *qhat, int64_t nq, const __nv_bfloat16 *Eb, int H, const int32_t *hgraph, int s,
                   const int32_t *start, int n_start, int L, int m_seeds, const int32_t *hub_nodes, int32_t medoid,
                   int bm_words, unsigned *counter, int32_t *out)
{
    extern __shared__ __align__(16) uint8_t nav_smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int sub = lane & 7, grp = lane >> 3;
    const int per_warp = 256 + 128 + 4 * bm_words;
    float *q = reinterpret_cast<float *>(nav_smem + wid * per_warp);
    int32_t *fresh_ids = reinterpret_cast<int32_t *>(nav_smem + wid * per_warp + 256);
    uint32_t *vis = reinterpret_cast<uint32_t *>(nav_smem + wid * per_warp + 384);
    for (;;) {
        // the next query from the launch's work queue (the grid holds only
        // resident warps, so the batch's last queries go to whichever warps
        // finish first)
        unsigned u = 0;
        if (lane == 0)
            u = atomicAdd(counter, 1u);
        const int64_t qi = __shfl_sync(kFull, u, 0);
        if (qi >= nq)
            break;
        if (lane < 16)
            reinterpret_cast<float4 *>(q)[lane] = reinterpret_cast<const float4 *>(qhat + qi * 64)[lane];
        for (int w = lane; w < bm_words; w += 32)
            vis[w] = 0u;
        __syncwarp();
        float qr[8];
        {
            const float4 lo = reinterpret_cast<const float4 *>(q)[2 * sub];
            const float4 hi = reinterpret_cast<const float4 *>(q)[2 * sub + 1];
            qr[0] = lo.x, qr[1] = lo.y, qr[2] = lo.z, qr[3] = lo.w;
            qr[4] = hi.x, qr[5] = hi.y, qr[6] = hi.z, qr[7] = hi.w;
        }
        uint64_t pool[NP];
#pragma unroll
        for (int r = 0; r < NP; ++r)
            pool[r] = kKeyMax;
        {
            // the initial pool (Algorithm 1 starts from a set of nodes): the
            // model's hub sample, or the entry hub alone; every distinct
            // start hub is evaluated once and the L best start the pool
            uint64_t cand = kKeyMax;
            if (lane < n_start) {
                const int32_t hb = __ldg(start + lane);
                const uint32_t bit = 1u << (hb & 31);
                if (!(atomicOr(&vis[hb >> 5], bit) & bit))
                    cand = make_key(f32_to_ord(hub_score(q, Eb + static_cast<int64_t>(hb) * 64)), hb);
            }
            nav_insert<NP>(pool, cand, L, lane);
        }
        for (;;) {
            // the first unexpanded entry in pool order
            int f = -1, fr = 0;
#pragma unroll
            for (int r = NP - 1; r >= 0; --r) {
                const unsigned um =
                    __ballot_sync(kFull, r * 32 + lane < L && pool[r] != kKeyMax && !(pool[r] & 1ull));
                if (um) {
                    f = __ffs(um) - 1;
                    fr = r;
                }
            }
            if (f < 0)
                break;
            int32_t node = 0;
#pragma unroll
            for (int r = 0; r < NP; ++r) {
                if (r == fr && lane == f)
                    pool[r] |= 1ull;
                const int32_t v = __shfl_sync(kFull, key_id(pool[r]), f);
                if (r == fr)
                    node = v;
            }
            // the adjacency row (lane j holds neighbour j; -1 pads a short
            // row), the visited test-and-set, the fresh ids compacted
            const int32_t nb = lane < s ? __ldg(hgraph + static_cast<int64_t>(node) * s + lane) : -1;
            bool fresh = false;
            if (nb >= 0 && nb < H) {
                const uint32_t bit = 1u << (nb & 31);
                fresh = !(atomicOr(&vis[nb >> 5], bit) & bit);
            }
            const unsigned fm = __ballot_sync(kFull, fresh);
            if (fresh)
                fresh_ids[__popc(fm & lanemask_lt())] = nb;
            __syncwarp();
            const int nf = __popc(fm);
            for (int p = 0; p < nf; p += 4) {
                const int i = p + grp;
                const int32_t hb = i < nf ? fresh_ids[i] : -1;
                float part = hb >= 0 ? hub_dot8(qr, Eb + static_cast<int64_t>(hb) * 64, sub) : 0.f;
                part += __shfl_xor_sync(kFull, part, 1);
                part += __shfl_xor_sync(kFull, part, 2);
                part += __shfl_xor_sync(kFull, part, 4);
                const uint64_t cand = hb >= 0 && sub == 0 ? make_key(f32_to_ord(-part), hb) : kKeyMax;
                nav_insert<NP>(pool, cand, L, lane);
            }
            __syncwarp();
        }
        if (lane < m_seeds) {
            const int32_t hub = pool[0] != kKeyMax ? key_id(pool[0]) : -1;
            out[qi * m_seeds + lane] = hub >= 0 ? hub_nodes[hub] : (lane == 0 ? medoid : -1);
        }
        __syncwarp();
    }
}

// medoid seed sets: the medoid first, the other slots unused
__global__ void fill_medoid_seeds(int32_t *out, int64_t nq, int m, int32_t medoid)
{
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i < nq * m)
        out[i] = i % m == 0 ? medoid : -1;
}

template <typename T>
T *dev_alloc(size_t count, cudaError_t &e)
{
    T *p = nullptr;
    if (e == cudaSuccess)
        e = cudaMalloc(reinterpret_cast<void **>(&p), count * sizeof(T));
    return p;
}

}  // namespace

void free_model(ann_entry_model *m)
{
    if (!m)
        return;
    cudaFree(m->W1);
    cudaFree(m->b1);
    cudaFree(m->W2);
    cudaFree(m->b2);
    cudaFree(m->E);
    cudaFree(m->W1t);
    cudaFree(m->W2t);
    cudaFree(m->En);
    cudaFree(m->Eb);
    cudaFree(m->packed);
    cudaFree(m->hub_nodes);
    cudaFree(m->hub_graph);
    cudaFree(m->hub_seeds);
    if (m->hub_index)
        ann_free_index(m->hub_index);
    delete m;
}

size_t packed_model_bytes(int in_dim, int H)
{
    return static_cast<size_t>((in_dim + 63) / 64 + 1 + (H + 255) / 256) * 32768;
}

ann_status prepare_model(ann_entry_model *m, cudaStream_t s)
{
    const int64_t total = static_cast<int64_t>(m->in_dim) * 256 + 256 * 64 + m->H;
    prepare_model_kernel<<<static_cast<unsigned>((total + 255) / 256), 256, 0, s>>>(
        m->W1, m->W2, m->E, m->in_dim, m->H, m->W1t, m->W2t, m->En, m->Eb);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && m->packed) {
        // W1^T in 64-wide k chunks of 256 rows, W2^T (64 rows x 256), the
        // hubs in tiles of 256 rows x 64
        const int nc1 = (m->in_dim + 63) / 64, nt = (m->H + 255) / 256;
        pack_canonical_kernel<<<256, 256, 0, s>>>(m->W1t, 256, m->in_dim, 256, 8, 1, nc1, m->packed);
        pack_canonical_kernel<<<256, 256, 0, s>>>(m->W2t, 64, 256, 64, 32, 1, 1,
                                                  m->packed + static_cast<size_t>(nc1) * 32768);
        pack_canonical_kernel<<<256, 256, 0, s>>>(m->Eb, m->H, 64, 256, 8, nt, 1,
                                                  m->packed + static_cast<size_t>(nc1 + 1) * 32768);
        e = cudaGetLastError();
    }
    return cuda_status(e);
}

ann_status launch_tower(const ann_entry_model *m, const Operand &X, int64_t nq, float *qhat,
                        __nv_bfloat16 *qhat_bf, float *z1, __nv_bfloat16 *a1, float *nrm, int *status,
                        cudaStream_t s)
{
    if (nq == 0)
        return ANN_OK;
    TowerArgs t{};
    t.X = X;
    t.W1t = m->W1t;
    t.in_dim = m->in_dim;
    t.b1 = m->b1;
    t.W2t = m->W2t;
    t.b2 = m->b2;
    t.nq = nq;
    t.qhat = qhat;
    t.qhat_bf = qhat_bf;
    t.z1 = z1;
    t.a1 = a1;
    t.nrm = nrm;
    t.status = status;
    cudaError_t e = cudaFuncSetAttribute(tower_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kTowerSmem);
    if (e != cudaSuccess)
        return cuda_status(e);
    tower_forward_kernel<<<static_cast<unsigned>((nq + 127) / 128), 128, kTowerSmem, s>>>(t);
    return cuda_status(cudaGetLastError());
}

template <int M>
ann_status launch_hub_topm(const ann_entry_model *m, const Operand &Q, int64_t nq, int32_t *out_node,
                           int32_t *out_hub, float *out_score, int *status, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(hub_argmax_kernel<M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kArgmaxSmem);
    if (e != cudaSuccess)
        return cuda_status(e);
    hub_argmax_kernel<M><<<static_cast<unsigned>((nq + 127) / 128), 128, kArgmaxSmem, s>>>(
        Q, m->Eb, m->H, nq, m->hub_nodes, out_node, out_hub, out_score, status);
    return cuda_status(cudaGetLastError());
}

ann_status launch_hub_argmax(const ann_entry_model *m, const Operand &Q, int64_t nq, int32_t *out_node,
                             int32_t *out_hub, float *out_score, int *status, cudaStream_t s, int topm)
{
    if (nq == 0)
        return ANN_OK;
    switch (topm) {
    case 1: return launch_hub_topm<1>(m, Q, nq, out_node, out_hub, out_score, status, s);
    case 2: return launch_hub_topm<2>(m, Q, nq, out_node, out_hub, out_score, status, s);
    case 3: return launch_hub_topm<3>(m, Q, nq, out_node, out_hub, out_score, status, s);
    case 4: return launch_hub_topm<4>(m, Q, nq, out_node, out_hub, out_score, status, s);
    case 5: return launch_hub_topm<5>(m, Q, nq, out_node, out_hub, out_score, status, s);
    case 6: return launch_hub_topm<6>(m, Q, nq, out_node, out_hub, out_score, status, s);
    case 7: return launch_hub_topm<7>(m, Q, nq, out_node, out_hub, out_score, status, s);
    case 8: return launch_hub_topm<8>(m, Q, nq, out_node, out_hub, out_score, status, s);
    default: return ANN_ERR_INVALID_ARG;
    }
}

template <int M>
ann_status launch_entry_topm(const ann_entry_model *m, const Operand &X, int64_t nq, float *qhat, int32_t *out_node,
                             int *status, cudaStream_t s)
{
    TowerArgs t{};
    t.X = X;
    t.W1t = m->W1t;
    t.in_dim = m->in_dim;
    t.b1 = m->b1;
    t.W2t = m->W2t;
    t.b2 = m->b2;
    t.nq = nq;
    t.qhat = qhat;
    t.status = status;
    cudaError_t e = cudaFuncSetAttribute(entry_exhaustive_kernel<M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kEntrySmem);
    if (e != cudaSuccess)
        return cuda_status(e);
    entry_exhaustive_kernel<M><<<static_cast<unsigned>((nq + 127) / 128), 128, kEntrySmem, s>>>(
        t, m->packed, m->H, m->hub_nodes, out_node);
    return cuda_status(cudaGetLastError());
}

ann_status launch_entry_exhaustive(const ann_entry_model *m, const Operand &X, int64_t nq, float *qhat,
                                   int32_t *out_node, int topm, int *status, cudaStream_t s)
{
    if (nq == 0)
        return ANN_OK;
    if (!m->packed)  // only index models carry the packed operand images
        return ANN_ERR_INVALID_ARG;
    switch (topm) {
    case 1: return launch_entry_topm<1>(m, X, nq, qhat, out_node, status, s);
    case 2: return launch_entry_topm<2>(m, X, nq, qhat, out_node, status, s);
    case 3: return launch_entry_topm<3>(m, X, nq, qhat, out_node, status, s);
    case 4: return launch_entry_topm<4>(m, X, nq, qhat, out_node, status, s);
    case 5: return launch_entry_topm<5>(m, X, nq, qhat, out_node, status, s);
    case 6: return launch_entry_topm<6>(m, X, nq, qhat, out_node, status, s);
    case 7: return launch_entry_topm<7>(m, X, nq, qhat, out_node, status, s);
    case 8: return launch_entry_topm<8>(m, X, nq, qhat, out_node, status, s);
    default: return ANN_ERR_INVALID_ARG;
    }
}

ann_status build_hub_index(ann_index *idx, ann_entry_model *m, const int32_t *hub_graph, int32_t hub_entry,
                           cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    if (!m->hub_graph)
        m->hub_graph = dev_alloc<int32_t>(static_cast<size_t>(m->H) * m->s, e);
    if (e != cudaSuccess)
        return cuda_status(e);
    if (hub_graph) {
        e = cudaMemcpyAsync(m->hub_graph, hub_graph, static_cast<size_t>(m->H) * m->s * 4, cudaMemcpyDefault, s);
    } else {
        // the s most cosine-similar other hubs (smaller index on ties)
        void *dd = nullptr;
        e = cudaMallocAsync(&dd, static_cast<size_t>(m->H) * m->s * 4, s);
        if (e == cudaSuccess) {
            ann_status st = knn_exact(m->En, m->H, 64, ANN_F32, ANN_IP, m->En, m->H, m->s, true, m->hub_graph, dd, s);
            cudaFreeAsync(dd, s);
            if (st != ANN_OK)
                return st;
        }
    }
    if (e != cudaSuccess)
        return cuda_status(e);
    if (hub_entry >= 0) {
        m->hub_entry = hub_entry;
    } else {
        int32_t *d = nullptr;
        e = cudaMallocAsync(reinterpret_cast<void **>(&d), 4, s);
        if (e == cudaSuccess) {
            hub_entry_kernel<<<1, 256, 0, s>>>(m->E, m->H, d);
            e = cudaMemcpyAsync(&m->hub_entry, d, 4, cudaMemcpyDeviceToHost, s);
            cudaFreeAsync(d, s);
        }
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(s);
        if (e != cudaSuccess)
            return cuda_status(e);
    }
    // the start list of the hub-graph search: the entry hub until a sample is
    // set (a rebuilt graph keeps the model's list)
    if (!m->hub_seeds) {
        m->hub_seeds = dev_alloc<int32_t>(ANN_MAX_SEEDS, e);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(m->hub_seeds, &m->hub_entry, 4, cudaMemcpyHostToDevice, s);
        m->n_hub_seeds = 0;
    }
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return cuda_status(e);
    if (m->hub_index) {
        ann_free_index(m->hub_index);
        m->hub_index = nullptr;
    }
    ann_index_desc d{};
    d.n = m->H;
    d.dim = 64;
    d.degree = m->s;
    d.dtype = ANN_BF16;
    d.metric = ANN_IP;
    d.base = m->Eb;
    d.graph = m->hub_graph;
    d.medoid = m->hub_entry;
    d.base_f32 = nullptr;
    ann_status st = ann_index_create(&d, idx->device, &m->hub_index);
    if (st == ANN_OK)
        m->hub_index->status_sink = idx->d_status;  // hub-graph search errors reach the parent's status
    return st;
}

}  // namespace ann

using namespace ann;

extern "C" {

ann_status ann_set_entry_model(ann_index *idx, const ann_entry_model_desc *md, void *stream)
{
    if (!idx || !md)
        return ANN_ERR_INVALID_ARG;
    if (md->in_dim != idx->dim || md->hidden != 256 || md->out_dim != 64 || md->in_dim > 512 ||
        md->n_hubs < 2 || md->hub_degree < 1 || md->hub_degree > 32 || md->hub_degree >= md->n_hubs ||
        !md->W1 || !md->b1 || !md->W2 || !md->b2 || !md->hub_nodes || !md->hub_emb ||
        md->hub_entry >= md->n_hubs)
        return ANN_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(idx->device);
    ann_entry_model *m = new (std::nothrow) ann_entry_model();
    if (!m) {
        cudaSetDevice(prev);
        return ANN_ERR_OOM;
    }
    m->in_dim = md->in_dim;
    m->H = md->n_hubs;
    m->s = md->hub_degree;
    const int H = m->H;
    cudaError_t e = cudaSuccess;
    m->W1 = dev_alloc<float>(static_cast<size_t>(m->in_dim) * 256, e);
    m->b1 = dev_alloc<float>(256, e);
    m->W2 = dev_alloc<float>(256 * 64, e);
    m->b2 = dev_alloc<float>(64, e);
    m->E = dev_alloc<float>(static_cast<size_t>(H) * 64, e);
    m->W1t = dev_alloc<__nv_bfloat16>(static_cast<size_t>(m->in_dim) * 256, e);
    m->W2t = dev_alloc<__nv_bfloat16>(256 * 64, e);
    m->En = dev_alloc<float>(static_cast<size_t>(H) * 64, e);
    m->Eb = dev_alloc<__nv_bfloat16>(static_cast<size_t>(H) * 64, e);
    m->packed = dev_alloc<uint8_t>(packed_model_bytes(m->in_dim, H), e);
    m->hub_nodes = dev_alloc<int32_t>(H, e);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->W1, md->W1, static_cast<size_t>(m->in_dim) * 256 * 4, cudaMemcpyDefault, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->b1, md->b1, 256 * 4, cudaMemcpyDefault, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->W2, md->W2, 256 * 64 * 4, cudaMemcpyDefault, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->b2, md->b2, 64 * 4, cudaMemcpyDefault, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->E, md->hub_emb, static_cast<size_t>(H) * 64 * 4, cudaMemcpyDefault, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m->hub_nodes, md->hub_nodes, static_cast<size_t>(H) * 4, cudaMemcpyDefault, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    ann_status st = cuda_status(e);
    if (st == ANN_OK) {
        // hub node ids must be valid nodes
        std::vector<int32_t> hn(H);
        st = cuda_status(cudaMemcpy(hn.data(), m->hub_nodes, static_cast<size_t>(H) * 4, cudaMemcpyDeviceToHost));
        for (int i = 0; st == ANN_OK && i < H; ++i)
            if (hn[i] < 0 || hn[i] >= idx->n)
                st = ANN_ERR_INVALID_ARG;
    }
    if (st == ANN_OK)
        st = prepare_model(m, s);
    if (st == ANN_OK)
        st = build_hub_index(idx, m, md->hub_graph, md->hub_entry, s);
    if (st != ANN_OK) {
        free_model(m);
        cudaSetDevice(prev);
        return st;
    }
    free_model(idx->model);
    idx->model = m;
    cudaSetDevice(prev);
    return ANN_OK;
}

ann_status ann_get_entry_model(const ann_index *idx, float *W1, float *b1, float *W2, float *b2, float *hub_emb,
                               int32_t *hub_nodes, int32_t *hub_graph, int32_t *hub_entry)
{
    if (!idx || !idx->model)
        return ANN_ERR_INVALID_ARG;
    const ann_entry_model *m = idx->model;
    cudaError_t e = cudaSuccess;
    auto cp = [&](void *dst, const void *src, size_t bytes) {
        if (dst && e == cudaSuccess)
            e = cudaMemcpy(dst, src, bytes, cudaMemcpyDefault);
    };
    cp(W1, m->W1, static_cast<size_t>(m->in_dim) * 256 * 4);
    cp(b1, m->b1, 256 * 4);
    cp(W2, m->W2, 256 * 64 * 4);
    cp(b2, m->b2, 64 * 4);
    cp(hub_emb, m->E, static_cast<size_t>(m->H) * 64 * 4);
    cp(hub_nodes, m->hub_nodes, static_cast<size_t>(m->H) * 4);
    cp(hub_graph, m->hub_graph, static_cast<size_t>(m->H) * m->s * 4);
    if (hub_entry)
        *hub_entry = m->hub_entry;
    return cuda_status(e);
}

ann_status ann_build_hub_graph(ann_index *idx, int32_t s_nn, int32_t max_degree, void *stream)
{
    if (!idx)
        return ANN_ERR_INVALID_ARG;
    ann_entry_model *m = idx->model;
    if (!m)
        return ANN_ERR_UNSUPPORTED;
    const int H = m->H;
    if (s_nn < 1 || s_nn > 32 || s_nn >= H || (max_degree != 0 && (max_degree < s_nn || max_degree > 32)))
        return ANN_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(idx->device);
    const int width = max_degree ? max_degree : s_nn;
    // each hub's s most cosine-similar other hubs (inner products of the
    // normalised embeddings, smaller index on ties)
    cudaError_t e = cudaSuccess;
    int32_t *d_ids = dev_alloc<int32_t>(static_cast<size_t>(H) * s_nn, e);
    float *d_sc = dev_alloc<float>(static_cast<size_t>(H) * s_nn, e);
    ann_status st = cuda_status(e);
    if (st == ANN_OK)
        st = knn_exact(m->En, H, 64, ANN_F32, ANN_IP, m->En, H, s_nn, true, d_ids, d_sc, s);
    std::vector<int32_t> nn(static_cast<size_t>(H) * s_nn);
    std::vector<float> En;
    if (st == ANN_OK)
        st = cuda_status(cudaMemcpyAsync(nn.data(), d_ids, nn.size() * 4, cudaMemcpyDeviceToHost, s));
    if (st == ANN_OK && max_degree) {
        En.resize(static_cast<size_t>(H) * 64);
        st = cuda_status(cudaMemcpyAsync(En.data(), m->En, En.size() * 4, cudaMemcpyDeviceToHost, s));
    }
    if (st == ANN_OK)
        st = cuda_status(cudaStreamSynchronize(s));
    cudaFree(d_ids);
    cudaFree(d_sc);
    std::vector<int32_t> rows(static_cast<size_t>(H) * width, -1);
    if (st == ANN_OK && !max_degree) {
        rows = nn;
    } else if (st == ANN_OK) {
        // undirected edges: u and v are linked when either lists the other;
        // a hub's neighbours in decreasing cosine (smaller index on ties), at
        // most max_degree of them (rows padded with -1)
        std::vector<std::vector<int32_t>> adj(H);
        for (int i = 0; i < H; ++i)
            for (int r = 0; r < s_nn; ++r) {
                const int32_t j = nn[static_cast<size_t>(i) * s_nn + r];
                if (j < 0 || j >= H || j == i)
                    continue;
                adj[i].push_back(j);
                adj[j].push_back(i);
            }
        for (int i = 0; i < H; ++i) {
            std::vector<int32_t> &a = adj[i];
            std::sort(a.begin(), a.end());
            a.erase(std::unique(a.begin(), a.end()), a.end());
            std::vector<std::pair<double, int32_t>> by(a.size());
            for (size_t t = 0; t < a.size(); ++t) {
                double c = 0.0;
                for (int k = 0; k < 64; ++k)
                    c += static_cast<double>(En[static_cast<size_t>(i) * 64 + k]) *
                         static_cast<double>(En[static_cast<size_t>(a[t]) * 64 + k]);
                by[t] = {-c, a[t]};
            }
            std::sort(by.begin(), by.end());
            for (size_t t = 0; t < by.size() && t < static_cast<size_t>(width); ++t)
                rows[static_cast<size_t>(i) * width + t] = by[t].second;
        }
    }
    if (st == ANN_OK) {
        // entry selections still in flight (on any stream) read the old graph
        st = cuda_status(cudaDeviceSynchronize());
    }
    if (st == ANN_OK) {
        cudaFree(m->hub_graph);
        m->hub_graph = nullptr;
        m->s = width;
        st = build_hub_index(idx, m, rows.data(), m->hub_entry, s);
    }
    cudaSetDevice(prev);
    return st;
}

ann_status ann_set_hub_seeds(ann_index *idx, const int32_t *seeds, int32_t n)
{
    if (!idx || n < 0 || n > ANN_MAX_SEEDS || (n > 0 && !seeds))
        return ANN_ERR_INVALID_ARG;
    ann_entry_model *m = idx->model;
    if (!m)
        return ANN_ERR_UNSUPPORTED;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(idx->device);
    int32_t h[ANN_MAX_SEEDS];
    cudaError_t e = cudaSuccess;
    if (n > 0)
        e = cudaMemcpy(h, seeds, static_cast<size_t>(n) * 4, cudaMemcpyDefault);
    else
        h[0] = m->hub_entry;  // back to the entry hub alone
    ann_status st = cuda_status(e);
    for (int i = 0; st == ANN_OK && i < n; ++i)
        if (h[i] < 0 || h[i] >= m->H)
            st = ANN_ERR_INVALID_ARG;
    if (st == ANN_OK) {
        // entry selections still in flight (on any stream) read the old list
        e = cudaDeviceSynchronize();
        if (e == cudaSuccess)
            e = cudaMemcpy(m->hub_seeds, h, static_cast<size_t>(std::max(n, 1)) * 4, cudaMemcpyHostToDevice);
        st = cuda_status(e);
    }
    if (st == ANN_OK)
        m->n_hub_seeds = n;
    cudaSetDevice(prev);
    return st;
}

ann_status ann_select_entry(ann_index *idx, const void *d_queries, int64_t nq, int32_t mode, int32_t L_hub,
                            int32_t *d_entry, float *d_qhat, void *stream)
{
    return ann_select_entries(idx, d_queries, nq, mode, L_hub, 1, d_entry, d_qhat, stream);
}

ann_status ann_select_entries(ann_index *idx, const void *d_queries, int64_t nq, int32_t mode, int32_t L_hub,
                              int32_t m_seeds, int32_t *d_entry, float *d_qhat, void *stream)
{
    if (!idx || nq < 0 || m_seeds < 1 || m_seeds > ANN_MAX_ENTRY_HUBS ||
        (mode != ANN_ENTRY_MEDOID && mode != ANN_ENTRY_LEARNED_NAV && mode != ANN_ENTRY_LEARNED_EXHAUSTIVE))
        return ANN_ERR_INVALID_ARG;
    if (nq == 0)
        return ANN_OK;
    if (!d_entry || !d_queries || (reinterpret_cast<uintptr_t>(d_queries) & 15) ||
        (reinterpret_cast<uintptr_t>(d_qhat) & 15))
        return ANN_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(idx->device);
    ann_status st = ANN_OK;
    const int64_t nm = nq * m_seeds;
    if (mode == ANN_ENTRY_MEDOID) {
        fill_medoid_seeds<<<static_cast<unsigned>((nm + 255) / 256), 256, 0, s>>>(d_entry, nq, m_seeds,
                                                                                  idx->medoid);
        st = cuda_status(cudaGetLastError());
        cudaSetDevice(prev);
        return st;
    }
    ann_entry_model *m = idx->model;
    if (!m || (mode == ANN_ENTRY_LEARNED_NAV && (L_hub < m_seeds || L_hub > ANN_MAX_L))) {
        cudaSetDevice(prev);
        return m ? ANN_ERR_INVALID_ARG : ANN_ERR_UNSUPPORTED;
    }
    if (mode == ANN_ENTRY_LEARNED_NAV && (!m->hub_graph || !m->hub_index)) {
        cudaSetDevice(prev);
        return ANN_ERR_UNSUPPORTED;  // a failed hub-graph rebuild left no graph
    }
    const Operand X{d_queries, idx->dtype == ANN_U8 ? OP_U8 : OP_F32, idx->dim, 1, nq, idx->dim, nullptr};
    if (mode == ANN_ENTRY_LEARNED_EXHAUSTIVE) {
        // the tower, the hub scores and the top-m in one launch, q_hat kept
        // in shared memory: no scratch
        st = launch_entry_exhaustive(m, X, nq, d_qhat, d_entry, m_seeds, idx->d_status, s);
        cudaSetDevice(prev);
        return st;
    }
    // pools of up to 64 hubs run in one launch of hub_nav_kernel (with a
    // 32-bit work counter), larger ones in the general search on the hub index
    const bool one_launch = L_hub <= kNavMaxPool && m->s <= 32 && nq <= INT32_MAX;
    // scratch: q_hat fp32 + bf16, hub ids, hub scores, the work counter, and
    // for the general search with a hub sample, every query's seed set
    const size_t qf = static_cast<size_t>(nq) * 64 * 4, qb = static_cast<size_t>(nq) * 64 * 2;
    const size_t hb = static_cast<size_t>(nm) * 4;
    const size_t sb = one_launch ? 0 : static_cast<size_t>(nq) * m->n_hub_seeds * 4;
    void *scr = nullptr;
    st = scratch_alloc(idx, qf + qb + 2 * hb + 256 + sb, s, &scr);
    if (st != ANN_OK) {
        cudaSetDevice(prev);
        return st;
    }
    float *qhat = d_qhat ? d_qhat : static_cast<float *>(scr);
    __nv_bfloat16 *qbf = reinterpret_cast<__nv_bfloat16 *>(static_cast<uint8_t *>(scr) + qf);
    int32_t *hid = reinterpret_cast<int32_t *>(static_cast<uint8_t *>(scr) + qf + qb);
    float *hsc = reinterpret_cast<float *>(static_cast<uint8_t *>(scr) + qf + qb + hb);
    st = launch_tower(m, X, nq, qhat, qbf, nullptr, nullptr, nullptr, idx->d_status, s);
    if (st == ANN_OK && one_launch) {
        const int bm_words = (m->H + 127) / 128 * 4;
        const size_t per_warp = 256 + 128 + 4 * static_cast<size_t>(bm_words);
        const size_t smem = per_warp * kNavWarps;
        auto kern = L_hub <= 32 ? hub_nav_kernel<1> : hub_nav_kernel<2>;
        cudaError_t e =
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e == cudaSuccess) {
            // a persistent grid of the CTAs that fit at once
            int per_sm = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * kNavWarps, smem);
            const int64_t blocks = std::min<int64_t>((nq + kNavWarps - 1) / kNavWarps,
                                                     static_cast<int64_t>(idx->num_sms) * std::max(per_sm, 1));
            unsigned *counter = reinterpret_cast<unsigned *>(static_cast<uint8_t *>(scr) + qf + qb + 2 * hb);
            if (e == cudaSuccess)
                e = cudaMemsetAsync(counter, 0, 4, s);
            if (e == cudaSuccess) {
                kern<<<static_cast<unsigned>(blocks), 32 * kNavWarps, smem, s>>>(
                    qhat, nq, m->Eb, m->H, m->hub_graph, m->s, m->hub_seeds, std::max(m->n_hub_seeds, 1), L_hub,
                    m_seeds, m->hub_nodes, idx->medoid, bm_words, counter, d_entry);
                e = cudaGetLastError();
            }
        }
        st = cuda_status(e);
    } else if (st == ANN_OK) {
        ann_search_params p{};
        p.k = m_seeds;
        p.L = L_hub;
        p.W = 1;
        SearchLaunch Ls{};
        Ls.queries = qhat;
        Ls.qbytes = 64 * 4;
        Ls.nq = nq;
        Ls.entries = nullptr;
        if (m->n_hub_seeds > 0) {
            int32_t *seeds = reinterpret_cast<int32_t *>(static_cast<uint8_t *>(scr) + qf + qb + 2 * hb + 256);
            const int64_t ns = nq * m->n_hub_seeds;
            broadcast_hub_seeds<<<static_cast<unsigned>((ns + 255) / 256), 256, 0, s>>>(m->hub_seeds,
                                                                                       m->n_hub_seeds, ns, seeds);
            st = cuda_status(cudaGetLastError());
            Ls.entries = seeds;
            p.n_entries = m->n_hub_seeds;
        }
        Ls.p = &p;
        Ls.ids = hid;
        Ls.dists = hsc;
        Ls.stats = nullptr;
        if (st == ANN_OK)
            st = launch_search(m->hub_index, Ls, s);
        if (st == ANN_OK) {
            map_hub_seeds<<<static_cast<unsigned>((nm + 255) / 256), 256, 0, s>>>(hid, nq, m_seeds, m->hub_nodes,
                                                                                 idx->medoid, d_entry);
            st = cuda_status(cudaGetLastError());
        }
    }
    scratch_free(idx, scr, s);
    cudaSetDevice(prev);
    return st;
}

}  // extern "C"
