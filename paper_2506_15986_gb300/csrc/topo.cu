// topo.cu -- per-hop topology tokens of hub nodes from the guided subgraph
// walk of Sec. 4.2 (the Graph2Vec-free structural feature of the
// topology-aware hub tower).
//
// The walk: MinDeg / MaxDeg are the smallest / largest numbers of valid
// neighbours over the graph.  A FIFO queue starts with the hub at hop 0.  A
// dequeued node u at hop < h ranks its deg(u) valid neighbours by (squared L2
// to u, id) and samples the ceil(x/2) nearest and the floor(x/2) farthest,
// x = ceil(MinDeg * deg(u) / MaxDeg); every sampled neighbour not yet in the
// subgraph joins it in rank order at hop(u) + 1 with parent u.  Hop-h nodes
// join but are not expanded; the subgraph stops at max_nodes nodes.
//
// Token l (0..h) summarises the hop-l nodes, s being the hub's mean squared
// distance to its valid neighbours (1 if none or 0): count / total, mean
// degree / MaxDeg, mean and max squared distance to the hub / s, mean squared
// distance to the parent / s, share sampled as farthest, l / h, 1.  Every
// float operation is rounded on its own and summed in a fixed order
// (coordinates 0..dim-1; a hop's nodes in joining order), so the ranking,
// an integer decision, and the tokens reproduce bit for bit.
//
// One warp per hub: lane r holds neighbour slot r (two slots per lane when
// the degree passes 32); the subgraph list lives in the CTA's shared memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace ann {
namespace {

constexpr int kTokenDim = 8;
constexpr int kMaxSlots = 2;  // neighbour slots per lane: degree <= 64

__device__ __forceinline__ float tdist(const float *x, int dim, int64_t a, int64_t b)
{
    const float *p = x + a * dim, *q = x + b * dim;
    float acc = 0.f;
    for (int t = 0; t < dim; t += 4) {
        const float4 u = *reinterpret_cast<const float4 *>(p + t);
        const float4 v = *reinterpret_cast<const float4 *>(q + t);
        float d = __fsub_rn(u.x, v.x);
        acc = __fadd_rn(acc, __fmul_rn(d, d));
        d = __fsub_rn(u.y, v.y);
        acc = __fadd_rn(acc, __fmul_rn(d, d));
        d = __fsub_rn(u.z, v.z);
        acc = __fadd_rn(acc, __fmul_rn(d, d));
        d = __fsub_rn(u.w, v.w);
        acc = __fadd_rn(acc, __fmul_rn(d, d));
    }
    return acc;
}

__device__ __forceinline__ uint64_t rank_key(float d, int32_t id)
{
    const uint32_t u = __float_as_uint(d);
    const uint32_t o = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return (static_cast<uint64_t>(o) << 32) | static_cast<uint32_t>(id);
}

__global__ void degree_range(const int32_t *graph, int64_t n, int R, int *mm)
{
    int lo = R, hi = 0;
    for (int64_t u = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; u < n;
         u += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        int dg = 0;
        for (int r = 0; r < R; ++r)
            dg += graph[u * R + r] >= 0;
        lo = min(lo, dg);
        hi = max(hi, dg);
    }
    atomicMin(mm, lo);
    atomicMax(mm + 1, hi);
}

__global__ void __launch_bounds__(32) topo_kernel(const float *x, int dim, int64_t n, const int32_t *graph, int R,
                                                  const int32_t *hubs, int H, int h, int max_nodes, const int *mm,
                                                  float *tokens, int32_t *nodes_out)
{
    extern __shared__ __align__(16) uint8_t smem[];
    int32_t *node = reinterpret_cast<int32_t *>(smem);
    int32_t *par = node + max_nodes;
    int32_t *hop = par + max_nodes;
    uint8_t *far = reinterpret_cast<uint8_t *>(hop + max_nodes);
    const int lane = threadIdx.x;
    const int mindeg = mm[0], maxdeg = mm[1];
    for (int v = blockIdx.x; v < H; v += gridDim.x) {
        const int32_t hub = hubs[v];
        float *tok = tokens + static_cast<int64_t>(v) * (h + 1) * kTokenDim;
        if (lane == 0) {
            node[0] = hub;
            par[0] = -1;
            hop[0] = 0;
            far[0] = 0;
        }
        __syncwarp();
        int cnt = 1, head = 0;
        while (head < cnt) {
            const int32_t u = node[head];
            const int hu = hop[head];
            ++head;
            if (hu >= h)
                continue;
            // rank the valid neighbours by (distance, id)
            uint64_t key[kMaxSlots];
            int32_t nbr[kMaxSlots];
            int dg = 0;
#pragma unroll
            for (int k = 0; k < kMaxSlots; ++k) {
                const int r = lane + 32 * k;
                nbr[k] = r < R ? graph[static_cast<int64_t>(u) * R + r] : -1;
                key[k] = nbr[k] >= 0 ? rank_key(tdist(x, dim, u, nbr[k]), nbr[k]) : ~0ull;
                dg += __popc(__ballot_sync(0xffffffffu, nbr[k] >= 0));
            }
            int rk[kMaxSlots] = {0, 0};
#pragma unroll
            for (int k2 = 0; k2 < kMaxSlots; ++k2)
                for (int src = 0; src < 32; ++src) {
                    const uint64_t o = __shfl_sync(0xffffffffu, key[k2], src);
#pragma unroll
                    for (int k = 0; k < kMaxSlots; ++k)
                        rk[k] += o < key[k];
                }
            const int xs = maxdeg > 0 ? (mindeg * dg + maxdeg - 1) / maxdeg : 0;
            const int near_n = (xs + 1) / 2, far_n = xs / 2;
            // sampled ranks in increasing order: [0, near_n) then [dg - far_n, dg)
            for (int a = 0; a < dg && cnt < max_nodes; ++a) {
                const bool is_far = a >= dg - far_n;
                if (a >= near_n && !is_far)
                    continue;
                int32_t w = -1;
#pragma unroll
                for (int k = 0; k < kMaxSlots; ++k) {
                    const unsigned bm = __ballot_sync(0xffffffffu, nbr[k] >= 0 && rk[k] == a);
                    if (bm)
                        w = __shfl_sync(0xffffffffu, nbr[k], __ffs(bm) - 1);
                }
                bool seen = false;
                for (int q = lane; q < cnt; q += 32)
                    seen |= node[q] == w;
                if (__any_sync(0xffffffffu, seen))
                    continue;
                if (lane == 0) {
                    node[cnt] = w;
                    par[cnt] = u;
                    hop[cnt] = hu + 1;
                    far[cnt] = is_far ? 1 : 0;
                }
                ++cnt;
                __syncwarp();
            }
        }
        if (lane == 0 && nodes_out)
            nodes_out[v] = cnt;
        // scale: the hub's mean squared distance to its valid neighbours, slots in order
        float ssum = 0.f;
        int sdeg = 0;
        for (int r = 0; r < R; ++r) {
            const int32_t w = graph[static_cast<int64_t>(hub) * R + r];
            if (w >= 0) {
                ssum = __fadd_rn(ssum, tdist(x, dim, hub, w));
                ++sdeg;
            }
        }
        float s = sdeg > 0 ? __fdiv_rn(ssum, static_cast<float>(sdeg)) : 1.f;
        if (!(s > 0.f))
            s = 1.f;
        // token l: lane l walks the subgraph list in joining order
        for (int l = lane; l <= h; l += 32) {
            float *t = tok + l * kTokenDim;
            int c = 0, fars = 0;
            int64_t degsum = 0;
            float dh = 0.f, dmax = 0.f, dpar = 0.f;
            for (int q = 0; q < cnt; ++q) {
                if (hop[q] != l)
                    continue;
                const float a = __fdiv_rn(tdist(x, dim, node[q], hub), s);
                const float b = par[q] >= 0 ? __fdiv_rn(tdist(x, dim, node[q], par[q]), s) : 0.f;
                int dgq = 0;
                for (int r = 0; r < R; ++r)
                    dgq += graph[static_cast<int64_t>(node[q]) * R + r] >= 0;
                ++c;
                degsum += dgq;
                fars += far[q];
                dh = __fadd_rn(dh, a);
                dmax = a > dmax ? a : dmax;
                dpar = __fadd_rn(dpar, b);
            }
            float f[kTokenDim] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (c > 0) {
                f[0] = __fdiv_rn(static_cast<float>(c), static_cast<float>(cnt));
                f[1] = maxdeg > 0 ? __fdiv_rn(static_cast<float>(degsum),
                                              __fmul_rn(static_cast<float>(c), static_cast<float>(maxdeg)))
                                  : 0.f;
                f[2] = __fdiv_rn(dh, static_cast<float>(c));
                f[3] = dmax;
                f[4] = __fdiv_rn(dpar, static_cast<float>(c));
                f[5] = __fdiv_rn(static_cast<float>(fars), static_cast<float>(c));
            }
            f[6] = __fdiv_rn(static_cast<float>(l), static_cast<float>(h));
            f[7] = 1.f;
#pragma unroll
            for (int j = 0; j < kTokenDim; ++j)
                t[j] = f[j];
        }
        __syncwarp();
    }
}

}  // namespace
}  // namespace ann

using namespace ann;

extern "C" {

ann_status ann_topo_tokens(ann_index *idx, const int32_t *d_hubs, int32_t H, int32_t h, int32_t max_nodes,
                           float *d_tokens, int32_t *d_nodes, void *stream)
{
    if (!idx || !d_hubs || !d_tokens || H < 1 || h < 1 || h > 64 || max_nodes < 1 || max_nodes > 8192)
        return ANN_ERR_INVALID_ARG;
    const float *x = idx->dtype == ANN_F32 ? static_cast<const float *>(idx->d_base) : idx->d_base_f32;
    if (!x || idx->degree > 32 * kMaxSlots || idx->dim % 4 != 0)
        return ANN_ERR_UNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(idx->device);
    // hub ids are checked on the host before any launch reads them
    std::vector<int32_t> hh(H);
    cudaError_t e = cudaMemcpyAsync(hh.data(), d_hubs, static_cast<size_t>(H) * 4, cudaMemcpyDefault, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaSetDevice(prev);
        return cuda_status(e);
    }
    for (int32_t v : hh)
        if (v < 0 || v >= idx->n) {
            cudaSetDevice(prev);
            return ANN_ERR_INVALID_ARG;
        }
    int *mm = nullptr;
    e = cudaMallocAsync(reinterpret_cast<void **>(&mm), 8, s);
    const int init[2] = {idx->degree, 0};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(mm, init, 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        degree_range<<<static_cast<unsigned>(std::min<int64_t>((idx->n + 255) / 256, 4096)), 256, 0, s>>>(
            idx->d_graph, idx->n, idx->degree, mm);
        const size_t smem = static_cast<size_t>(max_nodes) * 13;
        e = cudaFuncSetAttribute(topo_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e == cudaSuccess)
            topo_kernel<<<static_cast<unsigned>(std::min(H, 152 * 16)), 32, smem, s>>>(
                x, idx->dim, idx->n, idx->d_graph, idx->degree, d_hubs, H, h, max_nodes, mm, d_tokens, d_nodes);
        if (e == cudaSuccess)
            e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(s);
        // the init values above live on this stack frame: the copy has completed here
        cudaFreeAsync(mm, s);
    }
    cudaSetDevice(prev);
    return cuda_status(e);
}

}  // extern "C"
