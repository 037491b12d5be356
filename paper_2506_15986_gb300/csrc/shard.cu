// shard.cu -- the exchange-side kernels of base-partitioned search: the base
// set is split into shards (groups of whole hub clusters, Sec. 4.1 Def. 3),
// each shard has its own graph and is searched on its own, and a query's
// answer is the k best of the shards' answers under the (distance, id) order
// of Sec. 2.1, Problem 1.
//   - map_ids_kernel: shard-local row ids -> global ids through the shard's
//     row map (-1 stays -1);
//   - merge_kernel: per query, the k smallest (distance, id) keys of P sorted
//     lists of k; one warp per query, lane p < P holds the head of list p and
//     the warp takes the minimum head k times.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "device_util.cuh"
#include "internal.h"

namespace ann {
namespace {

constexpr int kMergeWarps = 8;

__global__ void map_ids_kernel(int32_t *ids, int64_t count, const int32_t *map, int64_t n_map, int *status)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < count;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int32_t v = ids[i];
        if (v < 0)
            continue;
        if (v >= n_map) {
            ids[i] = -1;  // not a row of this shard
            if (status)
                atomicOr(status, 1);
            continue;
        }
        ids[i] = map[v];
    }
}

// (distance, id) key of one list entry: order-preserving distance bits
// above the id; an empty entry (id -1) is the largest key
template <bool INT_DIST>
__device__ __forceinline__ uint64_t entry_key(const int32_t *ids, const void *dists, int64_t at)
{
    const int32_t id = ids[at];
    if (id < 0)
        return kKeyMax;
    const uint32_t db = INT_DIST ? static_cast<uint32_t>(static_cast<const int32_t *>(dists)[at])
                                 : f32_to_ord(static_cast<const float *>(dists)[at]);
    return (static_cast<uint64_t>(db) << 32) | static_cast<uint32_t>(id);
}

template <bool INT_DIST>
__global__ void __launch_bounds__(32 * kMergeWarps)
    merge_kernel(const int32_t *ids, const void *dists, int P, int64_t nq, int k, int32_t *out_ids,
                 void *out_dists)
{
    const int lane = threadIdx.x & 31;
    const int64_t q = blockIdx.x * static_cast<int64_t>(kMergeWarps) + (threadIdx.x >> 5);
    if (q >= nq)
        return;
    // lane p walks list p: its next entry is at position pos
    int pos = 0;
    auto at = [&](int p, int j) { return (static_cast<int64_t>(p) * nq + q) * k + j; };
    uint64_t head = lane < P ? entry_key<INT_DIST>(ids, dists, at(lane, 0)) : kKeyMax;
    for (int j = 0; j < k; ++j) {
        uint64_t m = head;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const uint64_t w = __shfl_xor_sync(kFull, m, o);
            m = w < m ? w : m;
        }
        if (lane == 0) {
            const bool ok = m != kKeyMax;
            out_ids[q * k + j] = ok ? static_cast<int32_t>(static_cast<uint32_t>(m)) : -1;
            const uint32_t db = static_cast<uint32_t>(m >> 32);
            if (INT_DIST)
                static_cast<int32_t *>(out_dists)[q * k + j] = ok ? static_cast<int32_t>(db) : INT32_MAX;
            else
                static_cast<float *>(out_dists)[q * k + j] = ok ? ord_to_f32(db) : __int_as_float(0x7f800000);
        }
        // the list whose head was taken advances (keys are distinct: ids are
        // distinct across shards, and an empty list never wins)
        if (lane < P && head == m && m != kKeyMax) {
            ++pos;
            head = pos < k ? entry_key<INT_DIST>(ids, dists, at(lane, pos)) : kKeyMax;
        }
    }
}

}  // namespace
}  // namespace ann

using namespace ann;

extern "C" {

ann_status ann_map_ids(int32_t *d_ids, int64_t count, const int32_t *d_map, int64_t n_map, int32_t *d_status,
                       void *stream)
{
    if (count < 0 || n_map < 0 || (count > 0 && (!d_ids || !d_map)))
        return ANN_ERR_INVALID_ARG;
    if (count == 0)
        return ANN_OK;
    const int64_t blocks = std::min<int64_t>((count + 255) / 256, 4096);
    map_ids_kernel<<<static_cast<unsigned>(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        d_ids, count, d_map, n_map, d_status);
    return cuda_status(cudaGetLastError());
}

ann_status ann_merge_shards(const int32_t *d_ids, const void *d_dists, int32_t P, int64_t nq, int32_t k,
                            int32_t int_dists, int32_t *d_out_ids, void *d_out_dists, void *stream)
{
    if (P < 1 || P > 32 || nq < 0 || k < 1 || (nq > 0 && (!d_ids || !d_dists || !d_out_ids || !d_out_dists)))
        return ANN_ERR_INVALID_ARG;
    if (nq == 0)
        return ANN_OK;
    const unsigned blocks = static_cast<unsigned>((nq + kMergeWarps - 1) / kMergeWarps);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (int_dists)
        merge_kernel<true><<<blocks, 32 * kMergeWarps, 0, s>>>(d_ids, d_dists, P, nq, k, d_out_ids, d_out_dists);
    else
        merge_kernel<false><<<blocks, 32 * kMergeWarps, 0, s>>>(d_ids, d_dists, P, nq, k, d_out_ids, d_out_dists);
    return cuda_status(cudaGetLastError());
}

}  // extern "C"
