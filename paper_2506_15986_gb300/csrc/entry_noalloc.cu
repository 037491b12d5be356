// entry_noalloc.cu -- exhaustive learned entry selection without any device
// allocation.
//
// Some callers cannot let a library allocate device memory on their behalf:
// a serving loop that has reserved all of HBM up front for the index and its
// own buffers; latency-critical code where a cudaMalloc could synchronise the
// device or stall on the allocator; host callbacks and other contexts where
// CUDA calls that allocate are not allowed.  For them this file keeps the
// scratch of the exhaustive entry selection (BF16 query embeddings, best hub
// index and score per query) in a statically sized device array instead of
// the index's stream-ordered pool.
//
// The array is a file-scope __device__ symbol, so every GPU that loads the
// library holds it until the process exits.  Host code cannot use the symbol's
// name as a device address; the address is looked up once per device with
// cudaGetSymbolAddress, with that device current, the first time the entry
// point runs on it.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "entry.h"
#include "internal.h"

namespace ann {
namespace {

// 16 MiB per device: 64 BF16 embedding values, a hub index and a score per
// query, i.e. 136 bytes; with room left for aligning the three regions to
// 256 bytes, at most 123,357 queries per call.
constexpr size_t kNoAllocScratchBytes = static_cast<size_t>(16) << 20;
constexpr size_t kNoAllocBytesPerQuery = 64 * 2 + 4 + 4;
constexpr int64_t kNoAllocMaxQueries = static_cast<int64_t>(kNoAllocScratchBytes / kNoAllocBytesPerQuery) - 4;

__device__ __align__(256) uint8_t g_entry_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_entry_scratch on the current device `dev`.
ann_status scratch_address(int dev, void **out)
{
    if (dev < 0 || dev >= kMaxDevices)
        return ANN_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_entry_scratch);
        if (e != cudaSuccess)
            return cuda_status(e);
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return ANN_OK;
}

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace
}  // namespace ann

using namespace ann;

extern "C" {

int64_t ann_select_entry_noalloc_max_queries(void) { return kNoAllocMaxQueries; }

ann_status ann_select_entry_noalloc(ann_index *idx, const void *d_queries, int64_t nq, int32_t *d_entry,
                                    float *d_qhat, void *stream)
{
    if (!idx || nq < 0)
        return ANN_ERR_INVALID_ARG;
    if (nq > kNoAllocMaxQueries)
        return ANN_ERR_CAPACITY;  // the batch needs more than the static scratch holds
    if (!idx->model)
        return ANN_ERR_UNSUPPORTED;
    if (nq == 0)
        return ANN_OK;
    if (!d_entry || !d_queries || (reinterpret_cast<uintptr_t>(d_queries) & 15) ||
        (reinterpret_cast<uintptr_t>(d_qhat) & 15))
        return ANN_ERR_INVALID_ARG;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess)
        return ANN_ERR_CUDA;
    if (cudaSetDevice(idx->device) != cudaSuccess)
        return ANN_ERR_CUDA;
    void *scratch = nullptr;
    ann_status st = scratch_address(idx->device, &scratch);
    if (st == ANN_OK) {
        // layout: q_hat BF16 [nq][64] | hub index [nq] | hub score [nq]; every
        // word is written before it is read, so nothing needs clearing
        uint8_t *base = static_cast<uint8_t *>(scratch);
        __nv_bfloat16 *qbf = reinterpret_cast<__nv_bfloat16 *>(base);
        int32_t *hub = reinterpret_cast<int32_t *>(base + up256(static_cast<size_t>(nq) * 128));
        float *score = reinterpret_cast<float *>(base + up256(static_cast<size_t>(nq) * 128) +
                                                 up256(static_cast<size_t>(nq) * 4));
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        const ann_entry_model *m = idx->model;
        const Operand X{d_queries, idx->dtype == ANN_U8 ? OP_U8 : OP_F32, idx->dim, 1, nq, idx->dim, nullptr};
        st = launch_tower(m, X, nq, d_qhat, qbf, nullptr, nullptr, nullptr, idx->d_status, s);
        if (st == ANN_OK) {
            const Operand Q{qbf, OP_BF16, 64, 1, nq, 64, nullptr};
            st = launch_hub_argmax(m, Q, nq, d_entry, hub, score, idx->d_status, s);
        }
    }
    cudaSetDevice(prev);
    return st;
}

}  // extern "C"
