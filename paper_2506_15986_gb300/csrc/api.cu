// api.cu -- the C ABI of libann: index lifetime, file format, search entry
// point and device status.  Every argument is checked on the host before any
// kernel is queued.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "entry.h"
#include "internal.h"

namespace ann {

int elem_size(int dtype)
{
    switch (dtype) {
    case ANN_U8: return 1;
    case ANN_F32: return 4;
    case ANN_F16: return 2;
    case ANN_BF16: return 2;
    case ANN_I8S: return 1;
    default: return 0;
    }
}

int64_t row_bytes(int dtype, int dim)
{
    if (dim < 1)
        return 0;
    if (dtype == ANN_I8S)
        return 16 + (static_cast<int64_t>(dim) + 15) / 16 * 16;
    return static_cast<int64_t>(dim) * elem_size(dtype);
}

ann_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess)
        return ANN_OK;
    if (e == cudaErrorMemoryAllocation)
        return ANN_ERR_OOM;
    return ANN_ERR_CUDA;
}

ann_status scratch_alloc(ann_index *idx, size_t bytes, cudaStream_t s, void **out)
{
    *out = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(out, bytes, idx->pool, s);
    return cuda_status(e);
}

void scratch_free(ann_index *idx, void *p, cudaStream_t s)
{
    (void)idx;
    if (p)
        cudaFreeAsync(p, s);
}

namespace {

__global__ void count_bad_ids(const int32_t *g, int64_t total, int64_t n, unsigned long long *bad)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        int32_t v = g[i];
        if (v < -1 || v >= n)
            atomicAdd(bad, 1ull);
    }
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess)
            prev = -1;
        cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0)
            cudaSetDevice(prev);
    }
};

void destroy(ann_index *idx)
{
    if (!idx)
        return;
    cudaDeviceSynchronize();
    cudaFree(idx->d_base);
    cudaFree(idx->d_graph);
    cudaFree(idx->d_base_f32);
    cudaFree(idx->d_status);
    free_model(idx->model);
    if (idx->pool)
        cudaMemPoolDestroy(idx->pool);
    delete idx;
}

// 64-bit FNV-1a
uint64_t fnv1a(uint64_t h, const void *data, size_t len)
{
    const uint8_t *p = static_cast<const uint8_t *>(data);
    for (size_t i = 0; i < len; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

constexpr uint64_t kFnvInit = 14695981039346656037ull;
constexpr char kMagic[8] = {'G', 'A', 'T', 'E', 'A', 'N', 'N', '1'};
constexpr uint32_t kVersion = 1;

struct FileHeader {
    char magic[8];
    uint32_t version;
    uint32_t header_bytes;
    int64_t n;
    int32_t dim, degree, dtype, metric, medoid;
    uint32_t flags;  // bit 0: fp32 copy present
    uint64_t bytes_base, bytes_graph, bytes_f32;
    uint64_t checksum;  // FNV-1a over the sections, in file order
};

}  // namespace
}  // namespace ann

namespace ann {
namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Tensor map over the base rows for four-row TMA gathers: a 2-D tensor of
// rowbytes / 4 four-byte elements by n rows, one-row boxes spanning a whole
// row (at most 256 elements, so rows up to 1 KiB; a multiple of 32 bytes so
// that four rows fill whole 128-byte lines of the staging area).  Leaves
// has_row_map at 0 when the row size does not qualify or the driver lacks
// the encoder, and the search then copies row by row.
void make_row_map(ann_index *idx)
{
    idx->has_row_map = 0;
    if (idx->rowbytes % 32 != 0 || idx->rowbytes > 1024)
        return;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return;
    const cuuint64_t dims[2] = {static_cast<cuuint64_t>(idx->rowbytes / 4), static_cast<cuuint64_t>(idx->n)};
    const cuuint64_t strides[1] = {static_cast<cuuint64_t>(idx->rowbytes)};
    const cuuint32_t box[2] = {static_cast<cuuint32_t>(idx->rowbytes / 4), 1};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = reinterpret_cast<EncodeTiledFn>(fn)(
        &idx->row_map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, idx->d_base, dims, strides, box, estr,
        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    idx->has_row_map = r == CUDA_SUCCESS ? 1 : 0;
}

}  // namespace
}  // namespace ann

using namespace ann;

extern "C" {

const char *ann_status_string(ann_status s)
{
    switch (s) {
    case ANN_OK: return "ok";
    case ANN_ERR_INVALID_ARG: return "invalid argument";
    case ANN_ERR_IO: return "i/o error";
    case ANN_ERR_FORMAT: return "bad index file format";
    case ANN_ERR_OOM: return "out of device memory";
    case ANN_ERR_CUDA: return "cuda error";
    case ANN_ERR_CAPACITY: return "visited-set capacity exceeded";
    case ANN_ERR_TIMEOUT: return "bounded device wait timed out";
    case ANN_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
    }
}


ann_status ann_index_create(const ann_index_desc *desc, int device, ann_index **out)
{
    if (!desc || !out)
        return ANN_ERR_INVALID_ARG;
    const int64_t rowbytes = row_bytes(desc->dtype, desc->dim);
    if (desc->n < 1 || desc->n > INT32_MAX || desc->dim < 1 || desc->degree < 1 ||
        desc->degree > ANN_MAX_STEP_CAND || rowbytes == 0 || (desc->metric != ANN_L2 && desc->metric != ANN_IP) ||
        !desc->base || !desc->graph || desc->medoid < 0 || desc->medoid >= desc->n)
        return ANN_ERR_INVALID_ARG;
    if (desc->dtype == ANN_U8 && desc->metric != ANN_L2)
        return ANN_ERR_UNSUPPORTED;
    if (rowbytes % 16 != 0 || rowbytes > 16384 || (desc->dtype == ANN_I8S && desc->dim % 4 != 0))
        return ANN_ERR_INVALID_ARG;
    if (desc->base_f32 && desc->dtype == ANN_U8)
        return ANN_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return ANN_ERR_CUDA;
    DeviceGuard guard(device);

    ann_index *idx = new (std::nothrow) ann_index();
    if (!idx)
        return ANN_ERR_OOM;
    idx->device = device;
    idx->n = desc->n;
    idx->dim = desc->dim;
    idx->degree = desc->degree;
    idx->dtype = desc->dtype;
    idx->metric = desc->metric;
    idx->medoid = desc->medoid;
    idx->rowbytes = static_cast<int32_t>(rowbytes);
    cudaDeviceGetAttribute(&idx->num_sms, cudaDevAttrMultiProcessorCount, device);

    const size_t bbytes = static_cast<size_t>(desc->n) * rowbytes;
    const size_t gbytes = static_cast<size_t>(desc->n) * desc->degree * sizeof(int32_t);
    cudaError_t e = cudaMalloc(&idx->d_base, bbytes);
    if (e == cudaSuccess)
        e = cudaMalloc(reinterpret_cast<void **>(&idx->d_graph), gbytes);
    if (e == cudaSuccess)
        e = cudaMalloc(reinterpret_cast<void **>(&idx->d_status), 256);
    if (e == cudaSuccess && desc->base_f32)
        e = cudaMalloc(reinterpret_cast<void **>(&idx->d_base_f32),
                       static_cast<size_t>(desc->n) * desc->dim * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMemcpy(idx->d_base, desc->base, bbytes, cudaMemcpyDefault);
    if (e == cudaSuccess)
        e = cudaMemcpy(idx->d_graph, desc->graph, gbytes, cudaMemcpyDefault);
    if (e == cudaSuccess && desc->base_f32)
        e = cudaMemcpy(idx->d_base_f32, desc->base_f32,
                       static_cast<size_t>(desc->n) * desc->dim * sizeof(float), cudaMemcpyDefault);
    if (e == cudaSuccess)
        e = cudaMemset(idx->d_status, 0, 256);
    if (e == cudaSuccess) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        e = cudaMemPoolCreate(&idx->pool, &props);
        if (e == cudaSuccess) {
            uint64_t keep = UINT64_MAX;  // keep freed scratch for the next call
            e = cudaMemPoolSetAttribute(idx->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    if (e == cudaSuccess) {
        // every adjacency entry must be a node id or a negative pad
        unsigned long long *d_bad = reinterpret_cast<unsigned long long *>(idx->d_status) + 8;
        const int64_t total = desc->n * static_cast<int64_t>(desc->degree);
        count_bad_ids<<<1024, 256>>>(idx->d_graph, total, desc->n, d_bad);
        unsigned long long bad = 0;
        e = cudaMemcpy(&bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            e = cudaMemset(idx->d_status, 0, 256);
        if (e == cudaSuccess && bad != 0) {
            destroy(idx);
            return ANN_ERR_INVALID_ARG;
        }
    }
    if (e != cudaSuccess) {
        ann_status st = cuda_status(e);
        destroy(idx);
        return st;
    }
    make_row_map(idx);
    *out = idx;
    return ANN_OK;
}

ann_status ann_free_index(ann_index *idx)
{
    if (!idx)
        return ANN_OK;
    DeviceGuard guard(idx->device);
    destroy(idx);
    return ANN_OK;
}

ann_status ann_index_info(const ann_index *idx, int64_t *n, int32_t *dim, int32_t *degree,
                          int32_t *dtype, int32_t *metric, int32_t *medoid, int32_t *n_hubs,
                          int32_t *has_model)
{
    if (!idx)
        return ANN_ERR_INVALID_ARG;
    if (n)
        *n = idx->n;
    if (dim)
        *dim = idx->dim;
    if (degree)
        *degree = idx->degree;
    if (dtype)
        *dtype = idx->dtype;
    if (metric)
        *metric = idx->metric;
    if (medoid)
        *medoid = idx->medoid;
    if (n_hubs)
        *n_hubs = idx->model ? idx->model->H : 0;
    if (has_model)
        *has_model = idx->model ? 1 : 0;
    return ANN_OK;
}

ann_status ann_save_index(const ann_index *idx, const char *path)
{
    if (!idx || !path)
        return ANN_ERR_INVALID_ARG;
    DeviceGuard guard(idx->device);
    FileHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, kMagic, 8);
    h.version = kVersion;
    h.header_bytes = sizeof(FileHeader);
    h.n = idx->n;
    h.dim = idx->dim;
    h.degree = idx->degree;
    h.dtype = idx->dtype;
    h.metric = idx->metric;
    h.medoid = idx->medoid;
    h.flags = idx->d_base_f32 ? 1u : 0u;
    h.bytes_base = static_cast<uint64_t>(idx->n) * idx->rowbytes;
    h.bytes_graph = static_cast<uint64_t>(idx->n) * idx->degree * 4;
    h.bytes_f32 = idx->d_base_f32 ? static_cast<uint64_t>(idx->n) * idx->dim * 4 : 0;
    std::vector<uint8_t> base, graph, f32;
    try {
        base.resize(h.bytes_base);
        graph.resize(h.bytes_graph);
        f32.resize(h.bytes_f32);
    } catch (...) {
        return ANN_ERR_OOM;
    }
    cudaError_t e = cudaMemcpy(base.data(), idx->d_base, h.bytes_base, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemcpy(graph.data(), idx->d_graph, h.bytes_graph, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h.bytes_f32)
        e = cudaMemcpy(f32.data(), idx->d_base_f32, h.bytes_f32, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_status(e);
    uint64_t c = fnv1a(kFnvInit, base.data(), base.size());
    c = fnv1a(c, graph.data(), graph.size());
    c = fnv1a(c, f32.data(), f32.size());
    h.checksum = c;
    FILE *f = fopen(path, "wb");
    if (!f)
        return ANN_ERR_IO;
    bool ok = fwrite(&h, sizeof(h), 1, f) == 1 && fwrite(base.data(), 1, base.size(), f) == base.size() &&
              fwrite(graph.data(), 1, graph.size(), f) == graph.size() &&
              fwrite(f32.data(), 1, f32.size(), f) == f32.size();
    ok = (fclose(f) == 0) && ok;
    return ok ? ANN_OK : ANN_ERR_IO;
}

ann_status ann_load_index(const char *path, int device, ann_index **out)
{
    if (!path || !out)
        return ANN_ERR_INVALID_ARG;
    FILE *f = fopen(path, "rb");
    if (!f)
        return ANN_ERR_IO;
    FileHeader h;
    if (fread(&h, sizeof(h), 1, f) != 1) {
        fclose(f);
        return ANN_ERR_FORMAT;
    }
    // the limits ann_index_create enforces are checked here too, before the
    // header's sizes drive any host allocation
    const int64_t rb = row_bytes(h.dtype, h.dim);
    bool sane = memcmp(h.magic, kMagic, 8) == 0 && h.version == kVersion &&
                h.header_bytes == sizeof(FileHeader) && h.n >= 1 && h.n <= INT32_MAX && h.dim >= 1 &&
                h.degree >= 1 && h.degree <= ANN_MAX_STEP_CAND && rb > 0 && rb % 16 == 0 && rb <= 16384 &&
                h.bytes_base == static_cast<uint64_t>(h.n) * rb &&
                h.bytes_graph == static_cast<uint64_t>(h.n) * h.degree * 4 &&
                h.bytes_f32 == ((h.flags & 1u) ? static_cast<uint64_t>(h.n) * h.dim * 4 : 0);
    if (!sane) {
        fclose(f);
        return ANN_ERR_FORMAT;
    }
    std::vector<uint8_t> base, graph, f32;
    try {
        base.resize(h.bytes_base);
        graph.resize(h.bytes_graph);
        f32.resize(h.bytes_f32);
    } catch (...) {
        fclose(f);
        return ANN_ERR_OOM;
    }
    bool ok = fread(base.data(), 1, base.size(), f) == base.size() &&
              fread(graph.data(), 1, graph.size(), f) == graph.size() &&
              fread(f32.data(), 1, f32.size(), f) == f32.size();
    fclose(f);
    if (!ok)
        return ANN_ERR_FORMAT;  // truncated
    uint64_t c = fnv1a(kFnvInit, base.data(), base.size());
    c = fnv1a(c, graph.data(), graph.size());
    c = fnv1a(c, f32.data(), f32.size());
    if (c != h.checksum)
        return ANN_ERR_FORMAT;
    ann_index_desc d;
    memset(&d, 0, sizeof(d));
    d.n = h.n;
    d.dim = h.dim;
    d.degree = h.degree;
    d.dtype = h.dtype;
    d.metric = h.metric;
    d.base = base.data();
    d.graph = reinterpret_cast<const int32_t *>(graph.data());
    d.medoid = h.medoid;
    d.base_f32 = h.bytes_f32 ? reinterpret_cast<const float *>(f32.data()) : nullptr;
    return ann_index_create(&d, device, out);
}

ann_status ann_search_batch(ann_index *idx, const void *d_queries, int64_t nq, const int32_t *d_entry,
                            const ann_search_params *p, int32_t *d_ids, void *d_dists, int32_t *d_stats,
                            void *stream)
{
    if (!idx || !p || nq < 0)
        return ANN_ERR_INVALID_ARG;
    if (p->L < 1 || p->L > ANN_MAX_L || p->k < 1 || p->k > p->L || p->W < 1 || p->W > ANN_MAX_W ||
        p->W * idx->degree > ANN_MAX_STEP_CAND ||
        (p->hash_bits != 0 && p->hash_bits != -1 && (p->hash_bits < 8 || p->hash_bits > 15)) ||
        p->stage_rows < 0 ||
        p->stage_rows > 32 || p->team < 0 || p->team > 32 || (p->team & (p->team - 1)) != 0 ||
        (p->spill_bits != 0 && (p->spill_bits < 10 || p->spill_bits > 16)) ||
        (p->gather != 0 && p->gather != 1 && p->gather != 4) || p->n_entries < 0 ||
        p->n_entries > ANN_MAX_SEEDS || (p->n_entries > 1 && !d_entry))
        return ANN_ERR_INVALID_ARG;
    if (p->flags & ~(ANN_SEARCH_RERANK | ANN_SEARCH_FAULT_WAIT | ANN_SEARCH_VISITED_L2 | ANN_SEARCH_GROUP_ENTRIES))
        return ANN_ERR_INVALID_ARG;
    if ((p->flags & ANN_SEARCH_RERANK) && !idx->d_base_f32)
        return ANN_ERR_UNSUPPORTED;  // the exact rerank needs the fp32 copy of the rows
    if (nq == 0)
        return ANN_OK;
    if (!d_queries || !d_ids || !d_dists)
        return ANN_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(d_queries) & 15) || (reinterpret_cast<uintptr_t>(d_ids) & 3) ||
        (reinterpret_cast<uintptr_t>(d_dists) & 3) || (reinterpret_cast<uintptr_t>(d_stats) & 3))
        return ANN_ERR_INVALID_ARG;
    DeviceGuard guard(idx->device);
    SearchLaunch L{};
    L.queries = d_queries;
    L.qbytes = idx->dtype == ANN_U8 ? idx->dim : idx->dim * 4;
    L.nq = nq;
    L.entries = d_entry;
    L.n_entries = p->n_entries;
    L.p = p;
    L.ids = d_ids;
    L.dists = d_dists;
    L.stats = d_stats;
    return launch_search(idx, L, static_cast<cudaStream_t>(stream));
}

ann_status ann_release_l2(ann_index *idx)
{
    if (!idx)
        return ANN_ERR_INVALID_ARG;
    DeviceGuard guard(idx->device);
    // the lines back to normal, and the set-aside back to zero: while it is
    // above zero, accesses without a persisting window use only the rest of L2
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
        e = cudaCtxResetPersistingL2Cache();
    if (e == cudaSuccess)
        e = cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, 0);
    return e == cudaSuccess ? ANN_OK : ANN_ERR_CUDA;
}

ann_status ann_sync_status(ann_index *idx, void *stream)
{
    if (!idx)
        return ANN_ERR_INVALID_ARG;
    DeviceGuard guard(idx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int word = 0;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess)
        e = cudaMemcpy(&word, idx->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemset(idx->d_status, 0, sizeof(int));
    if (e != cudaSuccess)
        return ANN_ERR_CUDA;
    if (word & kStatusBadInputBit)
        return ANN_ERR_INVALID_ARG;
    if (word & kStatusCapacityBit)
        return ANN_ERR_CAPACITY;
    if (word & kStatusTimeoutBit)
        return ANN_ERR_TIMEOUT;
    return ANN_OK;
}

}  // extern "C"
