// build.cu -- offline index construction on the GPU: exact k-NN (also the
// ground truth of recall@k), the proximity graph of Sec. 2.1 Def. 1 (K-NN
// candidates, relative-neighbourhood pruning, reachability repair from the
// navigating node) and the navigating node (medoid).
//
// k-NN: candidate scores come from a plain cuBLAS SGEMM (x.y per query chunk);
// a warp per row keeps the best KP = k + margin keys by the expanded distance
// |y|^2 - 2 x.y with a threshold filter, then the KP candidates are re-scored
// exactly (direct differences: int32 for uint8, fp32 otherwise) and sorted by
// (distance, id).
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "device_util.cuh"
#include "internal.h"

namespace ann {
namespace {

constexpr int kSelWarps = 4;

__global__ void u8_to_f32(const uint8_t *x, float *y, int64_t count)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < count;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        y[i] = static_cast<float>(x[i]);
}

// squared norms of fp32 rows (exact integers for uint8-valued rows)
__global__ void row_norms(const float *x, int64_t n, int dim, float *out)
{
    const int lane = threadIdx.x & 31;
    const int64_t row = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
    if (row >= n)
        return;
    float s = 0.f;
    for (int c = lane; c < dim; c += 32) {
        const float v = x[row * dim + c];
        s = fmaf(v, v, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        s += __shfl_xor_sync(kFull, s, o);
    if (lane == 0)
        out[row] = s;
}

// Per row of a chunk of scores S (rows x ld, row-major): keep the KP = 32*KPL
// smallest keys (expanded distance, column id).  L2: key distance =
// ny[j] - 2 S[r][j]; IP: -S[r][j].  Column self0 + r is skipped when
// exclude_self.  Output: KP candidate ids per row, best first.
template <int KPL>
__global__ void __launch_bounds__(32 * kSelWarps)
    select_topk(const float *S, int64_t ld, int64_t N, int rows, const float *ny, int metric,
                int64_t self0, int exclude_self, int32_t *out)
{
    constexpr int KP = 32 * KPL;
    constexpr int BCAP = 256;
    __shared__ uint64_t sh_top[kSelWarps][2][KP];
    __shared__ uint64_t sh_buf[kSelWarps][BCAP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int r = blockIdx.x * kSelWarps + w;
    if (r >= rows)
        return;
    uint64_t *T = sh_top[w][0];
    uint64_t *Tn = sh_top[w][1];
    uint64_t *B = sh_buf[w];
    for (int i = lane; i < KP; i += 32)
        T[i] = kKeyMax;
    __syncwarp();
    uint64_t thr = kKeyMax;
    int nb = 0;
    const float *row = S + static_cast<int64_t>(r) * ld;
    const int64_t self = exclude_self ? self0 + r : -1;

    auto flush = [&]() {
        // sort the buffer (pad to 256 with max keys) ...
        uint64_t k[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int e = t * 32 + lane;
            k[t] = e < nb ? B[e] : kKeyMax;
        }
        warp_sort_n<8>(k, lane);
        __syncwarp();
#pragma unroll
        for (int t = 0; t < 8; ++t)
            B[t * 32 + lane] = k[t];
        __syncwarp();
        // ... and merge it with the kept list by rank
        for (int i = lane; i < KP; i += 32) {
            const uint64_t v = T[i];
            const int pos = i + count_less_raw(B, nb, v);
            if (pos < KP)
                Tn[pos] = v;
        }
        for (int j = lane; j < nb; j += 32) {
            const uint64_t v = B[j];
            const int pos = j + count_less_raw(T, KP, v);
            if (pos < KP)
                Tn[pos] = v;
        }
        __syncwarp();
        uint64_t *t = T;
        T = Tn;
        Tn = t;
        thr = T[KP - 1];
        nb = 0;
    };

    for (int64_t j0 = 0; j0 < N; j0 += 128) {
        const int64_t j = j0 + 4 * lane;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j < N)
            v = *reinterpret_cast<const float4 *>(row + j);  // ld % 4 == 0, padded columns exist
        const float vs[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int64_t c = j + t;
            uint64_t key = kKeyMax;
            if (c < N && c != self) {
                const float d = metric == ANN_L2 ? fmaf(-2.f, vs[t], ny[c]) : -vs[t];
                key = make_key(f32_to_ord(d), static_cast<int32_t>(c)) >> 1;  // id in low 31 bits
            }
            const bool pass = key < thr;
            const unsigned m = __ballot_sync(kFull, pass);
            if (pass)
                B[nb + __popc(m & lanemask_lt())] = key;
            nb += __popc(m);
        }
        __syncwarp();
        if (nb >= BCAP - 128)
            flush();
    }
    if (nb > 0)
        flush();
    for (int i = lane; i < KP; i += 32) {
        const uint64_t v = T[i];
        out[static_cast<int64_t>(r) * KP + i] = v == kKeyMax ? -1 : static_cast<int32_t>(v & 0x7fffffffu);
    }
}

// exact distance between a base row and a query row (uint8: int32 squared L2)
template <int DT, int MT>
__device__ __forceinline__ uint32_t exact_dist_bits(const uint8_t *x, const uint8_t *q, int dim)
{
    if constexpr (DT == ANN_U8) {
        uint32_t acc = 0;
        for (int c = 0; c < dim / 4; ++c) {
            const uint32_t a = reinterpret_cast<const uint32_t *>(x)[c];
            const uint32_t b = reinterpret_cast<const uint32_t *>(q)[c];
            const uint32_t d = __vabsdiffu4(a, b);
            acc = __dp4a(d, d, acc);
        }
        return acc;
    } else {
        const float4 *x4 = reinterpret_cast<const float4 *>(x);
        const float4 *q4 = reinterpret_cast<const float4 *>(q);
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        for (int c = 0; c < dim / 4; ++c) {
            const float4 u = x4[c], v = q4[c];
            if constexpr (MT == ANN_L2) {
                const float d0 = u.x - v.x, d1 = u.y - v.y, d2 = u.z - v.z, d3 = u.w - v.w;
                a0 = fmaf(d0, d0, a0);
                a1 = fmaf(d1, d1, a1);
                a2 = fmaf(d2, d2, a2);
                a3 = fmaf(d3, d3, a3);
            } else {
                a0 = fmaf(u.x, v.x, a0);
                a1 = fmaf(u.y, v.y, a1);
                a2 = fmaf(u.z, v.z, a2);
                a3 = fmaf(u.w, v.w, a3);
            }
        }
        float s = (a0 + a1) + (a2 + a3);
        if constexpr (MT == ANN_IP)
            s = -s;
        return f32_to_ord(s);
    }
}

// Re-score the KP candidates of each query exactly, sort by (distance, id),
// write the best k ids and distances (int32 for uint8, fp32 otherwise).
template <int DT, int MT, int KPL>
__global__ void rescore_topk(const uint8_t *base, int rowbytes, const uint8_t *queries, int qbytes,
                             int dim, int64_t nq, const int32_t *cand, int k, int32_t *out_ids,
                             void *out_dists)
{
    constexpr int KP = 32 * KPL;
    const int lane = threadIdx.x & 31;
    const int64_t r = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
    if (r >= nq)
        return;
    const uint8_t *q = queries + r * qbytes;
    uint64_t key[KPL];
#pragma unroll
    for (int t = 0; t < KPL; ++t) {
        const int32_t id = cand[r * KP + t * 32 + lane];
        key[t] = id < 0 ? kKeyMax
                        : make_key(exact_dist_bits<DT, MT>(base + static_cast<int64_t>(id) * rowbytes, q, dim), id);
    }
    warp_sort_n<KPL>(key, lane);
#pragma unroll
    for (int t = 0; t < KPL; ++t) {
        const int e = t * 32 + lane;
        if (e < k) {
            const uint64_t v = key[t];
            const bool ok = v != kKeyMax;
            out_ids[r * k + e] = ok ? key_id(v) : -1;
            const uint32_t db = static_cast<uint32_t>(v >> 32);
            if constexpr (DT == ANN_U8)
                reinterpret_cast<int32_t *>(out_dists)[r * k + e] = ok ? static_cast<int32_t>(db) : INT32_MAX;
            else
                reinterpret_cast<float *>(out_dists)[r * k + e] = ok ? ord_to_f32(db) : __int_as_float(0x7f800000);
        }
    }
}

// Relative-neighbourhood pruning of node p's K candidates (sorted by exact
// (dist, id)): c is kept unless a node s kept before it has
// alpha * delta(s, c) <= delta(p, c); at most R are kept; -1 pads the row.
// STAGED: the K candidate rows are copied into shared memory first (when they
// fit); otherwise they are read from global memory (L1/L2-cached) in place.
template <int DT, bool STAGED>
__global__ void rng_prune(const uint8_t *base, int rowbytes, int dim, int64_t n, const int32_t *cand,
                          const void *cand_d, int K, int R, float alpha, int stride, int32_t *graph)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    const int64_t p = blockIdx.x;
    if (p >= n)
        return;
    uint8_t *rows = smem;
    int32_t *kept = reinterpret_cast<int32_t *>(smem + (STAGED ? static_cast<size_t>(K) * stride : 0));
    if constexpr (STAGED) {
        for (int c = 0; c < K; ++c) {
            const int32_t id = cand[p * K + c];
            if (id < 0)
                continue;
            const uint4 *src = reinterpret_cast<const uint4 *>(base + static_cast<int64_t>(id) * rowbytes);
            uint4 *dst = reinterpret_cast<uint4 *>(rows + c * stride);
            for (int o = lane; o < rowbytes / 16; o += 32)
                dst[o] = src[o];
        }
        __syncwarp();
    }
    auto row = [&](int c) -> const uint8_t * {
        if constexpr (STAGED)
            return rows + c * stride;
        else
            return base + static_cast<int64_t>(cand[p * K + c]) * rowbytes;
    };
    int nk = 0;
    for (int c = 0; c < K && nk < R; ++c) {
        const int32_t id = cand[p * K + c];
        if (id < 0)
            break;
        float dpc;
        if constexpr (DT == ANN_U8)
            dpc = static_cast<float>(reinterpret_cast<const int32_t *>(cand_d)[p * K + c]);
        else
            dpc = reinterpret_cast<const float *>(cand_d)[p * K + c];
        bool pruned = false;
        for (int j = lane; j < nk; j += 32) {
            const int s = kept[j];
            float dsc;
            if constexpr (DT == ANN_U8)
                dsc = static_cast<float>(exact_dist_bits<ANN_U8, ANN_L2>(row(s), row(c), dim));
            else
                dsc = ord_to_f32(exact_dist_bits<ANN_F32, ANN_L2>(row(s), row(c), dim));
            pruned |= alpha * dsc <= dpc;
        }
        if (!__any_sync(kFull, pruned)) {
            if (lane == 0)
                kept[nk] = c;
            ++nk;
        }
        __syncwarp();
    }
    for (int j = lane; j < R; j += 32)
        graph[p * R + j] = j < nk ? cand[p * K + kept[j]] : -1;
}

// ---- medoid ---------------------------------------------------------------

template <typename T, typename Acc>
__global__ void col_partial_sums(const T *x, int64_t n, int dim, int64_t rows_per, Acc *partial)
{
    const int64_t r0 = blockIdx.x * rows_per;
    const int64_t r1 = min(n, r0 + rows_per);
    for (int c = threadIdx.x; c < dim; c += blockDim.x) {
        Acc s = 0;
        for (int64_t r = r0; r < r1; ++r)
            s += static_cast<Acc>(x[r * dim + c]);
        partial[blockIdx.x * static_cast<int64_t>(dim) + c] = s;
    }
}

template <typename Acc>
__global__ void col_total(const Acc *partial, int blocks, int dim, Acc *total)
{
    for (int c = threadIdx.x; c < dim; c += blockDim.x) {
        Acc s = 0;
        for (int b = 0; b < blocks; ++b)
            s += partial[static_cast<int64_t>(b) * dim + c];
        total[c] = s;
    }
}

// fp32: key = (ord(|x - mean|^2), id), atomicMin gives the (dist, id) argmin
__global__ void medoid_f32(const float *x, int64_t n, int dim, const float *sum, unsigned long long *best)
{
    const int lane = threadIdx.x & 31;
    const int64_t row = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
    if (row >= n)
        return;
    const float inv = 1.0f / static_cast<float>(n);
    float s = 0.f;
    for (int c = lane; c < dim; c += 32) {
        const float d = x[row * dim + c] - sum[c] * inv;
        s = fmaf(d, d, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        s += __shfl_xor_sync(kFull, s, o);
    if (lane == 0)
        atomicMin(best, static_cast<unsigned long long>(make_key(f32_to_ord(s), static_cast<int32_t>(row)) >> 1));
}

// uint8: exact ||n x - sum||^2 in 64-bit integers; first pass the minimum
// value, second pass the smallest id attaining it
__global__ void medoid_u8_value(const uint8_t *x, int64_t n, int dim, const unsigned long long *sum,
                                unsigned long long *vals, unsigned long long *best)
{
    const int lane = threadIdx.x & 31;
    const int64_t row = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
    if (row >= n)
        return;
    unsigned long long s = 0;
    for (int c = lane; c < dim; c += 32) {
        const long long v = n * static_cast<long long>(x[row * dim + c]) - static_cast<long long>(sum[c]);
        s += static_cast<unsigned long long>(v * v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        s += __shfl_xor_sync(kFull, s, o);
    if (lane == 0) {
        vals[row] = s;
        atomicMin(best, s);
    }
}

__global__ void medoid_u8_id(const unsigned long long *vals, int64_t n, const unsigned long long *best,
                             unsigned long long *best_id)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        if (vals[i] == *best)
            atomicMin(best_id, static_cast<unsigned long long>(i));
}

// ---- reachability repair ----------------------------------------------------

// nearest eligible node to row u: key (ord distance, id), atomicMin
template <int DT>
__global__ void nearest_eligible(const uint8_t *base, int rowbytes, int dim, int64_t n, int64_t u,
                                 const uint8_t *eligible, unsigned long long *best)
{
    const int lane = threadIdx.x & 31;
    const int64_t w = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
    if (w >= n || !eligible[w])
        return;
    const uint8_t *xu = base + u * rowbytes;
    const uint8_t *xw = base + w * rowbytes;
    uint32_t bits;
    if constexpr (DT == ANN_U8) {
        uint32_t acc = 0;
        for (int c = lane; c < dim / 4; c += 32) {
            const uint32_t d = __vabsdiffu4(reinterpret_cast<const uint32_t *>(xu)[c],
                                            reinterpret_cast<const uint32_t *>(xw)[c]);
            acc = __dp4a(d, d, acc);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            acc += __shfl_xor_sync(kFull, acc, o);
        bits = acc;
    } else {
        float s = 0.f;
        for (int c = lane; c < dim; c += 32) {
            const float d = reinterpret_cast<const float *>(xu)[c] - reinterpret_cast<const float *>(xw)[c];
            s = fmaf(d, d, s);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            s += __shfl_xor_sync(kFull, s, o);
        bits = f32_to_ord(s);
    }
    if (lane == 0)
        atomicMin(best, static_cast<unsigned long long>(make_key(bits, static_cast<int32_t>(w)) >> 1));
}

__global__ void set_flags(uint8_t *flags, const int32_t *ids, int count, uint8_t v)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count)
        flags[ids[i]] = v;
}

struct Cublas {
    cublasHandle_t h = nullptr;
    ~Cublas()
    {
        if (h)
            cublasDestroy(h);
    }
};

template <typename T>
struct DevBuf {
    T *p = nullptr;
    cudaStream_t s = nullptr;
    cudaError_t alloc(size_t count, cudaStream_t st)
    {
        s = st;
        return cudaMallocAsync(reinterpret_cast<void **>(&p), count * sizeof(T), st);
    }
    ~DevBuf()
    {
        if (p)
            cudaFreeAsync(p, s);
    }
};

#define CK(x)                                \
    do {                                     \
        cudaError_t e_ = (x);                \
        if (e_ != cudaSuccess)               \
            return cuda_status(e_);          \
    } while (0)

size_t kp_for(int k) { return k <= 32 ? 64 : 128; }

}  // namespace

// Exact k-NN of nq query rows among n base rows (see file comment).
ann_status knn_exact(const void *d_base, int64_t n, int dim, int dtype, int metric, const void *d_queries,
                     int64_t nq, int k, bool exclude_self, int32_t *d_ids, void *d_dists, cudaStream_t s)
{
    const int es = elem_size(dtype);
    const int rowbytes = dim * es;
    const int qbytes = dtype == ANN_U8 ? dim : dim * 4;
    const int KP = static_cast<int>(kp_for(k));
    // fp32 views of base and queries for the GEMM
    DevBuf<float> bf, qf, ny, Sbuf;
    DevBuf<int32_t> cand;
    const float *B = static_cast<const float *>(d_base);
    const float *Q = static_cast<const float *>(d_queries);
    if (dtype == ANN_U8) {
        CK(bf.alloc(static_cast<size_t>(n) * dim, s));
        u8_to_f32<<<2048, 256, 0, s>>>(static_cast<const uint8_t *>(d_base), bf.p, n * dim);
        B = bf.p;
        if (d_queries == d_base) {
            Q = bf.p;
        } else {
            CK(qf.alloc(static_cast<size_t>(nq) * dim, s));
            u8_to_f32<<<2048, 256, 0, s>>>(static_cast<const uint8_t *>(d_queries), qf.p, nq * dim);
            Q = qf.p;
        }
    } else if (dtype != ANN_F32) {
        return ANN_ERR_UNSUPPORTED;
    }
    CK(ny.alloc(n, s));
    row_norms<<<static_cast<unsigned>((n * 32 + 255) / 256), 256, 0, s>>>(B, n, dim, ny.p);
    const int64_t ld = (n + 3) / 4 * 4;
    const size_t budget = static_cast<size_t>(4) << 30;  // bytes of scores per chunk
    int64_t qc = std::max<int64_t>(1, std::min<int64_t>(nq, static_cast<int64_t>(budget / (4 * ld))));
    CK(Sbuf.alloc(static_cast<size_t>(qc) * ld, s));
    CK(cand.alloc(static_cast<size_t>(qc) * KP, s));
    Cublas cb;
    if (cublasCreate(&cb.h) != CUBLAS_STATUS_SUCCESS)
        return ANN_ERR_CUDA;
    cublasSetStream(cb.h, s);
    cublasSetMathMode(cb.h, CUBLAS_PEDANTIC_MATH);  // true fp32, no reduced-precision modes
    const float one = 1.f, zero = 0.f;
    for (int64_t q0 = 0; q0 < nq; q0 += qc) {
        const int rows = static_cast<int>(std::min<int64_t>(qc, nq - q0));
        // S (rows x n, row-major, ld) = Q[q0:q0+rows] . B^T
        if (cublasSgemm(cb.h, CUBLAS_OP_T, CUBLAS_OP_N, static_cast<int>(n), rows, dim, &one, B, dim,
                        Q + q0 * dim, dim, &zero, Sbuf.p, static_cast<int>(ld)) != CUBLAS_STATUS_SUCCESS)
            return ANN_ERR_CUDA;
        const unsigned grid = (rows + kSelWarps - 1) / kSelWarps;
        if (KP == 64)
            select_topk<2><<<grid, 32 * kSelWarps, 0, s>>>(Sbuf.p, ld, n, rows, ny.p, metric, q0,
                                                           exclude_self ? 1 : 0, cand.p);
        else
            select_topk<4><<<grid, 32 * kSelWarps, 0, s>>>(Sbuf.p, ld, n, rows, ny.p, metric, q0,
                                                           exclude_self ? 1 : 0, cand.p);
        CK(cudaGetLastError());
        const uint8_t *qb = static_cast<const uint8_t *>(d_queries) + q0 * qbytes;
        const unsigned rgrid = static_cast<unsigned>((rows * 32 + 127) / 128);
        int32_t *oi = d_ids + q0 * k;
        void *od = static_cast<uint8_t *>(d_dists) + q0 * k * 4;
        const uint8_t *bb = static_cast<const uint8_t *>(d_base);
#define RESCORE(DT, MT, KPL) \
    rescore_topk<DT, MT, KPL><<<rgrid, 128, 0, s>>>(bb, rowbytes, qb, qbytes, dim, rows, cand.p, k, oi, od)
        if (dtype == ANN_U8)
            KP == 64 ? RESCORE(ANN_U8, ANN_L2, 2) : RESCORE(ANN_U8, ANN_L2, 4);
        else if (metric == ANN_L2)
            KP == 64 ? RESCORE(ANN_F32, ANN_L2, 2) : RESCORE(ANN_F32, ANN_L2, 4);
        else
            KP == 64 ? RESCORE(ANN_F32, ANN_IP, 2) : RESCORE(ANN_F32, ANN_IP, 4);
#undef RESCORE
        CK(cudaGetLastError());
    }
    return ANN_OK;
}

ann_status medoid_gpu(const void *d_base, int64_t n, int dim, int dtype, cudaStream_t s, int32_t *out)
{
    const int blocks = static_cast<int>(std::min<int64_t>(1024, n));
    const int64_t rows_per = (n + blocks - 1) / blocks;
    const unsigned rgrid = static_cast<unsigned>((n * 32 + 255) / 256);
    if (dtype == ANN_U8) {
        if (n > (1 << 20) || dim > 128)
            return ANN_ERR_UNSUPPORTED;  // keeps ||n x - sum||^2 within 64 bits
        DevBuf<unsigned long long> part, tot, vals, best;
        CK(part.alloc(static_cast<size_t>(blocks) * dim, s));
        CK(tot.alloc(dim, s));
        CK(vals.alloc(n, s));
        CK(best.alloc(2, s));
        CK(cudaMemsetAsync(best.p, 0xff, 16, s));
        col_partial_sums<uint8_t, unsigned long long><<<blocks, 128, 0, s>>>(
            static_cast<const uint8_t *>(d_base), n, dim, rows_per, part.p);
        col_total<unsigned long long><<<1, 128, 0, s>>>(part.p, blocks, dim, tot.p);
        medoid_u8_value<<<rgrid, 256, 0, s>>>(static_cast<const uint8_t *>(d_base), n, dim, tot.p, vals.p, best.p);
        medoid_u8_id<<<1024, 256, 0, s>>>(vals.p, n, best.p, best.p + 1);
        unsigned long long id = 0;
        CK(cudaMemcpyAsync(&id, best.p + 1, 8, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        *out = static_cast<int32_t>(id);
        return ANN_OK;
    }
    if (dtype != ANN_F32)
        return ANN_ERR_UNSUPPORTED;
    DevBuf<float> part, tot;
    DevBuf<unsigned long long> best;
    CK(part.alloc(static_cast<size_t>(blocks) * dim, s));
    CK(tot.alloc(dim, s));
    CK(best.alloc(1, s));
    CK(cudaMemsetAsync(best.p, 0xff, 8, s));
    col_partial_sums<float, float><<<blocks, 128, 0, s>>>(static_cast<const float *>(d_base), n, dim,
                                                          rows_per, part.p);
    col_total<float><<<1, 128, 0, s>>>(part.p, blocks, dim, tot.p);
    medoid_f32<<<rgrid, 256, 0, s>>>(static_cast<const float *>(d_base), n, dim, tot.p, best.p);
    unsigned long long key = 0;
    CK(cudaMemcpyAsync(&key, best.p, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *out = static_cast<int32_t>(key & 0x7fffffffu);
    return ANN_OK;
}

ann_status prune_rows(const void *d_base, int64_t n, int dim, int dtype, int K, int R, float alpha,
                      const int32_t *cand, const void *cand_d, int32_t *d_graph, cudaStream_t s);
ann_status repair_reachability(const void *d_base, int64_t n, int dim, int dtype, int R, int32_t *d_graph,
                               int32_t medoid_id, int64_t *repairs, cudaStream_t s);

ann_status build_graph_gpu(const void *d_base, int64_t n, int dim, int dtype, int K, int R, float alpha,
                           int32_t *d_graph, int32_t *medoid, int64_t *repairs, cudaStream_t s)
{
    // 1. exact K-NN candidates of every node (itself excluded)
    DevBuf<int32_t> cids;
    DevBuf<float> cd;
    CK(cids.alloc(static_cast<size_t>(n) * K, s));
    CK(cd.alloc(static_cast<size_t>(n) * K, s));
    ann_status st = knn_exact(d_base, n, dim, dtype, ANN_L2, d_base, n, K, true, cids.p, cd.p, s);
    if (st != ANN_OK)
        return st;
    // 2. relative-neighbourhood pruning
    if ((st = prune_rows(d_base, n, dim, dtype, K, R, alpha, cids.p, cd.p, d_graph, s)) != ANN_OK)
        return st;
    // 3. navigating node
    if (*medoid < 0 && (st = medoid_gpu(d_base, n, dim, dtype, s, medoid)) != ANN_OK)
        return st;
    // 4. reachability repair
    return repair_reachability(d_base, n, dim, dtype, R, d_graph, *medoid, repairs, s);
}

// Relative-neighbourhood pruning of n candidate rows (K per row, ascending
// (distance, id), -1 pads at the end) into the n adjacency rows at d_graph.
ann_status prune_rows(const void *d_base, int64_t n, int dim, int dtype, int K, int R, float alpha,
                      const int32_t *cand, const void *cand_d, int32_t *d_graph, cudaStream_t s)
{
    const int es = elem_size(dtype);
    const int rowbytes = dim * es;
    int s16 = rowbytes / 16;
    if ((s16 & 1) == 0)
        s16 += 1;
    const int stride = s16 * 16;
    const bool staged = static_cast<size_t>(K) * stride <= 64 * 1024;
    const size_t smem = (staged ? static_cast<size_t>(K) * stride : 0) + 4 * 64;
    const uint8_t *bb = static_cast<const uint8_t *>(d_base);
    const unsigned grid = static_cast<unsigned>(n);
#define PRUNE(DT, ST)                                                                                          \
    do {                                                                                                       \
        CK(cudaFuncSetAttribute(rng_prune<DT, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize,               \
                                static_cast<int>(smem)));                                                      \
        rng_prune<DT, ST><<<grid, 32, smem, s>>>(bb, rowbytes, dim, n, cand, cand_d, K, R, alpha, stride,      \
                                                 d_graph);                                                     \
    } while (0)
    if (dtype == ANN_U8 && staged)
        PRUNE(ANN_U8, true);
    else if (dtype == ANN_U8)
        PRUNE(ANN_U8, false);
    else if (staged)
        PRUNE(ANN_F32, true);
    else
        PRUNE(ANN_F32, false);
#undef PRUNE
    return cuda_status(cudaGetLastError());
}

// Reachability repair: nodes in id order; an unreachable node u gets the edge
// w -> u from the nearest reachable node w with a free slot; all that u
// reaches becomes reachable before the next node is taken.
ann_status repair_reachability(const void *d_base, int64_t n, int dim, int dtype, int R, int32_t *d_graph,
                               int32_t medoid_id, int64_t *repairs, cudaStream_t s)
{
    const int rowbytes = dim * elem_size(dtype);
    const int32_t *medoid = &medoid_id;
    std::vector<int32_t> g(static_cast<size_t>(n) * R);
    CK(cudaMemcpyAsync(g.data(), d_graph, g.size() * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::vector<uint8_t> reached(n, 0);
    std::vector<int32_t> deg(n, 0), queue;
    queue.reserve(n);
    for (int64_t v = 0; v < n; ++v) {
        int c = 0;
        while (c < R && g[v * R + c] >= 0)
            ++c;
        deg[v] = c;
    }
    auto bfs_from = [&](int32_t src, std::vector<int32_t> &newly) {
        newly.clear();
        if (reached[src])
            return;
        reached[src] = 1;
        newly.push_back(src);
        for (size_t h = 0; h < newly.size(); ++h) {
            const int32_t v = newly[h];
            for (int j = 0; j < R; ++j) {
                const int32_t x = g[static_cast<int64_t>(v) * R + j];
                if (x >= 0 && !reached[x]) {
                    reached[x] = 1;
                    newly.push_back(x);
                }
            }
        }
    };
    std::vector<int32_t> newly;
    bfs_from(*medoid, newly);
    int64_t added = 0;
    if (static_cast<int64_t>(newly.size()) < n) {
        DevBuf<uint8_t> elig;
        DevBuf<int32_t> ids;
        DevBuf<unsigned long long> best;
        CK(elig.alloc(n, s));
        CK(ids.alloc(n, s));
        CK(best.alloc(1, s));
        std::vector<uint8_t> eh(n);
        for (int64_t v = 0; v < n; ++v)
            eh[v] = reached[v] && deg[v] < R;
        CK(cudaMemcpyAsync(elig.p, eh.data(), n, cudaMemcpyHostToDevice, s));
        std::vector<int32_t> upd;
        for (int64_t u = 0; u < n; ++u) {
            if (reached[u])
                continue;
            CK(cudaMemsetAsync(best.p, 0xff, 8, s));
            const unsigned grid = static_cast<unsigned>((n * 32 + 255) / 256);
            if (dtype == ANN_U8)
                nearest_eligible<ANN_U8><<<grid, 256, 0, s>>>(static_cast<const uint8_t *>(d_base), rowbytes, dim, n,
                                                              u, elig.p, best.p);
            else
                nearest_eligible<ANN_F32><<<grid, 256, 0, s>>>(static_cast<const uint8_t *>(d_base), rowbytes, dim,
                                                               n, u, elig.p, best.p);
            unsigned long long key = 0;
            CK(cudaMemcpyAsync(&key, best.p, 8, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (key == ~0ull)
                return ANN_ERR_CAPACITY;  // no reachable node has a free slot
            const int32_t w = static_cast<int32_t>(key & 0x7fffffffu);
            g[static_cast<int64_t>(w) * R + deg[w]] = static_cast<int32_t>(u);
            CK(cudaMemcpyAsync(d_graph + static_cast<int64_t>(w) * R + deg[w], &g[static_cast<int64_t>(w) * R + deg[w]],
                               4, cudaMemcpyHostToDevice, s));
            deg[w]++;
            ++added;
            bfs_from(static_cast<int32_t>(u), newly);
            upd.clear();
            for (int32_t v : newly)
                if (deg[v] < R)
                    upd.push_back(v);
            if (!upd.empty()) {
                CK(cudaMemcpyAsync(ids.p, upd.data(), upd.size() * 4, cudaMemcpyHostToDevice, s));
                set_flags<<<static_cast<unsigned>((upd.size() + 255) / 256), 256, 0, s>>>(
                    elig.p, ids.p, static_cast<int>(upd.size()), 1);
            }
            if (deg[w] >= R) {
                CK(cudaMemsetAsync(elig.p + w, 0, 1, s));
            }
            CK(cudaStreamSynchronize(s));  // host vectors are reused next iteration
        }
    }
    if (repairs)
        *repairs = added;
    CK(cudaStreamSynchronize(s));
    return ANN_OK;
}

namespace {

constexpr int kInbox = 32;  // reverse-edge requests kept per node and batch

// every new node's out-edges become requests in their targets' inboxes
__global__ void reverse_collect(const int32_t *rows, int64_t b0, int64_t nb, int R, int32_t *inbox, int32_t *cnt,
                                int32_t *touched, int32_t *ntouched)
{
    const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (t >= nb * R)
        return;
    const int32_t q = rows[t];
    if (q < 0)
        return;
    const int slot = atomicAdd(&cnt[q], 1);
    if (slot == 0)
        touched[atomicAdd(ntouched, 1)] = q;
    if (slot < kInbox)
        inbox[static_cast<int64_t>(q) * kInbox + slot] = static_cast<int32_t>(b0 + t / R);
}

// A touched node's row: its neighbours plus its inbox; appended while they
// fit, else all of them sorted by (squared L2, id) and pruned to R as
// rng_prune does.  One warp per node (R <= 32: lane j holds slot j of the
// row and inbox entry j).
__global__ void reverse_prune(const float *x, int dim, const int32_t *touched, const int32_t *ntouched,
                              const int32_t *inbox, int32_t *cnt, int R, float alpha, int32_t *graph)
{
    __shared__ uint64_t keys[64];
    __shared__ int32_t kept[32];
    const int lane = threadIdx.x;
    const int nt = *ntouched;
    const uint8_t *xb = reinterpret_cast<const uint8_t *>(x);
    const int rowbytes = dim * 4;
    for (int w = blockIdx.x; w < nt; w += gridDim.x) {
        const int32_t q = touched[w];
        const int nin = min(cnt[q], kInbox);
        const int32_t c0 = lane < R ? graph[static_cast<int64_t>(q) * R + lane] : -1;
        const int32_t c1 = lane < nin ? inbox[static_cast<int64_t>(q) * kInbox + lane] : -1;
        const int deg = __popc(__ballot_sync(kFull, c0 >= 0));
        if (deg + nin <= R) {
            if (lane < nin)
                graph[static_cast<int64_t>(q) * R + deg + lane] = c1;
        } else {
            const uint8_t *xq = xb + static_cast<int64_t>(q) * rowbytes;
            uint64_t k0 = c0 >= 0 ? make_key(exact_dist_bits<ANN_F32, ANN_L2>(xb + static_cast<int64_t>(c0) * rowbytes,
                                                                               xq, dim), c0)
                                  : kKeyMax;
            uint64_t k1 = c1 >= 0 ? make_key(exact_dist_bits<ANN_F32, ANN_L2>(xb + static_cast<int64_t>(c1) * rowbytes,
                                                                               xq, dim), c1)
                                  : kKeyMax;
            warp_sort64(k0, k1, lane);
            keys[lane] = k0;
            keys[lane + 32] = k1;
            __syncwarp();
            int nk = 0;
            for (int c = 0; c < 64 && nk < R; ++c) {
                const uint64_t kc = keys[c];
                if (kc == kKeyMax)
                    break;
                const int32_t id = key_id(kc);
                const float dqc = ord_to_f32(static_cast<uint32_t>(kc >> 32));
                bool pruned = false;
                for (int j = lane; j < nk; j += 32)
                    pruned |= alpha * ord_to_f32(exact_dist_bits<ANN_F32, ANN_L2>(
                                          xb + static_cast<int64_t>(kept[j]) * rowbytes,
                                          xb + static_cast<int64_t>(id) * rowbytes, dim)) <= dqc;
                if (!__any_sync(kFull, pruned)) {
                    if (lane == 0)
                        kept[nk] = id;
                    ++nk;
                }
                __syncwarp();
            }
            if (lane < R)
                graph[static_cast<int64_t>(q) * R + lane] = lane < nk ? kept[lane] : -1;
        }
        __syncwarp();
        if (lane == 0)
            cnt[q] = 0;
    }
}

}  // namespace

// Insertion by search: the exact graph of the first n0 rows, then batches of
// rows each searched on the graph built so far (their k nearest found become
// their candidates, pruned to R), with the reverse edges added or re-pruned;
// then the navigating node of all rows and the reachability repair.
ann_status build_graph_insert(const float *x, int64_t n, int dim, int K, int R, float alpha, int64_t n0,
                              int64_t batch, int32_t *d_graph, int32_t *medoid, int64_t *repairs, cudaStream_t s)
{
    int device = 0;
    CK(cudaGetDevice(&device));
    int32_t m0 = -1;
    ann_status st = build_graph_gpu(x, n0, dim, ANN_F32, K, R, alpha, d_graph, &m0, nullptr, s);
    if (st != ANN_OK)
        return st;
    CK(cudaMemsetAsync(d_graph + n0 * R, 0xff, static_cast<size_t>(n - n0) * R * 4, s));
    DevBuf<int32_t> inbox, cnt, touched, ntouched, ids;
    DevBuf<float> dd;
    CK(inbox.alloc(static_cast<size_t>(n) * kInbox, s));
    CK(cnt.alloc(n, s));
    CK(touched.alloc(n, s));
    CK(ntouched.alloc(1, s));
    CK(ids.alloc(static_cast<size_t>(batch) * K, s));
    CK(dd.alloc(static_cast<size_t>(batch) * K, s));
    CK(cudaMemsetAsync(cnt.p, 0, n * 4, s));
    ann_search_params p{};
    p.k = K;
    p.L = std::max(K, 128);
    p.W = R <= 32 ? 4 : 2;
    for (int64_t b0 = n0, nb = 0; b0 < n; b0 += nb) {
        // a batch holds at most a quarter of the rows inserted so far: rows of
        // one batch do not see each other
        nb = std::min({batch, n - b0, std::max<int64_t>(1, b0 / 4)});
        // the graph so far (rows past b0 are empty, so unreachable)
        ann_index_desc desc{};
        desc.n = n;
        desc.dim = dim;
        desc.degree = R;
        desc.dtype = ANN_F32;
        desc.metric = ANN_L2;
        desc.base = x;
        desc.graph = d_graph;
        desc.medoid = m0;
        CK(cudaStreamSynchronize(s));
        ann_index *idx = nullptr;
        if ((st = ann_index_create(&desc, device, &idx)) != ANN_OK)
            return st;
        st = ann_search_batch(idx, x + b0 * dim, nb, nullptr, &p, ids.p, dd.p, nullptr, s);
        if (st == ANN_OK)
            st = ann_sync_status(idx, s);
        ann_free_index(idx);
        if (st != ANN_OK)
            return st;
        if ((st = prune_rows(x, nb, dim, ANN_F32, K, R, alpha, ids.p, dd.p, d_graph + b0 * R, s)) != ANN_OK)
            return st;
        CK(cudaMemsetAsync(ntouched.p, 0, 4, s));
        reverse_collect<<<static_cast<unsigned>((nb * R + 255) / 256), 256, 0, s>>>(
            d_graph + b0 * R, b0, nb, R, inbox.p, cnt.p, touched.p, ntouched.p);
        reverse_prune<<<152 * 8, 32, 0, s>>>(x, dim, touched.p, ntouched.p, inbox.p, cnt.p, R, alpha, d_graph);
        CK(cudaGetLastError());
    }
    if (*medoid < 0 && (st = medoid_gpu(x, n, dim, ANN_F32, s, medoid)) != ANN_OK)
        return st;
    return repair_reachability(x, n, dim, ANN_F32, R, d_graph, *medoid, repairs, s);
}

}  // namespace ann

using namespace ann;

extern "C" {

ann_status ann_knn(const void *d_base, int64_t n, int32_t dim, int32_t dtype, int32_t metric,
                   const void *d_queries, int64_t nq, int32_t k, int32_t exclude_self, int32_t *d_ids,
                   void *d_dists, void *stream)
{
    const int es = elem_size(dtype);
    if (!d_base || !d_queries || !d_ids || !d_dists || n < 1 || n > INT32_MAX || dim < 1 || nq < 0 ||
        k < 1 || k > 128 || k > n || es == 0 || (metric != ANN_L2 && metric != ANN_IP))
        return ANN_ERR_INVALID_ARG;
    if ((dtype != ANN_U8 && dtype != ANN_F32) || (dtype == ANN_U8 && metric != ANN_L2))
        return ANN_ERR_UNSUPPORTED;
    if ((static_cast<int64_t>(dim) * es) % 16 != 0 || (exclude_self && d_queries != d_base) ||
        (reinterpret_cast<uintptr_t>(d_base) & 15) || (reinterpret_cast<uintptr_t>(d_queries) & 15))
        return ANN_ERR_INVALID_ARG;
    if (nq == 0)
        return ANN_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ann_status st = knn_exact(d_base, n, dim, dtype, metric, d_queries, nq, k, exclude_self != 0, d_ids, d_dists, s);
    if (st == ANN_OK)
        st = cuda_status(cudaStreamSynchronize(s));
    return st;
}

ann_status ann_medoid(const void *d_base, int64_t n, int32_t dim, int32_t dtype, int32_t *medoid, void *stream)
{
    if (!d_base || !medoid || n < 1 || n > INT32_MAX || dim < 1)
        return ANN_ERR_INVALID_ARG;
    return medoid_gpu(d_base, n, dim, dtype, static_cast<cudaStream_t>(stream), medoid);
}

ann_status ann_build_graph_insert(const void *d_base, int64_t n, int32_t dim, int32_t dtype, int32_t K, int32_t R,
                                  float alpha, int64_t n_seed, int64_t batch, int32_t *d_graph, int32_t *medoid,
                                  int64_t *repairs, void *stream)
{
    if (!d_base || !d_graph || !medoid || n < 2 || n > INT32_MAX || dim < 4 || K < 1 || K > 128 || R < 1 ||
        R > K || R > 32 || !(alpha > 0.f) || n_seed < K + 1 || n_seed > n || batch < 1 || *medoid >= n)
        return ANN_ERR_INVALID_ARG;
    if (dtype != ANN_F32)
        return ANN_ERR_UNSUPPORTED;
    if ((static_cast<int64_t>(dim) * 4) % 16 != 0 || (reinterpret_cast<uintptr_t>(d_base) & 15))
        return ANN_ERR_INVALID_ARG;
    return build_graph_insert(static_cast<const float *>(d_base), n, dim, K, R, alpha, n_seed,
                              std::min<int64_t>(batch, n), d_graph, medoid, repairs,
                              static_cast<cudaStream_t>(stream));
}

ann_status ann_build_graph(const void *d_base, int64_t n, int32_t dim, int32_t dtype, int32_t K, int32_t R,
                           float alpha, int32_t *d_graph, int32_t *medoid, int64_t *repairs, void *stream)
{
    const int es = elem_size(dtype);
    if (!d_base || !d_graph || !medoid || n < 2 || n > INT32_MAX || dim < 1 || K < 1 || K > 128 ||
        K > n - 1 || R < 1 || R > K || R > 64 || !(alpha > 0.f) || es == 0)
        return ANN_ERR_INVALID_ARG;
    if (dtype != ANN_U8 && dtype != ANN_F32)
        return ANN_ERR_UNSUPPORTED;
    if ((static_cast<int64_t>(dim) * es) % 16 != 0 ||
        (reinterpret_cast<uintptr_t>(d_base) & 15) || *medoid >= n)
        return ANN_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return build_graph_gpu(d_base, n, dim, dtype, K, R, alpha, d_graph, medoid, repairs, s);
}

}  // extern "C"
