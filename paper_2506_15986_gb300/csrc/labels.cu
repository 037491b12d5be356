// labels.cu -- hub extraction and query-aware training labels on the GPU.
//
// Hubs (Sec. 4.1, Def. 3): Lloyd's k-means on a sample (a flat stand-in for
// the balanced hierarchical clustering of Algorithm 2), then, for each
// cluster of the full base set, the member nearest its centroid.
// Labels (Sec. 4.2, Def. 4 and the per-query assignment after it): for each
// training query q and candidate hub v, run the greedy search of Algorithm 1
// from v in label mode (stop after the step in which q's exact nearest
// neighbour is evaluated) and record the evaluations and expansions; then per
// query: best = argmin (evals, hops, hub), m = min hops, positive if
// hops <= m + t_pos, negative if hops >= m + t_neg, never reached, or not
// searched, otherwise unused.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "device_util.cuh"
#include "internal.h"

namespace ann {
namespace {

__global__ void gather_rows(const uint8_t *src, int rowbytes, const int64_t *rows, int64_t m, uint8_t *dst)
{
    const int64_t i = blockIdx.x;
    if (i >= m)
        return;
    const uint8_t *s = src + rows[i] * rowbytes;
    uint8_t *d = dst + i * rowbytes;
    for (int o = threadIdx.x * 16; o < rowbytes; o += blockDim.x * 16)
        *reinterpret_cast<uint4 *>(d + o) = *reinterpret_cast<const uint4 *>(s + o);
}

// centroid j = mean of its members (listed in id order by the host), in fp32
template <typename T>
__global__ void centroid_update(const T *x, int dim, const int64_t *order, const int64_t *start, float *cent)
{
    const int j = blockIdx.x;
    const int64_t a = start[j], b = start[j + 1];
    if (a == b)
        return;  // empty: re-seeded by the host
    for (int c = threadIdx.x; c < dim; c += blockDim.x) {
        float s = 0.f;
        for (int64_t i = a; i < b; ++i)
            s += static_cast<float>(x[order[i] * dim + c]);
        cent[static_cast<int64_t>(j) * dim + c] = s / static_cast<float>(b - a);
    }
}

template <typename T>
__global__ void set_centroid_rows(const T *x, int dim, const int64_t *rows, const int32_t *which, int count,
                                  float *cent)
{
    const int i = blockIdx.x;
    if (i >= count)
        return;
    for (int c = threadIdx.x; c < dim; c += blockDim.x)
        cent[static_cast<int64_t>(which[i]) * dim + c] = static_cast<float>(x[rows[i] * dim + c]);
}

__global__ void to_f32(const uint8_t *x, int64_t count, float *y)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < count;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        y[i] = static_cast<float>(x[i]);
}

// hub of cluster j: member with the smallest (distance to centroid, id)
__global__ void hub_argmin(const int32_t *assign, const void *dist, int dtype, int64_t n, unsigned long long *best)
{
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i >= n)
        return;
    const int j = assign[i];
    if (j < 0)
        return;
    const uint32_t bits = dtype == ANN_U8 ? static_cast<uint32_t>(static_cast<const int32_t *>(dist)[i])
                                          : f32_to_ord(static_cast<const float *>(dist)[i]);
    atomicMin(best + j, (static_cast<unsigned long long>(bits) << 31) | static_cast<unsigned long long>(i));
}

__global__ void hub_ids_from_keys(const unsigned long long *best, int k, int32_t *hubs)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < k)
        hubs[j] = best[j] == ~0ull ? -1 : static_cast<int32_t>(best[j] & 0x7fffffffull);
}

__global__ void expand_entries(const int32_t *cand, int64_t count, const int32_t *hub_nodes, int32_t *entries)
{
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i < count)
        entries[i] = hub_nodes[cand[i]];
}

// one thread per query: the label rule over its M searched hubs, written as
// labels aligned with the candidate list (hubs not listed are negatives)
__global__ void label_rule_kernel(const int32_t *evals, const int32_t *hops, const int32_t *cand, int64_t nq, int M,
                                  int t_pos, int t_neg, int8_t *lab, int32_t *best)
{
    const int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (q >= nq)
        return;
    int8_t *row = lab + q * M;
    const int32_t *ev = evals + q * M, *hp = hops + q * M, *cd = cand + q * M;
    int mh = INT32_MAX, be = -1;
    for (int j = 0; j < M; ++j) {
        if (hp[j] == INT32_MAX)
            continue;
        mh = min(mh, hp[j]);
        if (be < 0 || ev[j] < ev[be] || (ev[j] == ev[be] && (hp[j] < hp[be] || (hp[j] == hp[be] && cd[j] < cd[be]))))
            be = j;
    }
    if (best)
        best[q] = be >= 0 ? cd[be] : -1;
    for (int j = 0; j < M; ++j) {
        int8_t v;
        if (be < 0 || hp[j] == INT32_MAX)
            v = -1;  // no hub reached the target, or this one never did
        else if (hp[j] <= mh + t_pos)
            v = 1;
        else if (hp[j] >= mh + t_neg)
            v = -1;
        else
            v = 0;
        row[j] = v;
    }
}

#define CK(x)                            \
    do {                                 \
        cudaError_t e_ = (x);            \
        if (e_ != cudaSuccess)           \
            return cuda_status(e_);      \
    } while (0)

struct Scoped {
    void *p = nullptr;
    cudaStream_t s;
    explicit Scoped(cudaStream_t st) : s(st) {}
    cudaError_t alloc(size_t bytes) { return cudaMallocAsync(&p, std::max<size_t>(bytes, 16), s); }
    ~Scoped()
    {
        if (p)
            cudaFreeAsync(p, s);
    }
};

}  // namespace
}  // namespace ann

using namespace ann;

extern "C" {

ann_status ann_kmeans(const void *d_x, int64_t n, int32_t dim, int32_t dtype, const int64_t *sample_rows,
                      int64_t m, int32_t k, const int32_t *init, int32_t iters, float *d_centroids,
                      double *objective, void *stream)
{
    const int es = elem_size(dtype);
    if (!d_x || !sample_rows || !init || !d_centroids || n < 1 || dim < 1 || m < 1 || m > n || k < 1 || k > m ||
        k > 1 << 20 || iters < 0 || (dtype != ANN_U8 && dtype != ANN_F32) || (dim * es) % 16 != 0)
        return ANN_ERR_INVALID_ARG;
    for (int j = 0; j < k; ++j)
        if (init[j] < 0 || init[j] >= m)
            return ANN_ERR_INVALID_ARG;
    for (int64_t i = 0; i < m; ++i)
        if (sample_rows[i] < 0 || sample_rows[i] >= n)
            return ANN_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int rowbytes = dim * es;
    // the sample, as fp32 rows (the k-NN assignment runs on fp32 data)
    Scoped rows(s), xs(s), xf(s), ids(s), dd(s), ord(s), st(s), which(s), srows(s);
    CK(rows.alloc(m * 8));
    CK(xs.alloc(static_cast<size_t>(m) * rowbytes));
    CK(xf.alloc(static_cast<size_t>(m) * dim * 4));
    CK(ids.alloc(m * 4));
    CK(dd.alloc(m * 4));
    CK(ord.alloc(m * 8));
    CK(st.alloc((k + 1) * 8));
    CK(which.alloc(k * 4));
    CK(srows.alloc(k * 8));
    CK(cudaMemcpyAsync(rows.p, sample_rows, m * 8, cudaMemcpyHostToDevice, s));
    gather_rows<<<static_cast<unsigned>(m), 128, 0, s>>>(static_cast<const uint8_t *>(d_x), rowbytes,
                                                          static_cast<int64_t *>(rows.p), m,
                                                          static_cast<uint8_t *>(xs.p));
    float *X = static_cast<float *>(xf.p);
    if (dtype == ANN_U8)
        to_f32<<<1024, 256, 0, s>>>(static_cast<uint8_t *>(xs.p), m * dim, X);
    else
        CK(cudaMemcpyAsync(X, xs.p, static_cast<size_t>(m) * dim * 4, cudaMemcpyDeviceToDevice, s));
    // initial centroids: sample rows init[0..k)
    std::vector<int64_t> lr(k);
    std::vector<int32_t> wj(k);
    for (int j = 0; j < k; ++j) {
        lr[j] = init[j];
        wj[j] = j;
    }
    CK(cudaMemcpyAsync(srows.p, lr.data(), k * 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(which.p, wj.data(), k * 4, cudaMemcpyHostToDevice, s));
    set_centroid_rows<float><<<k, 128, 0, s>>>(X, dim, static_cast<int64_t *>(srows.p),
                                               static_cast<int32_t *>(which.p), k, d_centroids);
    std::vector<int32_t> asg(m);
    std::vector<float> dist(m);
    std::vector<int64_t> order(m), start(k + 1);
    for (int it = 0; it < iters; ++it) {
        ann_status r = knn_exact(d_centroids, k, dim, ANN_F32, ANN_L2, X, m, 1, false,
                                 static_cast<int32_t *>(ids.p), dd.p, s);
        if (r != ANN_OK)
            return r;
        CK(cudaMemcpyAsync(asg.data(), ids.p, m * 4, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(dist.data(), dd.p, m * 4, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        double obj = 0.0;
        for (int64_t i = 0; i < m; ++i)
            obj += dist[i];
        if (objective)
            objective[it] = obj;
        // members of each centroid in row order (counting sort)
        std::fill(start.begin(), start.end(), 0);
        for (int64_t i = 0; i < m; ++i)
            start[asg[i] + 1]++;
        for (int j = 0; j < k; ++j)
            start[j + 1] += start[j];
        std::vector<int64_t> fill(start.begin(), start.end() - 1);
        for (int64_t i = 0; i < m; ++i)
            order[fill[asg[i]]++] = i;
        CK(cudaMemcpyAsync(ord.p, order.data(), m * 8, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(st.p, start.data(), (k + 1) * 8, cudaMemcpyHostToDevice, s));
        centroid_update<float><<<k, 128, 0, s>>>(X, dim, static_cast<int64_t *>(ord.p),
                                                 static_cast<int64_t *>(st.p), d_centroids);
        // empty centroids move onto the rows farthest from their centroid
        // (larger distance first, smaller row on ties), each row used once
        std::vector<int32_t> empty;
        for (int j = 0; j < k; ++j)
            if (start[j] == start[j + 1])
                empty.push_back(j);
        if (!empty.empty()) {
            std::vector<int64_t> idx(m);
            std::iota(idx.begin(), idx.end(), 0);
            std::stable_sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) { return dist[a] > dist[b]; });
            for (size_t e = 0; e < empty.size(); ++e)
                lr[e] = idx[e];
            CK(cudaMemcpyAsync(srows.p, lr.data(), empty.size() * 8, cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(which.p, empty.data(), empty.size() * 4, cudaMemcpyHostToDevice, s));
            set_centroid_rows<float><<<static_cast<unsigned>(empty.size()), 128, 0, s>>>(
                X, dim, static_cast<int64_t *>(srows.p), static_cast<int32_t *>(which.p),
                static_cast<int>(empty.size()), d_centroids);
        }
        CK(cudaStreamSynchronize(s));  // host vectors are reused next iteration
    }
    CK(cudaStreamSynchronize(s));
    return ANN_OK;
}

ann_status ann_assign_hubs(const void *d_base, int64_t n, int32_t dim, int32_t dtype, const float *d_centroids,
                           int32_t k, int32_t *d_hubs, int32_t *d_assign, void *stream)
{
    const int es = elem_size(dtype);
    if (!d_base || !d_centroids || !d_hubs || n < 1 || dim < 1 || k < 1 || (dtype != ANN_U8 && dtype != ANN_F32) ||
        (dim * es) % 16 != 0)
        return ANN_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Scoped xf(s), asg(s), dd(s), best(s);
    const float *X = static_cast<const float *>(d_base);
    if (dtype == ANN_U8) {
        CK(xf.alloc(static_cast<size_t>(n) * dim * 4));
        to_f32<<<2048, 256, 0, s>>>(static_cast<const uint8_t *>(d_base), n * dim, static_cast<float *>(xf.p));
        X = static_cast<float *>(xf.p);
    }
    int32_t *A = d_assign;
    if (!A) {
        CK(asg.alloc(n * 4));
        A = static_cast<int32_t *>(asg.p);
    }
    CK(dd.alloc(n * 4));
    CK(best.alloc(static_cast<size_t>(k) * 8));
    ann_status r = knn_exact(d_centroids, k, dim, ANN_F32, ANN_L2, X, n, 1, false, A, dd.p, s);
    if (r != ANN_OK)
        return r;
    CK(cudaMemsetAsync(best.p, 0xff, static_cast<size_t>(k) * 8, s));
    hub_argmin<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(A, dd.p, ANN_F32, n,
                                                                        static_cast<unsigned long long *>(best.p));
    hub_ids_from_keys<<<(k + 255) / 256, 256, 0, s>>>(static_cast<unsigned long long *>(best.p), k, d_hubs);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    return ANN_OK;
}

ann_status ann_hub_costs(ann_index *idx, const void *d_queries, int64_t nq, const int32_t *d_targets,
                         const int32_t *d_cand, int32_t M, const int32_t *d_hub_nodes, int32_t L, int32_t W,
                         int32_t *d_evals, int32_t *d_hops, void *stream)
{
    if (!idx || !d_queries || !d_targets || !d_cand || !d_hub_nodes || !d_evals || !d_hops || nq < 0 || M < 1 ||
        L < 1 || L > ANN_MAX_L || W < 1 || W > ANN_MAX_W || W * idx->degree > ANN_MAX_STEP_CAND ||
        (reinterpret_cast<uintptr_t>(d_queries) & 15))
        return ANN_ERR_INVALID_ARG;
    if (nq == 0)
        return ANN_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t items = nq * M;
    Scoped ent(s), ids(s), dists(s), stats(s);
    CK(ent.alloc(items * 4));
    CK(ids.alloc(items * 4));
    CK(dists.alloc(items * 4));
    CK(stats.alloc(items * 8));
    expand_entries<<<static_cast<unsigned>((items + 255) / 256), 256, 0, s>>>(d_cand, items, d_hub_nodes,
                                                                              static_cast<int32_t *>(ent.p));
    ann_search_params p{};
    p.k = 1;
    p.L = L;
    p.W = W;
    p.d_target = d_targets;
    SearchLaunch Ls{};
    Ls.queries = d_queries;
    Ls.qbytes = idx->dtype == ANN_U8 ? idx->dim : idx->dim * 4;
    Ls.nq = items;
    Ls.qdiv = M;
    Ls.entries = static_cast<int32_t *>(ent.p);
    Ls.p = &p;
    Ls.ids = static_cast<int32_t *>(ids.p);
    Ls.dists = dists.p;
    Ls.stats = static_cast<int32_t *>(stats.p);
    ann_status r = launch_search(idx, Ls, s);
    if (r != ANN_OK)
        return r;
    // split {evals, hops} pairs
    CK(cudaMemcpy2DAsync(d_evals, 4, stats.p, 8, 4, items, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpy2DAsync(d_hops, 4, static_cast<uint8_t *>(stats.p) + 4, 8, 4, items, cudaMemcpyDeviceToDevice, s));
    return ANN_OK;
}

ann_status ann_hub_labels(const int32_t *d_evals, const int32_t *d_hops, const int32_t *d_cand, int64_t nq, int32_t M,
                          int32_t t_pos, int32_t t_neg, int8_t *d_labels, int32_t *d_best, void *stream)
{
    if (!d_evals || !d_hops || !d_cand || !d_labels || nq < 0 || M < 1 || t_pos < 0 || t_neg < 0)
        return ANN_ERR_INVALID_ARG;
    if (nq == 0)
        return ANN_OK;
    label_rule_kernel<<<static_cast<unsigned>((nq + 127) / 128), 128, 0, static_cast<cudaStream_t>(stream)>>>(
        d_evals, d_hops, d_cand, nq, M, t_pos, t_neg, d_labels, d_best);
    return cuda_status(cudaGetLastError());
}

}  // extern "C"
