// hbkm.cu -- hierarchical balanced k-means, HBKM (Sec. 4.1, Def. 2 and
// Algorithm 2), and the hub of every final cluster (Def. 3).
//
// Each of `levels` levels splits every cluster of the level above (level 0:
// the whole data set) into k children.  A split runs T iterations; each
// iteration empties the children, visits the cluster's members in
// increasing id and puts member x into
//     j = argmin_j ||x - mu_j||^2 + lam * (2 (c_j - m) + 1)
// (ties to the smaller j), c_j the child's current size and m = |C| / k.  The
// penalty is the increase of Def. 2's size-variance objective that adding x
// to child j causes; lam = lambda * sigma^2 / m, sigma^2 the members' mean
// squared distance to the cluster's centroid.  Every non-empty child then
// moves to its members' mean; an empty child keeps its centroid.  A split
// starts from its members with the min(k, |C|) smallest (key, id); children
// past |C| stay at the cluster's own centroid, empty.
//
// The assignment is an integer decided by float32 sums, so every float
// operation here is rounded on its own (no contraction) and summed in a fixed
// order: distances over coordinates 0..dim-1, sigma^2 and centroid sums over
// members in increasing id, division last.  The one sequential part, the
// visit in id order, runs as one warp per cluster (lane j = child j); the
// distances to the children, the centroid sums (one thread per coordinate)
// and the hub search are parallel.
//
// Layout: perm[] holds the row ids grouped by current cluster, increasing id
// inside a cluster; seg[] the clusters' first positions; own[] the cluster of
// each position.  A split's children keep that order (a stable partition), so
// each level's members are again in increasing id.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <utility>

#include "internal.h"

namespace ann {
namespace {

constexpr int kMaxBranch = 32;
constexpr int64_t kMaxClusters = int64_t{1} << 20;

// squared L2 over coordinates 0..dim-1, each step rounded on its own
__device__ __forceinline__ float dist_seq(const float *x, const float *mu, int dim)
{
    float acc = 0.f;
    for (int t = 0; t < dim; t += 4) {
        const float4 a = *reinterpret_cast<const float4 *>(x + t);
        const float4 b = *reinterpret_cast<const float4 *>(mu + t);
        float d = __fsub_rn(a.x, b.x);
        acc = __fadd_rn(acc, __fmul_rn(d, d));
        d = __fsub_rn(a.y, b.y);
        acc = __fadd_rn(acc, __fmul_rn(d, d));
        d = __fsub_rn(a.z, b.z);
        acc = __fadd_rn(acc, __fmul_rn(d, d));
        d = __fsub_rn(a.w, b.w);
        acc = __fadd_rn(acc, __fmul_rn(d, d));
    }
    return acc;
}

// order-preserving map of a float (finite or +inf) to unsigned bits
__device__ __forceinline__ uint32_t ord_bits(float v)
{
    const uint32_t u = __float_as_uint(v);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ void hb_setup_one(int64_t c, int k, float lambda, const int64_t *seg, const int32_t *perm,
                             const float *dp, const uint32_t *keys, float *lamv, float *mv, int32_t *kkv,
                             int32_t *init);
__device__ void hb_scan_one(int64_t c, int k, int lane, const int64_t *seg, const float *D, const float *lamv,
                            const float *mv, const int32_t *kkv, int32_t *lab, int32_t *cnt);
__device__ void hb_partition_one(int64_t c, int k, const int64_t *seg, const int32_t *perm, const int32_t *lab,
                                 const int32_t *cnt, int32_t *perm2, int32_t *own2, int64_t *seg2);
__device__ void hb_hub_one(int64_t c, int lane, const float *x, int dim, const int64_t *seg, const int32_t *perm,
                           const float *cent, int32_t *hubs);

// level 0: the mean of all rows, one thread per coordinate, rows in order
__global__ void hb_root(const float *x, int64_t n, int dim, float *cent)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < dim) {
        float s = 0.f;
        int64_t i = 0;
        for (; i + 8 <= n; i += 8) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                v[u] = x[(i + u) * dim + t];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                s = __fadd_rn(s, v[u]);
        }
        for (; i < n; ++i)
            s = __fadd_rn(s, x[i * dim + t]);
        cent[t] = __fdiv_rn(s, static_cast<float>(n));
    }
}

__global__ void hb_iota(int64_t n, int32_t *perm, int32_t *own)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        perm[i] = static_cast<int32_t>(i);
        own[i] = 0;
    }
}

// distance of every position's row to its cluster's centroid
__global__ void hb_dist_parent(const float *x, int dim, int64_t n, const int32_t *perm, const int32_t *own,
                               const float *cent, float *dp)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        dp[i] = dist_seq(x + static_cast<int64_t>(perm[i]) * dim, cent + static_cast<int64_t>(own[i]) * dim, dim);
}

// per cluster (one thread each): sigma^2, m, lam, and the starting members
__global__ void hb_setup(int64_t P, int k, float lambda, const int64_t *seg, const int32_t *perm, const float *dp,
                         const uint32_t *keys, float *lamv, float *mv, int32_t *kkv, int32_t *init)
{
    for (int64_t c = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; c < P;
         c += static_cast<int64_t>(gridDim.x) * blockDim.x)
        hb_setup_one(c, k, lambda, seg, perm, dp, keys, lamv, mv, kkv, init);
}

__device__ void hb_setup_one(int64_t c, int k, float lambda, const int64_t *seg, const int32_t *perm,
                             const float *dp, const uint32_t *keys, float *lamv, float *mv, int32_t *kkv,
                             int32_t *init)
{
    const int64_t b = seg[c], e = seg[c + 1], s = e - b;
    int32_t *ini = init + c * k;
    if (s == 0) {
        lamv[c] = 0.f;
        mv[c] = 0.f;
        kkv[c] = 0;
        for (int j = 0; j < k; ++j)
            ini[j] = -1;
        return;
    }
    float sig = 0.f;
    for (int64_t i = b; i < e; ++i)
        sig = __fadd_rn(sig, dp[i]);
    sig = __fdiv_rn(sig, static_cast<float>(s));
    const float m = __fdiv_rn(static_cast<float>(s), static_cast<float>(k));
    lamv[c] = __fdiv_rn(__fmul_rn(lambda, sig), m);
    mv[c] = m;
    const int kk = s < k ? static_cast<int>(s) : k;
    kkv[c] = kk;
    // the kk smallest (key, id), ascending, by insertion into a sorted list
    uint64_t top[kMaxBranch];
    int nt = 0;
    for (int64_t i = b; i < e; ++i) {
        const int32_t id = perm[i];
        const uint64_t v = (static_cast<uint64_t>(keys[id]) << 32) | static_cast<uint32_t>(id);
        if (nt == kk && v >= top[kk - 1])
            continue;
        int p = nt < kk ? nt++ : kk - 1;
        while (p > 0 && top[p - 1] > v) {
            top[p] = top[p - 1];
            --p;
        }
        top[p] = v;
    }
    for (int j = 0; j < k; ++j)
        ini[j] = j < kk ? static_cast<int32_t>(top[j] & 0xffffffffu) : -1;
}

// children's starting centroids: a starting member's row, else the parent's
__global__ void hb_init_children(const float *x, int dim, int k, const int32_t *init, const float *cent_p,
                                 float *cent_c)
{
    const int64_t cj = blockIdx.x;  // child c * k + j
    const int32_t id = init[cj];
    const float *src = id >= 0 ? x + static_cast<int64_t>(id) * dim : cent_p + (cj / k) * dim;
    for (int t = threadIdx.x; t < dim; t += blockDim.x)
        cent_c[cj * dim + t] = src[t];
}

// distance of every position's row to its cluster's k children (+inf past kk)
__global__ void hb_dist_children(const float *x, int dim, int64_t n, int k, const int32_t *perm,
                                 const int32_t *own, const int32_t *kkv, const float *cent_c, float *D)
{
    const int64_t total = n * k;
    for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < total;
         q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t i = q / k;
        const int j = static_cast<int>(q - i * k);
        const int32_t c = own[i];
        D[q] = j < kkv[c] ? dist_seq(x + static_cast<int64_t>(perm[i]) * dim,
                                     cent_c + (static_cast<int64_t>(c) * k + j) * dim, dim)
                          : __int_as_float(0x7f800000);
    }
}

// the visit in id order: one warp per cluster, lane j keeps child j's size
__global__ void hb_scan(int64_t P, int k, const int64_t *seg, const float *D, const float *lamv, const float *mv,
                        const int32_t *kkv, int32_t *lab, int32_t *cnt)
{
    const int lane = threadIdx.x & 31;
    const int64_t wpb = blockDim.x >> 5;
    for (int64_t c = blockIdx.x * wpb + (threadIdx.x >> 5); c < P; c += gridDim.x * wpb)
        hb_scan_one(c, k, lane, seg, D, lamv, mv, kkv, lab, cnt);
}

__device__ void hb_scan_one(int64_t c, int k, int lane, const int64_t *seg, const float *D, const float *lamv,
                            const float *mv, const int32_t *kkv, int32_t *lab, int32_t *cnt)
{
    const int64_t b = seg[c], e = seg[c + 1];
    const float lam = lamv[c], m = mv[c];
    const bool live = lane < kkv[c];
    int cj = 0;
    for (int64_t i0 = b; i0 < e; i0 += 8) {
        float dv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            dv[u] = (live && i0 + u < e) ? D[(i0 + u) * k + lane] : 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (i0 + u >= e)
                break;
            uint64_t key = ~0ull;
            if (live) {
                const float pen =
                    __fmul_rn(lam, __fadd_rn(__fmul_rn(2.f, __fsub_rn(static_cast<float>(cj), m)), 1.f));
                key = (static_cast<uint64_t>(ord_bits(__fadd_rn(dv[u], pen))) << 32) | static_cast<uint32_t>(lane);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const uint64_t other = __shfl_xor_sync(0xffffffffu, key, o);
                key = other < key ? other : key;
            }
            const int win = static_cast<int>(key & 0xffffffffu);
            if (lane == win)
                ++cj;
            if (lane == 0)
                lab[i0 + u] = win;
        }
    }
    if (lane < k)
        cnt[c * k + lane] = cj;
}

// children's means: one block per cluster, thread t sums coordinate t of
// every child in member order (shared sums: k x dim)
__global__ void hb_update(const float *x, int dim, int k, const int64_t *seg, const int32_t *perm,
                          const int32_t *lab, const int32_t *cnt, const int32_t *kkv, float *cent_c)
{
    extern __shared__ float sums[];
    const int64_t c = blockIdx.x;
    const int64_t b = seg[c], e = seg[c + 1];
    for (int q = threadIdx.x; q < k * dim; q += blockDim.x)
        sums[q] = 0.f;
    __syncthreads();
    for (int t = threadIdx.x; t < dim; t += blockDim.x) {
        int64_t i = b;
        for (; i + 8 <= e; i += 8) {
            int32_t r[8], j[8];
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                r[u] = perm[i + u];
                j[u] = lab[i + u];
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                v[u] = x[static_cast<int64_t>(r[u]) * dim + t];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                sums[j[u] * dim + t] = __fadd_rn(sums[j[u] * dim + t], v[u]);
        }
        for (; i < e; ++i)
            sums[lab[i] * dim + t] = __fadd_rn(sums[lab[i] * dim + t], x[static_cast<int64_t>(perm[i]) * dim + t]);
        const int kk = kkv[c];
        for (int j = 0; j < kk; ++j) {
            const int32_t cn = cnt[c * k + j];
            if (cn > 0)
                cent_c[(c * k + j) * dim + t] = __fdiv_rn(sums[j * dim + t], static_cast<float>(cn));
        }
    }
}

// stable partition of every cluster's members by child (one thread per cluster)
__global__ void hb_partition(int64_t P, int k, const int64_t *seg, const int32_t *perm, const int32_t *lab,
                             const int32_t *cnt, int32_t *perm2, int32_t *own2, int64_t *seg2)
{
    for (int64_t c = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; c < P;
         c += static_cast<int64_t>(gridDim.x) * blockDim.x)
        hb_partition_one(c, k, seg, perm, lab, cnt, perm2, own2, seg2);
}

__device__ void hb_partition_one(int64_t c, int k, const int64_t *seg, const int32_t *perm, const int32_t *lab,
                                 const int32_t *cnt, int32_t *perm2, int32_t *own2, int64_t *seg2)
{
    int64_t off[kMaxBranch];
    int64_t o = seg[c];
    for (int j = 0; j < k; ++j) {
        off[j] = o;
        seg2[c * k + j] = o;
        o += cnt[c * k + j];
    }
    for (int64_t i = seg[c]; i < seg[c + 1]; ++i) {
        const int j = lab[i];
        const int64_t d = off[j]++;
        perm2[d] = perm[i];
        own2[d] = static_cast<int32_t>(c * k + j);
    }
}

// hub of every final cluster: its member nearest the centroid (smaller id on
// ties), one warp per cluster; labels back in row order
__global__ void hb_hubs(const float *x, int dim, int64_t nc, const int64_t *seg, const int32_t *perm,
                        const float *cent, int32_t *hubs)
{
    const int lane = threadIdx.x & 31;
    const int64_t wpb = blockDim.x >> 5;
    for (int64_t c = blockIdx.x * wpb + (threadIdx.x >> 5); c < nc; c += gridDim.x * wpb)
        hb_hub_one(c, lane, x, dim, seg, perm, cent, hubs);
}

__device__ void hb_hub_one(int64_t c, int lane, const float *x, int dim, const int64_t *seg, const int32_t *perm,
                           const float *cent, int32_t *hubs)
{
    uint64_t best = ~0ull;
    for (int64_t i = seg[c] + lane; i < seg[c + 1]; i += 32) {
        const int32_t id = perm[i];
        const float d = dist_seq(x + static_cast<int64_t>(id) * dim, cent + c * dim, dim);
        const uint64_t key = (static_cast<uint64_t>(ord_bits(d)) << 32) | static_cast<uint32_t>(id);
        best = key < best ? key : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t other = __shfl_xor_sync(0xffffffffu, best, o);
        best = other < best ? other : best;
    }
    if (lane == 0)
        hubs[c] = best == ~0ull ? -1 : static_cast<int32_t>(best & 0xffffffffu);
}

__global__ void hb_labels(int64_t n, const int32_t *perm, const int32_t *own, int32_t *label)
{
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        label[perm[i]] = own[i];
}

struct Buf {
    void *p = nullptr;
    cudaStream_t s;
    explicit Buf(cudaStream_t st) : s(st) {}
    cudaError_t alloc(size_t bytes) { return cudaMallocAsync(&p, std::max<size_t>(bytes, 16), s); }
    template <typename T>
    T *as() const
    {
        return static_cast<T *>(p);
    }
    ~Buf()
    {
        if (p)
            cudaFreeAsync(p, s);
    }
};

#define HB_CK(x)                         \
    do {                                 \
        cudaError_t e_ = (x);            \
        if (e_ != cudaSuccess)           \
            return cuda_status(e_);      \
    } while (0)

unsigned grid_for(int64_t items, int per_block)
{
    return static_cast<unsigned>(std::min<int64_t>((items + per_block - 1) / per_block, 152 * 64));
}

}  // namespace
}  // namespace ann

using namespace ann;

extern "C" {

ann_status ann_hbkm(const float *d_x, int64_t n, int32_t dim, int32_t k, int32_t levels, double lambda, int32_t T,
                    const uint32_t *d_keys, int32_t *d_hubs, float *d_centroids, int32_t *d_label, void *stream)
{
    if (!d_x || !d_keys || !d_hubs || n < 1 || n > INT32_MAX || dim < 4 || dim % 4 != 0 || dim > 4096 || k < 2 ||
        k > kMaxBranch || levels < 1 || T < 1 || !(lambda >= 0.0) ||
        (reinterpret_cast<uintptr_t>(d_x) & 15) || (reinterpret_cast<uintptr_t>(d_centroids) & 15))
        return ANN_ERR_INVALID_ARG;
    int64_t nc = 1;
    for (int l = 0; l < levels; ++l) {
        nc *= k;
        if (nc > kMaxClusters)
            return ANN_ERR_INVALID_ARG;
    }
    const size_t smem = static_cast<size_t>(k) * dim * 4;
    if (smem > 227 * 1024)
        return ANN_ERR_UNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    HB_CK(cudaFuncSetAttribute(hb_update, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    Buf perm(s), perm2(s), own(s), own2(s), seg(s), seg2(s), cent(s), cent2(s), dp(s), D(s), lab(s), cnt(s),
        lamv(s), mv(s), kkv(s), init(s);
    const int64_t cl_max = nc;  // clusters of the last level; earlier levels have fewer
    HB_CK(perm.alloc(n * 4));
    HB_CK(perm2.alloc(n * 4));
    HB_CK(own.alloc(n * 4));
    HB_CK(own2.alloc(n * 4));
    HB_CK(seg.alloc((cl_max + 1) * 8));
    HB_CK(seg2.alloc((cl_max + 1) * 8));
    HB_CK(cent.alloc(cl_max * dim * 4));
    HB_CK(cent2.alloc(cl_max * dim * 4));
    HB_CK(dp.alloc(n * 4));
    HB_CK(D.alloc(n * k * 4));
    HB_CK(lab.alloc(n * 4));
    HB_CK(cnt.alloc(cl_max * 4));
    HB_CK(lamv.alloc(cl_max / k * 4));
    HB_CK(mv.alloc(cl_max / k * 4));
    HB_CK(kkv.alloc(cl_max / k * 4));
    HB_CK(init.alloc(cl_max * 4));

    hb_iota<<<grid_for(n, 256), 256, 0, s>>>(n, perm.as<int32_t>(), own.as<int32_t>());
    hb_root<<<(dim + 127) / 128, 128, 0, s>>>(d_x, n, dim, cent.as<float>());
    const int64_t seg0[2] = {0, n};
    HB_CK(cudaMemcpyAsync(seg.p, seg0, sizeof(seg0), cudaMemcpyHostToDevice, s));
    int64_t P = 1;
    for (int l = 1; l <= levels; ++l) {
        hb_dist_parent<<<grid_for(n, 256), 256, 0, s>>>(d_x, dim, n, perm.as<int32_t>(), own.as<int32_t>(),
                                                        cent.as<float>(), dp.as<float>());
        hb_setup<<<grid_for(P, 128), 128, 0, s>>>(P, k, static_cast<float>(lambda), seg.as<int64_t>(),
                                                  perm.as<int32_t>(), dp.as<float>(), d_keys, lamv.as<float>(),
                                                  mv.as<float>(), kkv.as<int32_t>(), init.as<int32_t>());
        hb_init_children<<<static_cast<unsigned>(P * k), 128, 0, s>>>(d_x, dim, k, init.as<int32_t>(),
                                                                       cent.as<float>(), cent2.as<float>());
        for (int it = 0; it < T; ++it) {
            hb_dist_children<<<grid_for(n * k, 256), 256, 0, s>>>(d_x, dim, n, k, perm.as<int32_t>(),
                                                                  own.as<int32_t>(), kkv.as<int32_t>(),
                                                                  cent2.as<float>(), D.as<float>());
            hb_scan<<<grid_for(P * 32, 128), 128, 0, s>>>(P, k, seg.as<int64_t>(), D.as<float>(), lamv.as<float>(),
                                                          mv.as<float>(), kkv.as<int32_t>(), lab.as<int32_t>(),
                                                          cnt.as<int32_t>());
            hb_update<<<static_cast<unsigned>(P), std::min(((dim + 31) / 32) * 32, 1024), smem, s>>>(
                d_x, dim, k, seg.as<int64_t>(), perm.as<int32_t>(), lab.as<int32_t>(), cnt.as<int32_t>(),
                kkv.as<int32_t>(), cent2.as<float>());
        }
        hb_partition<<<grid_for(P, 128), 128, 0, s>>>(P, k, seg.as<int64_t>(), perm.as<int32_t>(), lab.as<int32_t>(),
                                                      cnt.as<int32_t>(), perm2.as<int32_t>(), own2.as<int32_t>(),
                                                      seg2.as<int64_t>());
        P *= k;
        HB_CK(cudaMemcpyAsync(seg2.as<int64_t>() + P, &n, 8, cudaMemcpyHostToDevice, s));
        HB_CK(cudaStreamSynchronize(s));  // the host value of n above stays valid until here
        std::swap(perm.p, perm2.p);
        std::swap(own.p, own2.p);
        std::swap(seg.p, seg2.p);
        std::swap(cent.p, cent2.p);
        HB_CK(cudaGetLastError());
    }
    hb_hubs<<<grid_for(nc * 32, 128), 128, 0, s>>>(d_x, dim, nc, seg.as<int64_t>(), perm.as<int32_t>(),
                                                   cent.as<float>(), d_hubs);
    if (d_label)
        hb_labels<<<grid_for(n, 256), 256, 0, s>>>(n, perm.as<int32_t>(), own.as<int32_t>(), d_label);
    if (d_centroids)
        HB_CK(cudaMemcpyAsync(d_centroids, cent.p, nc * dim * 4, cudaMemcpyDeviceToDevice, s));
    HB_CK(cudaGetLastError());
    HB_CK(cudaStreamSynchronize(s));
    return ANN_OK;
}

}  // extern "C"
