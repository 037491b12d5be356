// fusion.cu -- forward and backward of the fusion embedding (Sec. 4.3,
// Eq. fusion); see fusion.h.  One CTA per hub holds the hub's vector, tokens,
// projections and attention weights in shared memory; the weights' gradients
// are sums over hubs (in hub order, one thread per weight), so they are
// deterministic.  The sizes are small (H hubs x T tokens x heads*dk), so
// plain FP32 arithmetic serves; no step here is a large dense contraction.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <new>

#include "fusion.h"

namespace ann {
namespace {

constexpr int kThreads = 128;

// shared layout for one hub: p [dp] | U [T*dU] | q [E] | K [T*E] | V [T*E] | A [heads*T] | O [E]
__global__ void __launch_bounds__(kThreads)
    fusion_fwd_kernel(const float *P, const float *U, const float *W, int H, int T, int dU, int heads, int dk,
                      int dp, int dF, float scale, float *Qc, float *Kc, float *Vc, float *Ac, float *Oc, float *F,
                      const float *Ebase, float *Eeff)
{
    extern __shared__ float sh[];
    const int E = heads * dk;
    const int hb = blockIdx.x;
    float *p = sh, *u = p + dp, *q = u + T * dU, *K = q + E, *V = K + T * E, *A = V + T * E, *O = A + heads * T;
    const float *WQ = W, *WK = WQ + static_cast<int64_t>(dp) * E, *WV = WK + dU * E, *WO = WV + dU * E;
    for (int i = threadIdx.x; i < dp; i += blockDim.x)
        p[i] = P[static_cast<int64_t>(hb) * dp + i];
    for (int i = threadIdx.x; i < T * dU; i += blockDim.x)
        u[i] = U[static_cast<int64_t>(hb) * T * dU + i];
    __syncthreads();
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        float acc = 0.f;
        for (int i = 0; i < dp; ++i)
            acc = fmaf(p[i], WQ[i * E + e], acc);
        q[e] = acc;
    }
    for (int te = threadIdx.x; te < T * E; te += blockDim.x) {
        const int t = te / E, e = te - t * E;
        float ak = 0.f, av = 0.f;
        for (int i = 0; i < dU; ++i) {
            ak = fmaf(u[t * dU + i], WK[i * E + e], ak);
            av = fmaf(u[t * dU + i], WV[i * E + e], av);
        }
        K[te] = ak;
        V[te] = av;
    }
    __syncthreads();
    for (int jt = threadIdx.x; jt < heads * T; jt += blockDim.x) {
        const int j = jt / T, t = jt - j * T;
        float acc = 0.f;
        for (int d = 0; d < dk; ++d)
            acc = fmaf(q[j * dk + d], K[t * E + j * dk + d], acc);
        A[jt] = acc * scale;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < heads; j += blockDim.x) {
        float mx = -INFINITY;
        for (int t = 0; t < T; ++t)
            mx = fmaxf(mx, A[j * T + t]);
        float sum = 0.f;
        for (int t = 0; t < T; ++t) {
            const float ex = expf(A[j * T + t] - mx);
            A[j * T + t] = ex;
            sum += ex;
        }
        for (int t = 0; t < T; ++t)
            A[j * T + t] /= sum;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const int j = e / dk;
        float acc = 0.f;
        for (int t = 0; t < T; ++t)
            acc = fmaf(A[j * T + t], V[t * E + e], acc);
        O[e] = acc;
    }
    __syncthreads();
    for (int f = threadIdx.x; f < dF; f += blockDim.x) {
        float acc = 0.f;
        for (int e = 0; e < E; ++e)
            acc = fmaf(O[e], WO[e * dF + f], acc);
        const int64_t o = static_cast<int64_t>(hb) * dF + f;
        F[o] = acc;
        if (Eeff)
            Eeff[o] = Ebase[o] + acc;
    }
    // the cache for the backward
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        Qc[static_cast<int64_t>(hb) * E + e] = q[e];
        Oc[static_cast<int64_t>(hb) * E + e] = O[e];
    }
    for (int te = threadIdx.x; te < T * E; te += blockDim.x) {
        Kc[static_cast<int64_t>(hb) * T * E + te] = K[te];
        Vc[static_cast<int64_t>(hb) * T * E + te] = V[te];
    }
    for (int jt = threadIdx.x; jt < heads * T; jt += blockDim.x)
        Ac[static_cast<int64_t>(hb) * heads * T + jt] = A[jt];
}

// per hub: dO = dF WO^T, then through the attention to dQ, dK, dV
// shared: dO [E] | dA [heads*T] | r [heads]
__global__ void __launch_bounds__(kThreads)
    fusion_bwd_kernel(const float *dF, const float *W, int H, int T, int dU, int heads, int dk, int dp, int dF_dim,
                      float scale, const float *Qc, const float *Kc, const float *Vc, const float *Ac, float *dQ,
                      float *dK, float *dV)
{
    extern __shared__ float sh[];
    const int E = heads * dk;
    const int hb = blockIdx.x;
    float *dO = sh, *dA = dO + E, *r = dA + heads * T;
    const float *WO = W + static_cast<int64_t>(dp) * E + 2 * dU * E;
    const float *A = Ac + static_cast<int64_t>(hb) * heads * T;
    const float *K = Kc + static_cast<int64_t>(hb) * T * E, *V = Vc + static_cast<int64_t>(hb) * T * E;
    const float *q = Qc + static_cast<int64_t>(hb) * E;
    const float *g = dF + static_cast<int64_t>(hb) * dF_dim;
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        float acc = 0.f;
        for (int f = 0; f < dF_dim; ++f)
            acc = fmaf(g[f], WO[e * dF_dim + f], acc);
        dO[e] = acc;
    }
    __syncthreads();
    for (int jt = threadIdx.x; jt < heads * T; jt += blockDim.x) {
        const int j = jt / T, t = jt - j * T;
        float acc = 0.f;
        for (int d = 0; d < dk; ++d)
            acc = fmaf(dO[j * dk + d], V[t * E + j * dk + d], acc);
        dA[jt] = acc;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < heads; j += blockDim.x) {
        float acc = 0.f;
        for (int t = 0; t < T; ++t)
            acc = fmaf(A[j * T + t], dA[j * T + t], acc);
        r[j] = acc;
    }
    __syncthreads();
    for (int te = threadIdx.x; te < T * E; te += blockDim.x) {
        const int t = te / E, e = te - t * E, j = e / dk;
        const float a = A[j * T + t];
        const float ds = a * (dA[j * T + t] - r[j]) * scale;
        dV[static_cast<int64_t>(hb) * T * E + te] = a * dO[e];
        dK[static_cast<int64_t>(hb) * T * E + te] = ds * q[e];
    }
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const int j = e / dk;
        float acc = 0.f;
        for (int t = 0; t < T; ++t) {
            const float a = A[j * T + t];
            acc = fmaf(a * (dA[j * T + t] - r[j]) * scale, K[t * E + e], acc);
        }
        dQ[static_cast<int64_t>(hb) * E + e] = acc;
    }
}

// out[r][c] = sum_i X[i][r] Y[i][c] over i in order (one thread per (r, c))
__global__ void wgrad_kernel(const float *X, const float *Y, int64_t N, int R, int C, float *out)
{
    const int64_t rc = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (rc >= static_cast<int64_t>(R) * C)
        return;
    const int r = static_cast<int>(rc / C), c = static_cast<int>(rc - static_cast<int64_t>(r) * C);
    float acc = 0.f;
    for (int64_t i = 0; i < N; ++i)
        acc = fmaf(X[i * R + r], Y[i * C + c], acc);
    out[rc] = acc;
}

unsigned blocks(int64_t items, int per)
{
    return static_cast<unsigned>((items + per - 1) / per);
}

template <typename T>
T *falloc(size_t count, cudaError_t &e)
{
    T *p = nullptr;
    if (e == cudaSuccess)
        e = cudaMalloc(reinterpret_cast<void **>(&p), std::max<size_t>(count, 1) * sizeof(T));
    return p;
}

}  // namespace

Fusion *fusion_create(int H, int T, int dU, int heads, int dk, int dp, const float *P, const float *U,
                      const float *WQ, const float *WK, const float *WV, const float *WO, cudaError_t &e)
{
    Fusion *f = new (std::nothrow) Fusion();
    if (!f) {
        e = cudaErrorMemoryAllocation;
        return nullptr;
    }
    f->H = H;
    f->T = T;
    f->dU = dU;
    f->heads = heads;
    f->dk = dk;
    f->E = heads * dk;
    f->dp = dp;
    const int64_t E = f->E;
    f->n_params = static_cast<int64_t>(dp) * E + 2 * static_cast<int64_t>(dU) * E + E * f->dF;
    f->P = falloc<float>(static_cast<size_t>(H) * dp, e);
    f->U = falloc<float>(static_cast<size_t>(H) * T * dU, e);
    f->params = falloc<float>(f->n_params, e);
    f->grads = falloc<float>(f->n_params, e);
    f->m = falloc<float>(f->n_params, e);
    f->v = falloc<float>(f->n_params, e);
    f->Q = falloc<float>(H * E, e);
    f->K = falloc<float>(static_cast<size_t>(H) * T * E, e);
    f->V = falloc<float>(static_cast<size_t>(H) * T * E, e);
    f->A = falloc<float>(static_cast<size_t>(H) * heads * T, e);
    f->O = falloc<float>(H * E, e);
    f->dQ = falloc<float>(H * E, e);
    f->dK = falloc<float>(static_cast<size_t>(H) * T * E, e);
    f->dV = falloc<float>(static_cast<size_t>(H) * T * E, e);
    f->F = falloc<float>(static_cast<size_t>(H) * f->dF, e);
    f->Eeff = falloc<float>(static_cast<size_t>(H) * f->dF, e);
    auto cp = [&](float *dst, const float *src, int64_t count) {
        if (e == cudaSuccess)
            e = cudaMemcpy(dst, src, count * 4, cudaMemcpyDefault);
    };
    cp(f->P, P, static_cast<int64_t>(H) * dp);
    cp(f->U, U, static_cast<int64_t>(H) * T * dU);
    cp(f->params + f->oWQ(), WQ, static_cast<int64_t>(dp) * E);
    cp(f->params + f->oWK(), WK, dU * E);
    cp(f->params + f->oWV(), WV, dU * E);
    cp(f->params + f->oWO(), WO, E * f->dF);
    if (e == cudaSuccess)
        e = cudaMemset(f->m, 0, f->n_params * 4);
    if (e == cudaSuccess)
        e = cudaMemset(f->v, 0, f->n_params * 4);
    if (e == cudaSuccess)
        e = cudaMemset(f->grads, 0, f->n_params * 4);
    if (e != cudaSuccess) {
        fusion_free(f);
        return nullptr;
    }
    return f;
}

void fusion_free(Fusion *f)
{
    if (!f)
        return;
    for (float *p : {f->P, f->U, f->params, f->grads, f->m, f->v, f->Q, f->K, f->V, f->A, f->O, f->dQ, f->dK, f->dV,
                     f->F, f->Eeff})
        if (p)
            cudaFree(p);
    delete f;
}

ann_status fusion_forward(Fusion *f, const float *E, cudaStream_t s)
{
    const int Ed = f->E;
    const size_t smem = (static_cast<size_t>(f->dp) + f->T * f->dU + Ed + 2 * f->T * Ed + f->heads * f->T + Ed) * 4;
    cudaError_t e = cudaFuncSetAttribute(fusion_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess)
        return cuda_status(e);
    fusion_fwd_kernel<<<f->H, kThreads, smem, s>>>(f->P, f->U, f->params, f->H, f->T, f->dU, f->heads, f->dk, f->dp,
                                                   f->dF, 1.f / sqrtf(static_cast<float>(f->dk)), f->Q, f->K, f->V,
                                                   f->A, f->O, f->F, E, E ? f->Eeff : nullptr);
    return cuda_status(cudaGetLastError());
}

ann_status fusion_backward(Fusion *f, const float *dF, cudaStream_t s)
{
    const int Ed = f->E;
    const size_t smem = (static_cast<size_t>(Ed) + f->heads * f->T + f->heads) * 4;
    fusion_bwd_kernel<<<f->H, kThreads, smem, s>>>(dF, f->params, f->H, f->T, f->dU, f->heads, f->dk, f->dp, f->dF,
                                                   1.f / sqrtf(static_cast<float>(f->dk)), f->Q, f->K, f->V, f->A,
                                                   f->dQ, f->dK, f->dV);
    const int64_t HT = static_cast<int64_t>(f->H) * f->T;
    wgrad_kernel<<<blocks(static_cast<int64_t>(f->dp) * Ed, 128), 128, 0, s>>>(f->P, f->dQ, f->H, f->dp, Ed,
                                                                               f->grads + f->oWQ());
    wgrad_kernel<<<blocks(static_cast<int64_t>(f->dU) * Ed, 128), 128, 0, s>>>(f->U, f->dK, HT, f->dU, Ed,
                                                                               f->grads + f->oWK());
    wgrad_kernel<<<blocks(static_cast<int64_t>(f->dU) * Ed, 128), 128, 0, s>>>(f->U, f->dV, HT, f->dU, Ed,
                                                                               f->grads + f->oWV());
    wgrad_kernel<<<blocks(static_cast<int64_t>(Ed) * f->dF, 128), 128, 0, s>>>(f->O, dF, f->H, Ed, f->dF,
                                                                               f->grads + f->oWO());
    return cuda_status(cudaGetLastError());
}

}  // namespace ann
