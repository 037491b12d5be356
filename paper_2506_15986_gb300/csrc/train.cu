// train.cu -- contrastive training of the two-tower entry model on the GPU
// (Sec. 4.3 Eq. loss; Sec. 5.1: Adam, batch 8,192).
//
// One step on a batch of B training queries with hub label rows (+1 positive,
// -1 negative, 0 unused):
//   forward   q_hat = tower(q) (tower_forward_kernel, saving Z1, A1, |Z2|);
//             e_hat = E / |E|; S = q_hat e_hat^T / tau        (tcgen05 GEMM)
//   loss      per query: -(1/|P|) sum_{v in P} log softmax_{P u N}(S)_v,
//             averaged over queries with |P| > 0               (infonce_kernel)
//   backward  dS = (softmax - 1[P]/|P|) / n_valid; dP = dS / tau
//             dq_hat = dP e_hat, de_hat = dP^T q_hat            (tcgen05 GEMMs)
//             through the normalisations, dZ2 -> dW2 = A1^T dZ2, db2,
//             dZ1 = (dZ2 W2^T) * [Z1 > 0] -> dW1 = X^T dZ1, db1 (tcgen05 GEMMs)
//   update    Adam with bias correction on W1, b1, W2, b2, E     (adam_kernel)
// Every GEMM runs BF16 x BF16 -> FP32 on the tensor cores; operands that a
// GEMM reads K-major from a row-major matrix's columns are transposed into
// BF16 scratch first.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "entry.h"
#include "fusion.h"
#include "internal.h"
#include "tc.cuh"

namespace ann {
namespace {

// hubs a trainer takes: one InfoNCE block holds a row's labels in shared memory
constexpr int kMaxTrainHubs = 65536;

// ---- generic tensor-core GEMM ------------------------------------------------

enum Epi { EPI_STORE = 0, EPI_RELU_MASK = 1 };

struct GemmArgs {
    Operand A, B;      // A: M x K, B: N x K (both read K-major)
    int64_t M, N, K;
    float alpha;            // out = alpha * scale[0] * acc (scale may be null)
    const float *scale;
    int epi;
    const float *aux;       // EPI_RELU_MASK: out *= (aux[r*ldo + c] > 0)
    float *out;
    int64_t ldo;
    int *status;
    int64_t ksplit;         // > 0: blockIdx.z takes K range [z*ksplit, (z+1)*ksplit) and adds into out
};

// the operand seen from column k0 on (k0 a multiple of 64: 16-byte alignment kept)
__device__ __forceinline__ Operand op_from_k(const Operand &o, int64_t k0)
{
    Operand r = o;
    const int es = o.type == OP_F32 ? 4 : (o.type == OP_BF16 ? 2 : 1);
    r.p = static_cast<const uint8_t *>(o.p) + k0 * o.sk * es;
    r.cols = o.cols - k0;
    return r;
}

template <int BN>
__global__ void __launch_bounds__(128) gemm_kernel(const GemmArgs g)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sA = smem;
    uint8_t *sB = smem + 16384;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 16384 + BN * 128);
    uint32_t *slot = reinterpret_cast<uint32_t *>(smem + 16384 + BN * 128 + 8);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r0 = static_cast<int64_t>(blockIdx.x) * 128;
    const int64_t c0 = static_cast<int64_t>(blockIdx.y) * BN;
    const int64_t row = r0 + warp * 32 + lane;
    constexpr uint32_t NCOL = BN < 32 ? 32 : BN;
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    if (warp == 0)
        tmem_alloc(slot, NCOL);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *slot;
    uint32_t phase = 0;
    const int64_t kb = g.ksplit > 0 ? static_cast<int64_t>(blockIdx.z) * g.ksplit : 0;
    const int64_t kl = g.ksplit > 0 ? min(g.ksplit, g.K - kb) : g.K;
    const bool ok = tc_gemm_tile<BN>(kb ? op_from_k(g.A, kb) : g.A, r0, kb ? op_from_k(g.B, kb) : g.B, c0, kl, sA,
                                     sB, bar, phase, tmem);
    if (ok) {
        const float a = g.alpha * (g.scale ? g.scale[0] : 1.f);
        const uint32_t my_lane = tmem + (static_cast<uint32_t>(warp * 32) << 16);
        for (int cc = 0; cc < BN; cc += 32) {
            float v[32];
            tmem_ld32(my_lane + cc, v);
            if (row < g.M) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int64_t col = c0 + cc + j;
                    if (col < g.N) {
                        float x = a * v[j];
                        if (g.epi == EPI_RELU_MASK && !(g.aux[row * g.ldo + col] > 0.f))
                            x = 0.f;
                        if (g.ksplit > 0)
                            atomicAdd(g.out + row * g.ldo + col, x);  // a partial sum over its K range
                        else
                            g.out[row * g.ldo + col] = x;
                    }
                }
            }
        }
    } else if (threadIdx.x == 0) {
        atomicOr(g.status, kStatusTimeoutBit);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, NCOL);
    }
}

template <int BN>
ann_status gemm(const GemmArgs &g, cudaStream_t s)
{
    // at least 100 KB: at most two CTAs, so at most 2 x 256 TMEM columns, per SM
    const int smem = std::max(16384 + BN * 128 + 64, 100 * 1024);
    cudaError_t e = cudaFuncSetAttribute(gemm_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess)
        return cuda_status(e);
    dim3 grid(static_cast<unsigned>((g.M + 127) / 128), static_cast<unsigned>((g.N + BN - 1) / BN));
    // few output tiles over a long reduction: split K over CTAs (linear
    // epilogue only), at least 512 columns each, up to about two CTAs per SM
    GemmArgs h = g;
    h.ksplit = 0;
    const int64_t tiles = static_cast<int64_t>(grid.x) * grid.y;
    if (g.epi == EPI_STORE && tiles < 128 && g.K >= 1024) {
        const int64_t want = std::min<int64_t>(g.K / 512, std::max<int64_t>(1, 256 / tiles));
        if (want > 1) {
            h.ksplit = ((g.K + want - 1) / want + 63) / 64 * 64;
            grid.z = static_cast<unsigned>((g.K + h.ksplit - 1) / h.ksplit);
            // the partial sums add into a zeroed M x N block (rows ldo apart)
            e = cudaMemset2DAsync(g.out, static_cast<size_t>(g.ldo) * 4, 0, static_cast<size_t>(g.N) * 4,
                                  static_cast<size_t>(g.M), s);
            if (e != cudaSuccess)
                return cuda_status(e);
        }
    }
    gemm_kernel<BN><<<grid, 128, smem, s>>>(h);
    return cuda_status(cudaGetLastError());
}

// ---- elementwise / row kernels --------------------------------------------

// dst[c][r] = bf16(src(r, c)) for r < rows, c < cols; src row r read through rowmap
__global__ void transpose_bf16(const Operand src, int64_t rows, int64_t cols, __nv_bfloat16 *dst)
{
    __shared__ float tile[32][33];
    const int64_t r0 = static_cast<int64_t>(blockIdx.y) * 32, c0 = static_cast<int64_t>(blockIdx.x) * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t r = r0 + i, c = c0 + threadIdx.x;
        float v = 0.f;
        if (r < rows && c < cols)
            v = op_at(src, src.rowmap ? src.rowmap[r] : r, c);
        tile[i][threadIdx.x] = v;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t c = c0 + i, r = r0 + threadIdx.x;
        if (r < rows && c < cols)
            dst[c * rows + r] = __float2bfloat16_rn(tile[threadIdx.x][i]);
    }
}

// Sum (or maximum) over the block of one value per thread; every thread gets
// the result.  red holds 32 slots; blockDim.x is a multiple of 32.
template <bool MAX>
__device__ __forceinline__ float block_reduce(float v, float *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float w = __shfl_xor_sync(kFull, v, o);
        v = MAX ? fmaxf(v, w) : v + w;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();  // red is free again
    if (lane == 0)
        red[wid] = v;
    __syncthreads();
    v = lane < nw ? red[lane] : (MAX ? -INFINITY : 0.f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float w = __shfl_xor_sync(kFull, v, o);
        v = MAX ? fmaxf(v, w) : v + w;
    }
    return v;
}

// One block per batch row: masked multi-positive InfoNCE over the labelled
// hubs.  The row's labels come as its M listed hubs (cand, lab); every hub
// not listed is a negative, so the row's H labels are first laid out in
// shared memory (all -1, then the listed ones).  Writes the row loss, a
// validity flag (|P| > 0) and the unscaled gradient softmax_{P u N}(S) -
// 1[P]/|P| (0 outside P u N and on invalid rows).
__global__ void infonce_kernel(const float *S, int64_t B, int H, const int32_t *cand, const int8_t *lab, int M,
                               const int32_t *rowmap, float *dS, float *row_loss, int *valid)
{
    extern __shared__ int8_t lrow[];
    __shared__ float red[32];
    const int64_t r = blockIdx.x;
    const int64_t mr = rowmap ? rowmap[r] : r;
    for (int c = threadIdx.x; c < H; c += blockDim.x)
        lrow[c] = -1;
    __syncthreads();
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        const int32_t h = cand[mr * M + j];
        if (h >= 0 && h < H)
            lrow[h] = lab[mr * M + j];
    }
    __syncthreads();
    const float *s = S + r * H;
    float mx = -INFINITY, np = 0.f;
    for (int c = threadIdx.x; c < H; c += blockDim.x) {
        if (lrow[c] != 0)
            mx = fmaxf(mx, s[c]);
        np += lrow[c] > 0 ? 1.f : 0.f;
    }
    mx = block_reduce<true>(mx, red);
    const int npos = static_cast<int>(block_reduce<false>(np, red));
    float z = 0.f, sp = 0.f;
    for (int c = threadIdx.x; c < H; c += blockDim.x) {
        if (lrow[c] != 0)
            z += expf(s[c] - mx);
        if (lrow[c] > 0)
            sp += s[c];
    }
    z = block_reduce<false>(z, red);
    sp = block_reduce<false>(sp, red);
    const float lse = mx + logf(z);
    const bool ok = npos > 0;
    const float inv_np = ok ? 1.f / static_cast<float>(npos) : 0.f;
    for (int c = threadIdx.x; c < H; c += blockDim.x) {
        float g = 0.f;
        if (ok && lrow[c] != 0)
            g = expf(s[c] - lse) - (lrow[c] > 0 ? inv_np : 0.f);
        dS[r * H + c] = g;
    }
    if (threadIdx.x == 0) {
        row_loss[r] = ok ? -(sp - npos * lse) * inv_np : 0.f;
        valid[r] = ok ? 1 : 0;
    }
}

// loss = mean row loss over valid rows; scale[0] = 1 / (n_valid * tau)
__global__ void finalize_loss_kernel(const float *row_loss, const int *valid, int64_t B, float tau, float *loss,
                                     float *scale)
{
    __shared__ float sl[256];
    __shared__ int sv[256];
    float l = 0.f;
    int v = 0;
    for (int64_t i = threadIdx.x; i < B; i += blockDim.x) {
        l += row_loss[i];
        v += valid[i];
    }
    sl[threadIdx.x] = l;
    sv[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sl[threadIdx.x] += sl[threadIdx.x + o];
            sv[threadIdx.x] += sv[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int nv = sv[0];
        loss[0] = nv > 0 ? sl[0] / nv : 0.f;
        scale[0] = nv > 0 ? 1.f / (nv * tau) : 0.f;
    }
}

// dZ = (dY - Y (Y . dY)) / n per row of width W (gradient of y = z / |z|)
__global__ void norm_backward_kernel(const float *Y, const float *n, const float *dY, int64_t rows, int W,
                                     float *dZ)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
    if (r >= rows)
        return;
    float dot = 0.f;
    for (int c = lane; c < W; c += 32)
        dot = fmaf(Y[r * W + c], dY[r * W + c], dot);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        dot += __shfl_xor_sync(kFull, dot, o);
    const float inv = n[r] > 0.f ? 1.f / n[r] : 0.f;
    for (int c = lane; c < W; c += 32)
        dZ[r * W + c] = (dY[r * W + c] - Y[r * W + c] * dot) * inv;
}

__global__ void colsum_kernel(const float *X, int64_t rows, int cols, float *out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols)
        return;
    float s = 0.f;
    for (int64_t r = 0; r < rows; ++r)
        s += X[r * cols + c];
    out[c] = s;
}

__global__ void row_norms_kernel(const float *E, int64_t rows, int W, float *n)
{
    const int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (r >= rows)
        return;
    float ss = 0.f;
    for (int c = 0; c < W; ++c)
        ss = fmaf(E[r * W + c], E[r * W + c], ss);
    n[r] = sqrtf(ss);
}

// Adam with bias correction (Kingma & Ba), fp32 state
__global__ void adam_kernel(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                            float eps, float bc1, float bc2)
{
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i >= n)
        return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / bc1, vh = vi / bc2;
    p[i] -= lr * mh / (sqrtf(vh) + eps);
}

inline unsigned blocks_for(int64_t n, int per) { return static_cast<unsigned>((n + per - 1) / per); }

}  // namespace
}  // namespace ann

using namespace ann;

// Trainer: parameters (flat fp32: W1 | b1 | W2 | b2 | E), Adam state, and
// per-batch scratch.  The model struct reuses the inference launchers.
struct ann_trainer {
    int device = 0;
    int64_t batch = 0;
    int in_dim = 0, H = 0;
    float tau = 0.07f, lr = 5e-5f, beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
    int64_t step = 0;
    int64_t n_params = 0;
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    ann_entry_model model;  // views into params + BF16 copies
    // scratch
    float *z1 = nullptr, *qhat = nullptr, *nrm = nullptr, *S = nullptr, *dS = nullptr, *row_loss = nullptr;
    float *dQ = nullptr, *dEh = nullptr, *dZ2 = nullptr, *dZ1 = nullptr, *Enrm = nullptr;
    float *loss = nullptr, *scale = nullptr;
    int *valid = nullptr, *status = nullptr;
    __nv_bfloat16 *a1 = nullptr, *qbf = nullptr, *EnT = nullptr, *dST = nullptr, *qT = nullptr, *a1T = nullptr,
                  *dZ2T = nullptr, *xT = nullptr, *dZ1T = nullptr;
    std::vector<void *> owned;
    ann::Fusion *fu = nullptr;  // topology-aware hub tower: hub rows are E + F
};

namespace {

template <typename T>
T *talloc(ann_trainer *t, size_t count, cudaError_t &e)
{
    T *p = nullptr;
    if (e == cudaSuccess) {
        e = cudaMalloc(reinterpret_cast<void **>(&p), std::max<size_t>(count, 1) * sizeof(T));
        if (e == cudaSuccess)
            t->owned.push_back(p);
    }
    return p;
}

void trainer_free(ann_trainer *t)
{
    if (!t)
        return;
    cudaDeviceSynchronize();
    for (void *p : t->owned)
        cudaFree(p);
    fusion_free(t->fu);
    delete t;
}

// one Adam step over every parameter block
void adam_all(ann_trainer *t, cudaStream_t s)
{
    t->step += 1;
    const float bc1 = 1.f - powf(t->beta1, static_cast<float>(t->step));
    const float bc2 = 1.f - powf(t->beta2, static_cast<float>(t->step));
    adam_kernel<<<blocks_for(t->n_params, 256), 256, 0, s>>>(t->params, t->grads, t->m, t->v, t->n_params, t->lr,
                                                             t->beta1, t->beta2, t->eps, bc1, bc2);
    if (t->fu)
        adam_kernel<<<blocks_for(t->fu->n_params, 256), 256, 0, s>>>(t->fu->params, t->fu->grads, t->fu->m,
                                                                     t->fu->v, t->fu->n_params, t->lr, t->beta1,
                                                                     t->beta2, t->eps, bc1, bc2);
}

// offsets of the parameter blocks inside the flat vector
struct Offs {
    int64_t W1, b1, W2, b2, E, total;
};
Offs offsets(int in_dim, int H)
{
    Offs o;
    o.W1 = 0;
    o.b1 = o.W1 + static_cast<int64_t>(in_dim) * 256;
    o.W2 = o.b1 + 256;
    o.b2 = o.W2 + 256 * 64;
    o.E = o.b2 + 64;
    o.total = o.E + static_cast<int64_t>(H) * 64;
    return o;
}

// forward + loss + backward for one batch; grads written to t->grads
ann_status trainer_grads(ann_trainer *t, const float *d_queries, const int32_t *rows, int64_t B,
                         const int32_t *d_cand, const int8_t *d_lab, int n_listed, cudaStream_t s)
{
    ann_entry_model &M = t->model;
    const Offs o = offsets(t->in_dim, t->H);
    const int H = t->H, D = t->in_dim;
    ann_status st = ANN_OK;
    if (t->fu) {
        // the hub rows the model scores: E + F (Eq. fusion)
        if ((st = fusion_forward(t->fu, t->params + o.E, s)) != ANN_OK)
            return st;
        M.E = t->fu->Eeff;
    }
    st = prepare_model(&M, s);
    M.E = t->params + o.E;
    if (st != ANN_OK)
        return st;
    const float *Erows = t->fu ? t->fu->Eeff : M.E;
    row_norms_kernel<<<blocks_for(H, 256), 256, 0, s>>>(Erows, H, 64, t->Enrm);
    const Operand X{d_queries, OP_F32, D, 1, B, D, rows};
    st = launch_tower(&M, X, B, t->qhat, t->qbf, t->z1, t->a1, t->nrm, t->status, s);
    if (st != ANN_OK)
        return st;
    // logits
    GemmArgs g{};
    g.status = t->status;
    g.A = Operand{t->qbf, OP_BF16, 64, 1, B, 64, nullptr};
    g.B = Operand{M.Eb, OP_BF16, 64, 1, H, 64, nullptr};
    g.M = B;
    g.N = H;
    g.K = 64;
    g.alpha = 1.f / t->tau;
    g.out = t->S;
    g.ldo = H;
    if ((st = gemm<128>(g, s)) != ANN_OK)
        return st;
    infonce_kernel<<<static_cast<unsigned>(B), 256, H, s>>>(t->S, B, H, d_cand, d_lab, n_listed, rows, t->dS,
                                                             t->row_loss, t->valid);
    finalize_loss_kernel<<<1, 256, 0, s>>>(t->row_loss, t->valid, B, t->tau, t->loss, t->scale);
    // dq_hat = scale * dS e_hat  (B x 64, K = H)
    transpose_bf16<<<dim3(blocks_for(64, 32), blocks_for(H, 32)), dim3(32, 8), 0, s>>>(
        Operand{M.En, OP_F32, 64, 1, H, 64, nullptr}, H, 64, t->EnT);
    g = GemmArgs{};
    g.status = t->status;
    g.A = Operand{t->dS, OP_F32, H, 1, B, H, nullptr};
    g.B = Operand{t->EnT, OP_BF16, H, 1, 64, H, nullptr};
    g.M = B;
    g.N = 64;
    g.K = H;
    g.alpha = 1.f;
    g.scale = t->scale;
    g.out = t->dQ;
    g.ldo = 64;
    if ((st = gemm<64>(g, s)) != ANN_OK)
        return st;
    // de_hat = scale * dS^T q_hat  (H x 64, K = B)
    transpose_bf16<<<dim3(blocks_for(H, 32), blocks_for(B, 32)), dim3(32, 8), 0, s>>>(
        Operand{t->dS, OP_F32, H, 1, B, H, nullptr}, B, H, t->dST);
    transpose_bf16<<<dim3(blocks_for(64, 32), blocks_for(B, 32)), dim3(32, 8), 0, s>>>(
        Operand{t->qhat, OP_F32, 64, 1, B, 64, nullptr}, B, 64, t->qT);
    g.A = Operand{t->dST, OP_BF16, B, 1, H, B, nullptr};
    g.B = Operand{t->qT, OP_BF16, B, 1, 64, B, nullptr};
    g.M = H;
    g.N = 64;
    g.K = B;
    g.out = t->dEh;
    if ((st = gemm<64>(g, s)) != ANN_OK)
        return st;
    // through the normalisations
    norm_backward_kernel<<<blocks_for(B * 32, 256), 256, 0, s>>>(t->qhat, t->nrm, t->dQ, B, 64, t->dZ2);
    norm_backward_kernel<<<blocks_for(static_cast<int64_t>(H) * 32, 256), 256, 0, s>>>(M.En, t->Enrm, t->dEh, H, 64,
                                                                                      t->grads + o.E);
    // dL/dF = dL/d(E + F) = dL/dE
    if (t->fu && (st = fusion_backward(t->fu, t->grads + o.E, s)) != ANN_OK)
        return st;
    // dW2 = A1^T dZ2 (256 x 64, K = B); db2
    transpose_bf16<<<dim3(blocks_for(256, 32), blocks_for(B, 32)), dim3(32, 8), 0, s>>>(
        Operand{t->a1, OP_BF16, 256, 1, B, 256, nullptr}, B, 256, t->a1T);
    transpose_bf16<<<dim3(blocks_for(64, 32), blocks_for(B, 32)), dim3(32, 8), 0, s>>>(
        Operand{t->dZ2, OP_F32, 64, 1, B, 64, nullptr}, B, 64, t->dZ2T);
    g = GemmArgs{};
    g.status = t->status;
    g.A = Operand{t->a1T, OP_BF16, B, 1, 256, B, nullptr};
    g.B = Operand{t->dZ2T, OP_BF16, B, 1, 64, B, nullptr};
    g.M = 256;
    g.N = 64;
    g.K = B;
    g.alpha = 1.f;
    g.out = t->grads + o.W2;
    g.ldo = 64;
    if ((st = gemm<64>(g, s)) != ANN_OK)
        return st;
    colsum_kernel<<<1, 64, 0, s>>>(t->dZ2, B, 64, t->grads + o.b2);
    // dZ1 = (dZ2 W2^T) * [Z1 > 0]  (B x 256, K = 64): B operand row n = W2[n][:]
    g.A = Operand{t->dZ2, OP_F32, 64, 1, B, 64, nullptr};
    g.B = Operand{M.W2, OP_F32, 64, 1, 256, 64, nullptr};
    g.M = B;
    g.N = 256;
    g.K = 64;
    g.epi = EPI_RELU_MASK;
    g.aux = t->z1;
    g.out = t->dZ1;
    g.ldo = 256;
    if ((st = gemm<256>(g, s)) != ANN_OK)
        return st;
    colsum_kernel<<<1, 256, 0, s>>>(t->dZ1, B, 256, t->grads + o.b1);
    // dW1 = X^T dZ1  (D x 256, K = B)
    transpose_bf16<<<dim3(blocks_for(D, 32), blocks_for(B, 32)), dim3(32, 8), 0, s>>>(X, B, D, t->xT);
    transpose_bf16<<<dim3(blocks_for(256, 32), blocks_for(B, 32)), dim3(32, 8), 0, s>>>(
        Operand{t->dZ1, OP_F32, 256, 1, B, 256, nullptr}, B, 256, t->dZ1T);
    g = GemmArgs{};
    g.status = t->status;
    g.A = Operand{t->xT, OP_BF16, B, 1, D, B, nullptr};
    g.B = Operand{t->dZ1T, OP_BF16, B, 1, 256, B, nullptr};
    g.M = D;
    g.N = 256;
    g.K = B;
    g.alpha = 1.f;
    g.out = t->grads + o.W1;
    g.ldo = 256;
    if ((st = gemm<256>(g, s)) != ANN_OK)
        return st;
    return cuda_status(cudaGetLastError());
}

}  // namespace

extern "C" {

ann_status ann_trainer_create(int device, int32_t in_dim, int32_t n_hubs, const float *W1, const float *b1,
                              const float *W2, const float *b2, const float *hub_emb, int64_t max_batch,
                              float tau, float lr, float beta1, float beta2, float eps, ann_trainer **out)
{
    if (!out || !W1 || !b1 || !W2 || !b2 || !hub_emb || in_dim < 1 || in_dim > 512 || n_hubs < 2 ||
        n_hubs > kMaxTrainHubs ||
        max_batch < 1 || max_batch > (1 << 20) || !(tau > 0.f) || !(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) ||
        !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return ANN_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return ANN_ERR_CUDA;
    cudaSetDevice(device);
    if (cudaFuncSetAttribute(infonce_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, n_hubs) != cudaSuccess)
        return ANN_ERR_CUDA;
    ann_trainer *t = new (std::nothrow) ann_trainer();
    if (!t)
        return ANN_ERR_OOM;
    t->device = device;
    t->batch = max_batch;
    t->in_dim = in_dim;
    t->H = n_hubs;
    t->tau = tau;
    t->lr = lr;
    t->beta1 = beta1;
    t->beta2 = beta2;
    t->eps = eps;
    const Offs o = offsets(in_dim, n_hubs);
    t->n_params = o.total;
    const int64_t B = max_batch, H = n_hubs;
    cudaError_t e = cudaSuccess;
    t->params = talloc<float>(t, o.total, e);
    t->grads = talloc<float>(t, o.total, e);
    t->m = talloc<float>(t, o.total, e);
    t->v = talloc<float>(t, o.total, e);
    t->z1 = talloc<float>(t, B * 256, e);
    t->a1 = talloc<__nv_bfloat16>(t, B * 256, e);
    t->qhat = talloc<float>(t, B * 64, e);
    t->qbf = talloc<__nv_bfloat16>(t, B * 64, e);
    t->nrm = talloc<float>(t, B, e);
    t->S = talloc<float>(t, B * H, e);
    t->dS = talloc<float>(t, B * H, e);
    t->row_loss = talloc<float>(t, B, e);
    t->valid = talloc<int>(t, B, e);
    t->dQ = talloc<float>(t, B * 64, e);
    t->dEh = talloc<float>(t, H * 64, e);
    t->dZ2 = talloc<float>(t, B * 64, e);
    t->dZ1 = talloc<float>(t, B * 256, e);
    t->Enrm = talloc<float>(t, H, e);
    t->loss = talloc<float>(t, 2, e);
    t->scale = talloc<float>(t, 2, e);
    t->status = talloc<int>(t, 4, e);
    t->EnT = talloc<__nv_bfloat16>(t, H * 64, e);
    t->dST = talloc<__nv_bfloat16>(t, B * H, e);
    t->qT = talloc<__nv_bfloat16>(t, B * 64, e);
    t->a1T = talloc<__nv_bfloat16>(t, B * 256, e);
    t->dZ2T = talloc<__nv_bfloat16>(t, B * 64, e);
    t->xT = talloc<__nv_bfloat16>(t, B * in_dim, e);
    t->dZ1T = talloc<__nv_bfloat16>(t, B * 256, e);
    ann_entry_model &M = t->model;
    M.in_dim = in_dim;
    M.H = n_hubs;
    M.W1t = talloc<__nv_bfloat16>(t, static_cast<size_t>(in_dim) * 256, e);
    M.W2t = talloc<__nv_bfloat16>(t, 256 * 64, e);
    M.En = talloc<float>(t, H * 64, e);
    M.Eb = talloc<__nv_bfloat16>(t, H * 64, e);
    if (e == cudaSuccess) {
        M.W1 = t->params + o.W1;
        M.b1 = t->params + o.b1;
        M.W2 = t->params + o.W2;
        M.b2 = t->params + o.b2;
        M.E = t->params + o.E;
        e = cudaMemcpy(M.W1, W1, static_cast<size_t>(in_dim) * 256 * 4, cudaMemcpyDefault);
    }
    if (e == cudaSuccess)
        e = cudaMemcpy(M.b1, b1, 256 * 4, cudaMemcpyDefault);
    if (e == cudaSuccess)
        e = cudaMemcpy(M.W2, W2, 256 * 64 * 4, cudaMemcpyDefault);
    if (e == cudaSuccess)
        e = cudaMemcpy(M.b2, b2, 64 * 4, cudaMemcpyDefault);
    if (e == cudaSuccess)
        e = cudaMemcpy(M.E, hub_emb, static_cast<size_t>(H) * 64 * 4, cudaMemcpyDefault);
    if (e == cudaSuccess)
        e = cudaMemset(t->m, 0, o.total * 4);
    if (e == cudaSuccess)
        e = cudaMemset(t->v, 0, o.total * 4);
    if (e == cudaSuccess)
        e = cudaMemset(t->grads, 0, o.total * 4);
    if (e == cudaSuccess)
        e = cudaMemset(t->status, 0, 16);
    if (e != cudaSuccess) {
        ann_status st = cuda_status(e);
        trainer_free(t);
        return st;
    }
    *out = t;
    return ANN_OK;
}

ann_status ann_trainer_free(ann_trainer *t)
{
    trainer_free(t);
    return ANN_OK;
}

ann_status ann_trainer_step(ann_trainer *t, const float *d_queries, const int32_t *d_rows, int64_t nb,
                            const int32_t *d_cand, const int8_t *d_labels, int32_t M, int32_t apply_update,
                            float *loss_out, void *stream)
{
    if (!t || !d_queries || !d_cand || !d_labels || M < 1 || M > t->H || nb < 1 || nb > t->batch ||
        (reinterpret_cast<uintptr_t>(d_queries) & 15))
        return ANN_ERR_INVALID_ARG;
    cudaSetDevice(t->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ann_status st = trainer_grads(t, d_queries, d_rows, nb, d_cand, d_labels, M, s);
    if (st != ANN_OK)
        return st;
    if (apply_update) {
        adam_all(t, s);
        st = cuda_status(cudaGetLastError());
    }
    if (st == ANN_OK && loss_out) {
        cudaError_t e = cudaMemcpyAsync(loss_out, t->loss, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(s);
        st = cuda_status(e);
    }
    return st;
}

ann_status ann_trainer_get(const ann_trainer *t, float *W1, float *b1, float *W2, float *b2, float *hub_emb,
                           int32_t gradients)
{
    if (!t)
        return ANN_ERR_INVALID_ARG;
    const Offs o = offsets(t->in_dim, t->H);
    const float *src = gradients ? t->grads : t->params;
    cudaError_t e = cudaDeviceSynchronize();
    auto cp = [&](float *dst, int64_t off, int64_t count) {
        if (dst && e == cudaSuccess)
            e = cudaMemcpy(dst, src + off, count * 4, cudaMemcpyDefault);
    };
    cp(W1, o.W1, static_cast<int64_t>(t->in_dim) * 256);
    cp(b1, o.b1, 256);
    cp(W2, o.W2, 256 * 64);
    cp(b2, o.b2, 64);
    if (hub_emb && t->fu && !gradients && e == cudaSuccess) {
        // the hub rows the model scores: E + F with the current weights
        ann_status st = fusion_forward(t->fu, t->params + o.E, nullptr);
        if (st != ANN_OK)
            return st;
        e = cudaMemcpy(hub_emb, t->fu->Eeff, static_cast<size_t>(t->H) * 64 * 4, cudaMemcpyDefault);
    } else {
        cp(hub_emb, o.E, static_cast<int64_t>(t->H) * 64);
    }
    if (e == cudaSuccess) {
        int st = 0;
        e = cudaMemcpy(&st, t->status, 4, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && st)
            return ANN_ERR_TIMEOUT;
    }
    return cuda_status(e);
}

ann_status ann_trainer_fit(ann_trainer *t, const float *d_queries, int64_t nt, const int32_t *d_cand,
                           const int8_t *d_labels, int32_t M, const int32_t *d_order, int32_t epochs,
                           float *d_losses, void *stream)
{
    if (!t || !d_queries || !d_cand || !d_labels || M < 1 || M > t->H || nt < 1 || epochs < 0 ||
        (reinterpret_cast<uintptr_t>(d_queries) & 15))
        return ANN_ERR_INVALID_ARG;
    cudaSetDevice(t->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int32_t *iota = nullptr;
    if (!d_order) {
        std::vector<int32_t> h(nt);
        std::iota(h.begin(), h.end(), 0);
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&iota), nt * 4, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(iota, h.data(), nt * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(s);
        if (e != cudaSuccess)
            return cuda_status(e);
    }
    const int64_t spe = (nt + t->batch - 1) / t->batch;
    ann_status st = ANN_OK;
    for (int ep = 0; ep < epochs && st == ANN_OK; ++ep) {
        const int32_t *ord = d_order ? d_order + static_cast<int64_t>(ep) * nt : iota;
        for (int64_t i = 0; i < spe && st == ANN_OK; ++i) {
            const int64_t nb = std::min<int64_t>(t->batch, nt - i * t->batch);
            st = trainer_grads(t, d_queries, ord + i * t->batch, nb, d_cand, d_labels, M, s);
            if (st != ANN_OK)
                break;
            adam_all(t, s);
            if (d_losses)
                cudaMemcpyAsync(d_losses + ep * spe + i, t->loss, 4, cudaMemcpyDeviceToDevice, s);
            st = cuda_status(cudaGetLastError());
        }
    }
    if (iota)
        cudaFreeAsync(iota, s);
    if (st == ANN_OK)
        st = cuda_status(cudaStreamSynchronize(s));
    return st;
}

ann_status ann_trainer_attach(const ann_trainer *t, ann_index *idx, const int32_t *hub_nodes, int32_t hub_degree,
                              void *stream)
{
    if (!t || !idx || !hub_nodes)
        return ANN_ERR_INVALID_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess)
        return cuda_status(e);
    ann_entry_model_desc d{};
    d.in_dim = t->in_dim;
    d.hidden = 256;
    d.out_dim = 64;
    d.W1 = t->model.W1;
    d.b1 = t->model.b1;
    d.W2 = t->model.W2;
    d.b2 = t->model.b2;
    d.n_hubs = t->H;
    d.hub_nodes = hub_nodes;
    d.hub_emb = t->model.E;
    if (t->fu) {
        ann_status st = fusion_forward(t->fu, t->model.E, nullptr);
        if (st == ANN_OK)
            st = cuda_status(cudaDeviceSynchronize());
        if (st != ANN_OK)
            return st;
        d.hub_emb = t->fu->Eeff;
    }
    d.hub_degree = hub_degree;
    d.hub_graph = nullptr;
    d.hub_entry = -1;
    return ann_set_entry_model(idx, &d, stream);
}

ann_status ann_trainer_set_fusion(ann_trainer *t, const float *d_hub_vecs, const float *d_tokens, int32_t T,
                                  int32_t token_dim, int32_t heads, int32_t head_dim, const float *WQ, const float *WK,
                                  const float *WV, const float *WO)
{
    if (!t || !d_hub_vecs || !d_tokens || !WQ || !WK || !WV || !WO || t->fu || t->step != 0 || T < 1 || T > 64 ||
        token_dim < 1 || token_dim > 64 || heads < 1 || head_dim < 1 || heads * head_dim > 256)
        return ANN_ERR_INVALID_ARG;
    cudaSetDevice(t->device);
    cudaError_t e = cudaSuccess;
    t->fu = fusion_create(t->H, T, token_dim, heads, head_dim, t->in_dim, d_hub_vecs, d_tokens, WQ, WK, WV, WO, e);
    return cuda_status(e);
}

ann_status ann_trainer_get_fusion(const ann_trainer *t, float *WQ, float *WK, float *WV, float *WO, int32_t gradients)
{
    if (!t || !t->fu)
        return ANN_ERR_INVALID_ARG;
    const Fusion *f = t->fu;
    const float *src = gradients ? f->grads : f->params;
    cudaError_t e = cudaDeviceSynchronize();
    auto cp = [&](float *dst, int64_t off, int64_t count) {
        if (dst && e == cudaSuccess)
            e = cudaMemcpy(dst, src + off, count * 4, cudaMemcpyDefault);
    };
    cp(WQ, f->oWQ(), static_cast<int64_t>(f->dp) * f->E);
    cp(WK, f->oWK(), static_cast<int64_t>(f->dU) * f->E);
    cp(WV, f->oWV(), static_cast<int64_t>(f->dU) * f->E);
    cp(WO, f->oWO(), static_cast<int64_t>(f->E) * f->dF);
    return cuda_status(e);
}

ann_status ann_adam_update(float *d_params, const float *d_grads, float *d_m, float *d_v, int64_t n, int64_t step,
                           float lr, float beta1, float beta2, float eps, void *stream)
{
    if (!d_params || !d_grads || !d_m || !d_v || n < 0 || step < 1 || !(lr > 0.f) || !(eps > 0.f))
        return ANN_ERR_INVALID_ARG;
    if (n == 0)
        return ANN_OK;
    const float bc1 = 1.f - powf(beta1, static_cast<float>(step));
    const float bc2 = 1.f - powf(beta2, static_cast<float>(step));
    adam_kernel<<<blocks_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(d_params, d_grads, d_m, d_v, n, lr,
                                                                                     beta1, beta2, eps, bc1, bc2);
    return cuda_status(cudaGetLastError());
}

}  // extern "C"
