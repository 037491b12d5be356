// tc.cuh -- 5th-generation tensor-core (tcgen05) building blocks for sm_103a:
// TMEM allocation, shared-memory matrix descriptors, the kind::f16 MMA with a
// BF16 x BF16 -> FP32 accumulator in TMEM, commit to an mbarrier, and TMEM
// loads for the epilogue.  Operands are staged by the CTA's threads into the
// canonical K-major, no-swizzle layout: 8-row x 16-byte core matrices, stored
// so that 16-byte chunk number c of a tile holds row (c / (8*KG))*8 + c%8 and
// k-chunk (c / 8) % KG, with KG = K_tile / 8.  With that order the leading
// byte offset (next core matrix along K) is 128 B and the stride byte offset
// (next 8 rows) is KG * 128 B.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "device_util.cuh"

namespace ann {

// ---- TMEM -------------------------------------------------------------------

// Allocate `ncols` (power of 2, >= 32) TMEM columns; executed by one whole warp.
// The base address is written to *slot (shared memory).
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// ---- descriptors ------------------------------------------------------------

// Shared-memory matrix descriptor: start address, leading and stride byte
// offsets (all >> 4), descriptor version 1, no swizzle, base offset 0.
__device__ __forceinline__ uint64_t smem_desc(const void *p, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = static_cast<uint64_t>((smem_addr(p) & 0x3FFFFu) >> 4);
    d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
    d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
    d |= static_cast<uint64_t>(1) << 46;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, no negation, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
           (static_cast<uint32_t>(M >> 4) << 24);
}

// D[tmem] (+)= A * B^T for one K=16 slice; issued by a single thread.
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on `bar` once every MMA issued so far by this thread has completed.
__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i)
        v[i] = __uint_as_float(r[i]);
}

// ---- operands -------------------------------------------------------------

enum OpType { OP_F32 = 0, OP_BF16 = 1, OP_U8 = 2 };

// A logical row-major matrix view: element (r, k) = p[map(r) * sr + k * sk],
// r < rows and k < cols (zero outside).  map(r) = rowmap ? rowmap[r] : r.
struct Operand {
    const void *p;
    int type;
    int64_t sr, sk;
    int64_t rows, cols;
    const int32_t *rowmap;
};

__device__ __forceinline__ float op_at(const Operand &o, int64_t rr, int64_t k)
{
    const int64_t off = rr * o.sr + k * o.sk;
    if (o.type == OP_F32)
        return static_cast<const float *>(o.p)[off];
    if (o.type == OP_BF16)
        return __bfloat162float(static_cast<const __nv_bfloat16 *>(o.p)[off]);
    return static_cast<float>(static_cast<const uint8_t *>(o.p)[off]);
}

// 8 consecutive k values of row r as packed BF16 (round to nearest even)
__device__ __forceinline__ uint4 op_load8(const Operand &o, int64_t r, int64_t k)
{
    uint4 out = make_uint4(0u, 0u, 0u, 0u);
    if (r >= o.rows || k >= o.cols)
        return out;
    const int64_t rr = o.rowmap ? o.rowmap[r] : r;
    if (o.sk == 1 && k + 8 <= o.cols) {
        const int64_t off = rr * o.sr + k;
        if (o.type == OP_BF16 && (off & 7) == 0)
            return *reinterpret_cast<const uint4 *>(static_cast<const __nv_bfloat16 *>(o.p) + off);
        if (o.type == OP_F32 && (off & 3) == 0) {
            const float4 a = *reinterpret_cast<const float4 *>(static_cast<const float *>(o.p) + off);
            const float4 b = *reinterpret_cast<const float4 *>(static_cast<const float *>(o.p) + off + 4);
            __nv_bfloat162 h0 = __floats2bfloat162_rn(a.x, a.y), h1 = __floats2bfloat162_rn(a.z, a.w);
            __nv_bfloat162 h2 = __floats2bfloat162_rn(b.x, b.y), h3 = __floats2bfloat162_rn(b.z, b.w);
            out.x = *reinterpret_cast<uint32_t *>(&h0);
            out.y = *reinterpret_cast<uint32_t *>(&h1);
            out.z = *reinterpret_cast<uint32_t *>(&h2);
            out.w = *reinterpret_cast<uint32_t *>(&h3);
            return out;
        }
    }
    float f[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
        f[j] = (k + j < o.cols) ? op_at(o, rr, k + j) : 0.f;
    __nv_bfloat162 h0 = __floats2bfloat162_rn(f[0], f[1]), h1 = __floats2bfloat162_rn(f[2], f[3]);
    __nv_bfloat162 h2 = __floats2bfloat162_rn(f[4], f[5]), h3 = __floats2bfloat162_rn(f[6], f[7]);
    out.x = *reinterpret_cast<uint32_t *>(&h0);
    out.y = *reinterpret_cast<uint32_t *>(&h1);
    out.z = *reinterpret_cast<uint32_t *>(&h2);
    out.w = *reinterpret_cast<uint32_t *>(&h3);
    return out;
}

// Stage rows [r0, r0+ROWS) x k [k0, k0+8*KG) of `o` into a canonical tile.
// In a 128-thread CTA each thread takes chunks threadIdx.x, +128, ... and
// loads up to four of them before storing any, so their global loads are in
// flight together instead of one after another.
template <int ROWS, int KG>
__device__ __forceinline__ void stage_tile(uint8_t *tile, const Operand &o, int64_t r0, int64_t k0)
{
    constexpr int CHUNKS = ROWS * KG;
    if (CHUNKS % 128 == 0 && blockDim.x == 128) {
        constexpr int PER = CHUNKS / 128;
        constexpr int NB = PER < 4 ? PER : 4;
        for (int b0 = 0; b0 < PER; b0 += NB) {
            uint4 v[NB];
#pragma unroll
            for (int i = 0; i < NB; ++i) {
                const int c = (b0 + i) * 128 + static_cast<int>(threadIdx.x);
                v[i] = op_load8(o, r0 + (c / (8 * KG)) * 8 + (c & 7), k0 + ((c >> 3) % KG) * 8);
            }
#pragma unroll
            for (int i = 0; i < NB; ++i)
                *reinterpret_cast<uint4 *>(tile + ((b0 + i) * 128 + threadIdx.x) * 16) = v[i];
        }
        return;
    }
    for (int c = threadIdx.x; c < CHUNKS; c += blockDim.x) {
        const int r = (c / (8 * KG)) * 8 + (c & 7);
        const int kg = (c >> 3) % KG;
        *reinterpret_cast<uint4 *>(tile + c * 16) = op_load8(o, r0 + r, k0 + kg * 8);
    }
}

// byte offset of element (r, k) in a canonical K-major tile with KG k-chunks
__device__ __forceinline__ int canon_off(int r, int k, int KG)
{
    return (r >> 3) * (KG * 128) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

constexpr int kTcWaitIters = 1 << 22;  // polls of up to 1 us each

// Bounded wait of the whole CTA for the MMAs committed to `bar` (phase
// `phase`).  On success the phase flips and true is returned uniformly.  If
// any thread ran out of polls, every thread polls once more (bounded) so that
// MMAs still in flight can drain before the caller frees TMEM, and false is
// returned uniformly.
__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t &phase)
{
    const bool ok = mbar_wait_bounded(bar, phase, kTcWaitIters);
    if (__syncthreads_or(!ok)) {
        mbar_wait_bounded(bar, phase, kTcWaitIters);
        return false;
    }
    phase ^= 1u;
    tc_fence_after();
    return true;
}

// D (TMEM columns [tcol, tcol+BN) of lanes 0..127) = A[r0:r0+128, 0:K] *
// B[c0:c0+BN, 0:K]^T, K in chunks of 64 staged through sA (16 KB) and sB
// (BN*128 B).  Every thread of the 128-thread CTA must call it.  Returns false
// (uniformly) if a bounded wait on the commit barrier ran out.
template <int BN>
__device__ bool tc_gemm_tile(const Operand &A, int64_t r0, const Operand &B, int64_t c0, int64_t K,
                             uint8_t *sA, uint8_t *sB, uint64_t *bar, uint32_t &phase, uint32_t tmem_d)
{
    constexpr uint32_t IDESC = idesc_bf16_f32(128, BN);
    for (int64_t k0 = 0; k0 < K; k0 += 64) {
        stage_tile<128, 8>(sA, A, r0, k0);
        stage_tile<BN, 8>(sB, B, c0, k0);
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                tc_mma(tmem_d, smem_desc(sA + kk * 256, 128, 1024), smem_desc(sB + kk * 256, 128, 1024), IDESC,
                       (k0 > 0 || kk > 0) ? 1u : 0u);
            tc_commit(bar);
        }
        if (!tc_wait(bar, phase))
            return false;
    }
    return true;
}

}  // namespace ann
