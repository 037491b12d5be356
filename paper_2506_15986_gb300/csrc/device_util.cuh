// device_util.cuh -- small sm_103a device helpers shared by the libann kernels:
// mbarrier / bulk-copy (TMA) wrappers with bounded waits, warp bitonic sorts on
// 64-bit (distance, id) keys, and order-preserving distance encodings.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace ann {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint64_t kKeyMax = ~0ull;

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ---- mbarrier + cp.async.bulk (TMA engine, non-tensor form) ---------------

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// orders this thread's generic-proxy shared-memory accesses before later
// async-proxy (TMA / tensor core) accesses, and vice versa
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Like mbar_try_wait, but the thread may be suspended for up to `hint_ns`
// nanoseconds waiting for the phase instead of returning at once.
__device__ __forceinline__ bool mbar_try_wait_hint(uint64_t *bar, uint32_t parity, uint32_t hint_ns)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity to complete.  Returns false
// when `max_iters` polls went by without completion (the caller reports a
// timeout instead of spinning forever).  Each poll may sleep up to 1 us, so
// a waiting warp leaves its issue slots to the others.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int max_iters)
{
    for (int i = 0; i < max_iters; ++i)
        if (mbar_try_wait_hint(bar, parity, 1000u))
            return true;
    return false;
}

// One bulk global->shared copy of `bytes` (multiple of 16, both addresses
// 16-byte aligned) that signals `bar` with complete_tx on arrival.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// ---- keys -------------------------------------------------------------------
// A pool entry is one 64-bit key: high word = order-preserving distance bits,
// bits 31..1 = node id, bit 0 = "expanded" flag.  Comparing keys with bit 0
// cleared is the (distance, id) order; ids are < 2^31.

// Order-preserving bits of a float distance.  -0 is folded into +0 first
// (x + 0 rounds -0 to +0 and leaves every other value unchanged), so the two
// zeros are one distance and ties between them go to the smaller id.
__device__ __forceinline__ uint32_t f32_to_ord(float f)
{
    const uint32_t u = __float_as_uint(__fadd_rn(f, 0.0f));
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float ord_to_f32(uint32_t u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__device__ __forceinline__ uint64_t make_key(uint32_t dbits, int32_t id)
{
    return (static_cast<uint64_t>(dbits) << 32) | (static_cast<uint64_t>(static_cast<uint32_t>(id)) << 1);
}

__device__ __forceinline__ int32_t key_id(uint64_t k)
{
    return static_cast<int32_t>((static_cast<uint32_t>(k)) >> 1);
}

__device__ __forceinline__ uint64_t key_plain(uint64_t k) { return k & ~1ull; }

// ---- warp bitonic sorts (ascending) ------------------------------------------

__device__ __forceinline__ uint64_t kmin(uint64_t a, uint64_t b) { return a < b ? a : b; }
__device__ __forceinline__ uint64_t kmax(uint64_t a, uint64_t b) { return a < b ? b : a; }

// 32 keys, one per lane; element index = lane.
__device__ __forceinline__ uint64_t warp_sort32(uint64_t k, int lane)
{
#pragma unroll
    for (int kk = 2; kk <= 32; kk <<= 1) {
#pragma unroll
        for (int j = kk >> 1; j > 0; j >>= 1) {
            uint64_t o = __shfl_xor_sync(kFull, k, j);
            bool lower = (lane & j) == 0;
            bool asc = (lane & kk) == 0;
            k = (lower == asc) ? kmin(k, o) : kmax(k, o);
        }
    }
    return k;
}

// Keys of lanes [0, width) sorted ascending (width a power of two <= 32);
// lanes at or above width exchange only among themselves.  The whole warp
// must call it.
__device__ __forceinline__ uint64_t warp_sort_lanes(uint64_t k, int lane, int width)
{
    for (int kk = 2; kk <= width; kk <<= 1) {
        for (int j = kk >> 1; j > 0; j >>= 1) {
            const uint64_t o = __shfl_xor_sync(kFull, k, j);
            const bool lower = (lane & j) == 0;
            const bool asc = (lane & kk) == 0;
            k = (lower == asc) ? kmin(k, o) : kmax(k, o);
        }
    }
    return k;
}

// 64 keys, two per lane: element lane in k0, element lane+32 in k1.
__device__ __forceinline__ void warp_sort64(uint64_t &k0, uint64_t &k1, int lane)
{
#pragma unroll
    for (int kk = 2; kk <= 64; kk <<= 1) {
#pragma unroll
        for (int j = kk >> 1; j > 0; j >>= 1) {
            if (j == 32) {
                uint64_t lo = kmin(k0, k1), hi = kmax(k0, k1);
                k0 = lo;
                k1 = hi;
            } else {
                uint64_t o0 = __shfl_xor_sync(kFull, k0, j);
                uint64_t o1 = __shfl_xor_sync(kFull, k1, j);
                bool lower = (lane & j) == 0;
                bool asc0 = (lane & kk) == 0;
                bool asc1 = ((lane + 32) & kk) == 0;
                k0 = (lower == asc0) ? kmin(k0, o0) : kmax(k0, o0);
                k1 = (lower == asc1) ? kmin(k1, o1) : kmax(k1, o1);
            }
        }
    }
}

// NPL*32 keys, NPL per lane: element r*32+lane lives in k[r].  NPL is a power of 2.
template <int NPL>
__device__ __forceinline__ void warp_sort_n(uint64_t (&k)[NPL], int lane)
{
    constexpr int N = NPL * 32;
#pragma unroll
    for (int kk = 2; kk <= N; kk <<= 1) {
#pragma unroll
        for (int j = kk >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
                const int rj = j >> 5;
#pragma unroll
                for (int r = 0; r < NPL; ++r) {
                    if ((r & rj) == 0) {
                        const bool asc = ((r * 32 + lane) & kk) == 0;
                        const uint64_t a = k[r], b = k[r | rj];
                        k[r] = asc ? kmin(a, b) : kmax(a, b);
                        k[r | rj] = asc ? kmax(a, b) : kmin(a, b);
                    }
                }
            } else {
#pragma unroll
                for (int r = 0; r < NPL; ++r) {
                    const uint64_t o = __shfl_xor_sync(kFull, k[r], j);
                    const bool lower = (lane & j) == 0;
                    const bool asc = ((r * 32 + lane) & kk) == 0;
                    k[r] = (lower == asc) ? kmin(k[r], o) : kmax(k[r], o);
                }
            }
        }
    }
}

// number of entries of the sorted array a[0..len) whose plain key is < v
__device__ __forceinline__ int count_less(const uint64_t *a, int len, uint64_t v)
{
    int lo = 0, hi = len;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (key_plain(a[mid]) < v)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// number of entries of the sorted array a[0..len) that are < v (full keys)
__device__ __forceinline__ int count_less_raw(const uint64_t *a, int len, uint64_t v)
{
    int lo = 0, hi = len;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < v)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

}  // namespace ann
