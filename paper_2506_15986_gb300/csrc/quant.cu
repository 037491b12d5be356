// quant.cu -- int8 storage with one scale per row (the precision line's
// int8 variant of reduced-precision base vectors).  A packed row is a 16-byte
// header (fp32 scale, 12 zero bytes), then the int8 codes, then zero bytes to
// a multiple of 16, so every row still moves as one 16-byte-aligned bulk copy
// and the codes start on a 16-byte boundary.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "internal.h"

namespace ann {
namespace {

// One warp per row: the row maximum of |x| by a warp reduction, then every
// code from an IEEE fp32 division rounded half to even.
__global__ void quantize_i8s_kernel(const float *x, int64_t n, int dim, int rowbytes, uint8_t *rows)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    for (int64_t r = blockIdx.x * static_cast<int64_t>(blockDim.x >> 5) + (threadIdx.x >> 5); r < n; r += warps) {
        const float *xr = x + r * dim;
        float m = 0.f;
        for (int j = lane; j < dim; j += 32)
            m = fmaxf(m, fabsf(xr[j]));
        for (int o = 16; o > 0; o >>= 1)
            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        const float scale = m / 127.f;
        uint8_t *out = rows + r * rowbytes;
        if (lane < 4)
            reinterpret_cast<float *>(out)[lane] = lane == 0 ? scale : 0.f;
        int8_t *codes = reinterpret_cast<int8_t *>(out + 16);
        for (int j = lane; j < rowbytes - 16; j += 32) {
            int c = 0;
            if (j < dim && scale > 0.f)
                c = static_cast<int>(fminf(127.f, fmaxf(-127.f, rintf(xr[j] / scale))));
            codes[j] = static_cast<int8_t>(c);
        }
    }
}

}  // namespace
}  // namespace ann

using namespace ann;

extern "C" {

int32_t ann_i8s_row_bytes(int32_t dim)
{
    return static_cast<int32_t>(row_bytes(ANN_I8S, dim));
}

ann_status ann_quantize_i8s(const float *d_x, int64_t n, int32_t dim, void *d_rows, void *stream)
{
    if (!d_x || !d_rows || n < 0 || dim < 1 || dim % 4 != 0 || row_bytes(ANN_I8S, dim) > 16384 ||
        (reinterpret_cast<uintptr_t>(d_rows) & 15) || (reinterpret_cast<uintptr_t>(d_x) & 3))
        return ANN_ERR_INVALID_ARG;
    if (n == 0)
        return ANN_OK;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t blocks = std::min<int64_t>((n + 7) / 8, static_cast<int64_t>(sms) * 16);
    quantize_i8s_kernel<<<static_cast<unsigned>(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        d_x, n, dim, static_cast<int>(row_bytes(ANN_I8S, dim)), static_cast<uint8_t *>(d_rows));
    return cuda_status(cudaGetLastError());
}

}  // extern "C"
