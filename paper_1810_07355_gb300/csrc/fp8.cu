// FP8 e4m3 copy of a vector set with per-dimension scales, for the FP8 search
// form (no paper counterpart; the paper searches float vectors).
//   scale_j = max_i |x_ij| / 448 in float32 (1 for an all-zero column), so the
//             scaled coordinates x_ij / scale_j fill e4m3's finite range
//   code_ij = e4m3(x_ij / scale_j): nearest finite value, ties to even,
//             magnitudes above 448 saturate (the hardware conversion)
// The search dequantises a coordinate as the float32 product scale_j * e4m3.
#include <cuda_fp8.h>

#include <algorithm>

#include "common.cuh"

namespace onng {
namespace {

// column maxima of |x| as float bits (non-negative floats order like their bits)
__global__ void fp8_colmax_kernel(const float *__restrict__ X, int64_t n, int d, unsigned *__restrict__ mx)
{
    const int j = blockIdx.x * 32 + (threadIdx.x & 31);
    if (j >= d)
        return;
    unsigned m = 0;
    for (int64_t i = blockIdx.y * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < n;
         i += (int64_t)gridDim.y * (blockDim.x >> 5))
        m = max(m, __float_as_uint(fabsf(X[i * d + j])));
    atomicMax(&mx[j], m);
}

__global__ void fp8_scale_kernel(unsigned *__restrict__ mx, int d)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d)
        return;
    const float m = __uint_as_float(mx[j]);
    reinterpret_cast<float *>(mx)[j] = m > 0.f ? __fdiv_rn(m, 448.f) : 1.f;
}

__global__ void fp8_quantize_kernel(const float *__restrict__ X, int64_t count, int d,
                                    const float *__restrict__ scale, uint8_t *__restrict__ out)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x)
        out[e] = __nv_cvt_float_to_fp8(__fdiv_rn(X[e], scale[e % d]), __NV_SATFINITE, __NV_E4M3);
}

}  // namespace
}  // namespace onng

using namespace onng;

extern "C" int onng_to_fp8(const float *X, int64_t n, int32_t d, float *scale, uint8_t *out, onng_stream_t stream)
{
    ONNG_RANGE("onng_to_fp8");
    ONNG_REQUIRE(n >= 0 && d > 0, ONNG_E_INVAL, "onng_to_fp8: bad sizes");
    ONNG_REQUIRE(X && scale && out, ONNG_E_INVAL, "onng_to_fp8: NULL pointer");
    cudaStream_t s = to_cuda(stream);
    unsigned *mx = reinterpret_cast<unsigned *>(scale);
    ONNG_CUDA_TRY(cudaMemsetAsync(mx, 0, sizeof(unsigned) * (size_t)d, s), "onng_to_fp8: clear maxima");
    if (n > 0) {
        const int gy = (int)std::min<int64_t>((n + 7) / 8, std::max(1, num_sms() * 8 / ((d + 31) / 32)));
        fp8_colmax_kernel<<<dim3((unsigned)((d + 31) / 32), (unsigned)std::max(1, gy)), 256, 0, s>>>(X, n, d, mx);
        ONNG_CUDA_TRY(cudaGetLastError(), "onng_to_fp8: column maxima");
    }
    fp8_scale_kernel<<<(unsigned)((d + 255) / 256), 256, 0, s>>>(mx, d);
    ONNG_CUDA_TRY(cudaGetLastError(), "onng_to_fp8: scales");
    const int64_t count = n * (int64_t)d;
    if (count > 0) {
        const int blocks = (int)std::min<int64_t>((count + 255) / 256, (int64_t)num_sms() * 16);
        fp8_quantize_kernel<<<blocks, 256, 0, s>>>(X, count, d, scale, out);
    }
    return check_launch("onng_to_fp8");
}
