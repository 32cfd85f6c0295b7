// Error reporting, version, device queries and the bfloat16 conversion entry point.
#include <cuda_bf16.h>
#include <stdarg.h>

#include <algorithm>

#include "common.cuh"

namespace onng {

static thread_local char g_err[512] = "";

int set_error(int status, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return status;
}

int num_sms()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return 1;
    return sms;
}

// bfloat16 round-to-nearest-even of each float32 (NaNs stay NaN).
__global__ void to_bf16_kernel(const float *__restrict__ x, int64_t count, uint16_t *__restrict__ y)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        __nv_bfloat16 b = __float2bfloat16_rn(x[i]);
        y[i] = *reinterpret_cast<uint16_t *>(&b);
    }
}

}  // namespace onng

extern "C" const char *onng_last_error(void) { return onng::g_err; }

extern "C" int onng_version(void) { return 1; }

extern "C" int onng_to_bf16(const float *X, int64_t count, uint16_t *out, onng_stream_t stream)
{
    ONNG_RANGE("onng_to_bf16");
    ONNG_REQUIRE(count >= 0, ONNG_E_INVAL, "onng_to_bf16: negative count");
    if (count == 0)
        return ONNG_OK;
    ONNG_REQUIRE(X && out, ONNG_E_INVAL, "onng_to_bf16: NULL pointer");
    int blocks = (int)std::min<int64_t>((count + 255) / 256, (int64_t)onng::num_sms() * 8);
    onng::to_bf16_kernel<<<blocks, 256, 0, onng::to_cuda(stream)>>>(X, count, out);
    return onng::check_launch("onng_to_bf16");
}
