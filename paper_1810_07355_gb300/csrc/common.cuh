// Shared helpers of the onng CUDA library: status reporting, launch checks and
// small device utilities.  Host code sets a thread-local error message that
// onng_last_error() returns.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/onng.h"

namespace onng {

int set_error(int status, const char *fmt, ...);

inline cudaStream_t to_cuda(onng_stream_t s) { return reinterpret_cast<cudaStream_t>(s); }

// Returns ONNG_E_CUDA with the CUDA error text if the last launch failed.
inline int check_launch(const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_error(ONNG_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return ONNG_OK;
}

#define ONNG_CUDA_TRY(call, what)                                                      \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return ::onng::set_error(ONNG_E_CUDA, "%s: %s", what, cudaGetErrorString(e_)); \
    } while (0)

#define ONNG_REQUIRE(cond, status, ...)                     \
    do {                                                    \
        if (!(cond))                                        \
            return ::onng::set_error(status, __VA_ARGS__);  \
    } while (0)

// A named host range around an entry point for timeline tools (NVTX); costs a
// branch when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
#define ONNG_RANGE(name) ::onng::NvtxRange onng_range_(name)

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int num_sms();

// Carves aligned sub-buffers out of a caller workspace.
struct WsCarver {
    char *base;
    size_t used = 0;
    explicit WsCarver(void *p) : base(static_cast<char *>(p)) {}
    template <class T> T *take(size_t count)
    {
        used = align_up(used, 256);
        T *p = reinterpret_cast<T *>(base ? base + used : nullptr);
        used += count * sizeof(T);
        return p;
    }
};

// (distance, id) ordering used everywhere: smaller distance first, then smaller id.
__device__ __forceinline__ bool pair_lt(float da, int ia, float db, int ib)
{
    return da < db || (da == db && ia < ib);
}

// 64-bit sortable key of a non-negative float and an id: (float bits, id).
__device__ __forceinline__ unsigned long long pack_key(float d, int id)
{
    return (static_cast<unsigned long long>(__float_as_uint(d)) << 32) | static_cast<unsigned int>(id);
}

}  // namespace onng
