// One instantiation of the search kernels (search_kernel.cuh): vector type
// ONNG_INST_T (0 float32, 1 bfloat16, 2 FP8 e4m3), ONNG_INST_V float4 chunks per
// lane and a kept list of 32 ONNG_INST_KR keys at most (1 or 4).  The build
// compiles this file once per triple, in parallel.
#include "search_kernel.cuh"

#if !defined(ONNG_INST_T) || !defined(ONNG_INST_V) || !defined(ONNG_INST_KR)
#error "search_inst.cu is compiled with -DONNG_INST_T=<0|1|2> -DONNG_INST_V=<1|2|4|8> -DONNG_INST_KR=<1|4>"
#endif

namespace onng {
namespace sk {

#if ONNG_INST_T == 0
using InstT = float;
#elif ONNG_INST_T == 1
using InstT = __nv_bfloat16;
#else
using InstT = __nv_fp8_e4m3;
#endif

template <> Launch pick<InstT, ONNG_INST_V, ONNG_INST_KR>()
{
    constexpr size_t sm = sizeof(WarpSmem<Tune<InstT>::hv, Tune<InstT>::ovf>) * kWarpsPerCta;
    return {search_kernel<ONNG_INST_V, InstT, Tune<InstT>::hv, ONNG_INST_KR>, sm};
}

}  // namespace sk
}  // namespace onng
