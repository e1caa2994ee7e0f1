// FP16 / BF16 storage of K: two entries packed into one 32-bit word, and the value an entry
// takes once stored (round to nearest even), for the kernels that write half-precision K.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

namespace popcorn {
namespace hstore {

template <typename TH>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
    static_assert(std::is_same<TH, __half>::value || std::is_same<TH, __nv_bfloat16>::value, "FP16 or BF16");
    if constexpr (std::is_same<TH, __half>::value) {
        const __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<const uint32_t*>(&h);
    } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<const uint32_t*>(&h);
    }
}

template <typename TH>
__device__ __forceinline__ float round_trip(float a) {
    if constexpr (std::is_same<TH, __half>::value) return __half2float(__float2half_rn(a));
    else return __bfloat162float(__float2bfloat16_rn(a));
}

}  // namespace hstore
}  // namespace popcorn
