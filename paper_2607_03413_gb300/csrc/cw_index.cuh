// cw_index.cuh -- index helpers shared by the DSS and solver kernels.
#pragma once
#include <cstdint>

namespace cw {

// 32-bit division by a runtime constant: q = umulhi(x, floor((2^32-1)/d)) is floor(x/d) or one less
// (the deficit x (1/d - m/2^32) stays below x/2^32 < 1), corrected once. Valid for x + d < 2^32.
struct FastDiv {
    uint32_t d, m;
    static FastDiv make(uint32_t d) { return FastDiv{d, 0xFFFFFFFFu / d}; }
    __device__ __forceinline__ uint32_t div(uint32_t x) const
    {
        uint32_t q = __umulhi(x, m);
        if ((q + 1) * d <= x) ++q;
        return q;
    }
};

}  // namespace cw
