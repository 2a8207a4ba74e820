// Device helpers shared by the tile kernels: the fault bits, the exact
// float64 -> fixed-point conversion and the per-arithmetic traits.
#pragma once

#include <cuda_runtime.h>

#include "fsi_plan.h"

namespace ttfsi {

enum : int { kErrNonFinite = 1, kErrTimeout = 2 };

// ----------------------------------------------------------------------------
// float64 -> fixed point by integer operations only (GB300's float64 units,
// conversions included, run at about 2 per clock per SM; its integer ALUs at
// 64-128).  E is the tile's largest biased exponent, P the headroom:
// V = trunc(v * 2^(P + 1022 - E)), toward zero (an error below one unit,
// 2^-P of the tile's largest |v|; rounding to nearest cost the ALU-bound
// tile kernel 1.2 % of its time for half of that).
// ----------------------------------------------------------------------------
__device__ __forceinline__ long long to_fixed(unsigned long long bits, int E, int P) {
    int e = (int)((bits >> 52) & 0x7ff);
    unsigned long long mant = bits & 0x000FFFFFFFFFFFFFull;
    if (e != 0)
        mant |= (1ull << 52);
    else
        e = 1;
    int sh = 53 - P + (E - e);
    unsigned long long r;
    if (sh <= 0)
        r = mant;  // P = 53 and e = E: exact
    else if (sh >= 64)
        r = 0;
    else
        r = mant >> sh;  // toward zero
    long long x = (long long)r;
    return (bits >> 63) ? -x : x;
}

// to_fixed for a tile whose largest biased exponent E satisfies E >= P + 1
// (and P <= 52), with C = 53 - P + E: the shift C - e is then at least 1,
// and a zero or subnormal input (e = 0) has C >= 54, so it converts to 0
// whether or not the implicit bit is set.  Same results as to_fixed, with no
// branches: the implicit bit is always set, the shift is capped at 54 (any
// shift of at least 53 already gives 0) and the sign is applied as
// (r ^ s) - s.
__device__ __forceinline__ long long to_fixed_big_tile(unsigned long long bits, int C) {
    const unsigned hi = (unsigned)(bits >> 32);
    const int e = (int)((hi >> 20) & 0x7ff);
    const unsigned long long mant = (bits & 0x000FFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = min(C - e, 54);
    const long long r = (long long)(mant >> sh);
    const long long sg = (long long)((int)hi >> 31);
    return (r ^ sg) - sg;
}

template <typename Acc>
struct TileTraits;
template <>
struct TileTraits<long long> {
    using In = unsigned long long;
    static constexpr bool exact = true;
};
template <>
struct TileTraits<double> {
    using In = double;
    static constexpr bool exact = false;
};
template <>
struct TileTraits<float> {
    using In = float;
    static constexpr bool exact = false;
};

}  // namespace ttfsi
