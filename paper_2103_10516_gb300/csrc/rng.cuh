// Counter-based Rademacher probes on the device.
//
// Probe id p, row i: z_i = +1 when bit 63 of mix64(((p << 32) | i) ^ seedmix) is
// clear, -1 otherwise, with seedmix = seed * 0x9E3779B97F4A7C15 and mix64 the
// SplitMix64 output finaliser (Steele, Lea, Flood, OOPSLA 2014).  The paper only
// asks for +-1 entries with equal probability (Section 2.1); a counter-based
// generator lets any kernel produce any entry without stored state.
#pragma once

#include <cstdint>

namespace mlt {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t splitmix_finalise(uint64_t x)
{
    x ^= x >> 30;
    x *= 0xBF58476D1CE4E5B9ull;
    x ^= x >> 27;
    x *= 0x94D049BB133111EBull;
    x ^= x >> 31;
    return x;
}

// true when z_i of probe p is -1
__host__ __device__ __forceinline__ bool probe_negative(uint64_t seedmix, uint64_t p, uint64_t i)
{
    const uint64_t key = (p << 32) | (i & 0xFFFFFFFFull);
    return (splitmix_finalise(key ^ seedmix) >> 63) != 0;
}

}  // namespace mlt
