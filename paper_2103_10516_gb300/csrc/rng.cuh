// Counter-based Rademacher probes on the device.
//
// One 64-bit hash serves 64 consecutive probe ids at one row: for probe id p
// and row i, with q = p / 64,
//   h   = mix64(((q << 32) | i) ^ seedmix),   seedmix = seed * 0x9E3779B97F4A7C15,
//   z_i = -1 when bit (p mod 64) of h is set, +1 otherwise,
// mix64 the SplitMix64 output finaliser (Steele, Lea, Flood, OOPSLA 2014).
// The paper only asks for +-1 entries with equal probability (Section 2.1); a
// counter-based generator lets any kernel produce any entry without stored
// state, and 64 signs per hash keep sign generation cheap.
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

// The 64 signs of probes 64q .. 64q+63 at row i (bit t set: probe 64q+t is -1).
__host__ __device__ __forceinline__ uint64_t probe_word(uint64_t seedmix, uint64_t q, uint64_t i)
{
    return splitmix_finalise(((q << 32) | (i & 0xFFFFFFFFull)) ^ seedmix);
}

// true when z_i of probe p is -1
__host__ __device__ __forceinline__ bool probe_negative(uint64_t seedmix, uint64_t p, uint64_t i)
{
    return (probe_word(seedmix, p >> 6, i) >> (p & 63)) & 1u;
}

}  // namespace mlt
