// prng.cuh -- the generator of compressed key-switching keys (Sec. 5.3:
// half of a key is uniformly random, so it is regenerated from a short seed
// instead of being read from HBM).
//
// SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014) as a counter-based generator: draw c of seed s is
// mix(s + (c + 1) * gamma), gamma = 0x9E3779B97F4A7C15, with the finaliser
//   z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31.
// Element (j, l, n) of the key half a (digit j, key limb l of the L+k,
// coefficient n, evaluation form) uses draws 16e .. 16e+15 with
// e = (j*(L+k) + l)*N + n: the first draw whose top b bits (b = bit length of
// q_l) are below q_l is the element; if none is (probability < 2^-16 even for
// a prime just above a power of two), the last one's top bits mod q_l.
// Any element can be generated on its own, in any order, on any thread.
#pragma once

#include "common.cuh"

namespace ckks {

constexpr u64 kSplitMixGamma = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ u64 splitmix_finalise(u64 z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// shift = 64 - bit length of q
__device__ __forceinline__ u64 key_a_element(u64 seed, u64 e, u64 q, int shift) {
    u64 z = seed + (16 * e + 1) * kSplitMixGamma;
    u64 v = 0;
#pragma unroll 1
    for (int r = 0; r < 16; r++, z += kSplitMixGamma) {
        v = splitmix_finalise(z) >> shift;
        if (v < q) return v;
    }
    return v % q;
}

}  // namespace ckks
