// Counter-based Philox4x32-10 for device code (Salmon, Moraes, Dror, Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11).
//
// Each round multiplies counter words 0 and 2 by two odd 32-bit constants
// (high and low halves of the 64-bit products), permutes the words and mixes the
// high halves with the other two words and the round key; the key advances by
// two Weyl increments between rounds.  The round keys depend only on the seed,
// so callers precompute them once (PhiloxKeys) and every draw costs the ten
// rounds alone.
#pragma once
#include <cstdint>

namespace spn {

struct PhiloxKeys {
  uint32_t k0[10];
  uint32_t k1[10];
};

__host__ __device__ inline PhiloxKeys philox_keys(uint64_t seed) {
  PhiloxKeys K;
  uint32_t a = (uint32_t)(seed & 0xffffffffu), b = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    K.k0[r] = a;
    K.k1[r] = b;
    a += 0x9E3779B9u;
    b += 0xBB67AE85u;
  }
  return K;
}

struct U4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                       const PhiloxKeys& K) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c0;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
    c0 = hi1 ^ c1 ^ K.k0[r];
    c1 = lo1;
    c2 = hi0 ^ c3 ^ K.k1[r];
    c3 = lo0;
  }
  return U4{c0, c1, c2, c3};
}

__device__ __forceinline__ uint32_t u4_word(const U4& v, int i) {
  return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// Purposes carried in bits 1.. of the third counter word (bit 0 is the colour).
enum : uint32_t {
  kMetropolis = 0u,  // Metropolis u, stored across 32 bit planes
  kInit = 1u,        // hot start (most significant plane)
  kExchange = 2u,    // replica exchange (full 32-bit words)
};

}  // namespace spn
