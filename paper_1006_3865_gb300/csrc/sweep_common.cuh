// Device building blocks shared by the sweep kernels: warp reductions, the
// bit-sliced neighbour counts and Metropolis decisions over 32-site words, and
// the bulk-copy / mbarrier helpers of the shared-memory pipelines.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "philox.cuh"
#include "spn_internal.h"

namespace spn {

// ------------------------------------------------------------------ helpers

static __device__ __forceinline__ void warp_reduce_add2(long long& a, long long& b) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
}

// Block-wide sum of (a, b), one atomic pair per warp.
static __device__ __forceinline__ void block_accumulate(long long a, long long b, unsigned long long* out2) {
  warp_reduce_add2(a, b);
  if ((threadIdx.x & 31) == 0 && (a | b)) {
    atomicAdd(out2 + 0, (unsigned long long)a);
    atomicAdd(out2 + 1, (unsigned long long)b);
  }
}

// Metropolis decision for 32 sites.  cls[q-1]: sites whose move has dE = 4q > 0;
// acc: sites already accepted (dE <= 0).  Plane p of the group (counter c0 + p/4)
// holds bit 31 - p of every site's u; a site of class q is accepted iff
// u < T.t[q] (or T.always has bit q).  Planes are compared from the most
// significant down until no site is undecided anywhere in the warp.  Must be
// called by all 32 lanes of a warp together.
template <int NC>
__device__ __forceinline__ uint32_t lazy_accept(uint32_t acc, const uint32_t (&cls)[NC], const DevThr& T,
                                                const PhiloxKeys& K, uint32_t c0, uint32_t sweep, uint32_t c2,
                                                uint32_t stream_id) {
  uint32_t eq[NC];
  uint32_t pend = 0;
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    const bool always = (T.always >> (q + 1)) & 1u;
    acc |= always ? cls[q] : 0u;
    eq[q] = always ? 0u : cls[q];
    pend |= eq[q];
  }
#pragma unroll 1
  for (uint32_t call = 0; call < 8u && __any_sync(0xffffffffu, pend != 0u); ++call) {
    const U4 P = philox10(c0 + call, sweep, c2, stream_id, K);
    const uint32_t planes[4] = {P.x, P.y, P.z, P.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t u = planes[j];
      const uint32_t bit = 31u - (4u * call + (uint32_t)j);
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        if ((T.t[q + 1] >> bit) & 1u) {  // threshold bit 1: a 0 bit of u decides "below"
          acc |= eq[q] & ~u;
          eq[q] &= u;
        } else {
          eq[q] &= ~u;
        }
      }
    }
    pend = 0;
#pragma unroll
    for (int q = 0; q < NC; ++q) pend |= eq[q];
  }
  return acc;
}

// u < t on the top NP bit planes for all 32 sites of a word at once, with t
// the threshold of each site's own class (the class masks eq[k] are disjoint,
// so one selected threshold plane serves every class).  Least significant
// plane first: below' = maj(~u_p, t_p, below); equal keeps the sites whose NP
// bits all match.  tm[k][p] is 0 / ~0 for bit 31 - p of class k's threshold.
// The sites found below join acc; eq keeps only the sites still tied.
template <int NC, int NP>
__device__ __forceinline__ void compare_top(uint32_t& acc, uint32_t (&eq)[NC], const uint32_t (&pl)[NP],
                                            const uint32_t (*tm)[32]) {
  uint32_t below = 0, equal = 0xffffffffu;
#pragma unroll
  for (int p = NP - 1; p >= 0; --p) {
    uint32_t t = tm[0][p];
#pragma unroll
    for (int k = 1; k < NC; ++k) t = (eq[k] & tm[k][p]) | (~eq[k] & t);
    const uint32_t nu = ~pl[p];
    below = (nu & t) | (nu & below) | (t & below);
    equal &= ~(pl[p] ^ t);
  }
  uint32_t any = 0;
#pragma unroll
  for (int k = 0; k < NC; ++k) any |= eq[k];
  acc |= any & below;
#pragma unroll
  for (int k = 0; k < NC; ++k) eq[k] &= equal;
}

// Classes of one 32-site word from the anti-aligned counts k = s0 + 2 s1 + 4 s2
// out of 2*ND neighbours: cls[q-1] = sites with dE = 4q > 0; returns the sites
// with dE <= 0 (always accepted).
template <int ND>
__device__ __forceinline__ uint32_t classes(uint32_t s0, uint32_t s1, uint32_t s2, uint32_t valid,
                                            uint32_t (&cls)[ND]) {
  if constexpr (ND == 2) {
    const uint32_t hi = s1 | s2;  // k >= 2
    cls[0] = s0 & ~hi & valid;    // k = 1, dE = 4
    cls[1] = ~s0 & ~hi & valid;   // k = 0, dE = 8
    return hi & valid;
  } else {
    cls[0] = ~s0 & s1 & ~s2 & valid;  // k = 2, dE = 4
    cls[1] = s0 & ~s1 & ~s2 & valid;  // k = 1, dE = 8
    cls[2] = ~s0 & ~s1 & ~s2 & valid;  // k = 0, dE = 12
    return (s2 | (s0 & s1)) & valid;   // k >= 3
  }
}

// dE = sum 4 (ND - k) and dM = sum -2 s over the accepted sites of a word.
template <int ND>
__device__ __forceinline__ void tally(uint32_t acc, uint32_t b, uint32_t s0, uint32_t s1, uint32_t s2, int& de,
                                      int& dm) {
  const int nf = __popc(acc);
  de += 4 * (ND * nf - (__popc(acc & s0) + 2 * __popc(acc & s1) + 4 * __popc(acc & s2)));
  dm += 2 * (2 * __popc(acc & b) - nf);
}

// Bit-sliced count of anti-aligned neighbours: inputs are the neighbour words
// XOR-ed with the centre (1 = anti-aligned); output k = s0 + 2 s1 + 4 s2.
static __device__ __forceinline__ void count4(uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint32_t& s0, uint32_t& s1,
                                       uint32_t& s2) {
  const uint32_t h1 = a ^ b, c1 = a & b, h2 = c ^ d, c2 = c & d;
  const uint32_t c3 = h1 & h2;
  s0 = h1 ^ h2;
  s1 = c1 ^ c2 ^ c3;
  s2 = c1 & c2;
}

static __device__ __forceinline__ void count6(uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint32_t e, uint32_t f,
                                       uint32_t& s0, uint32_t& s1, uint32_t& s2) {
  const uint32_t x1 = a ^ b ^ c, y1 = (a & b) | (c & (a ^ b));
  const uint32_t x2 = d ^ e ^ f, y2 = (d & e) | (f & (d ^ e));
  s0 = x1 ^ x2;
  const uint32_t cc = x1 & x2;
  s1 = y1 ^ y2 ^ cc;
  s2 = (y1 & y2) | (cc & (y1 ^ y2));
}

// Classes and decision for one 32-site word: b = spin bits, k = (s0, s1, s2)
// anti-aligned counts out of 2*ND neighbours, valid = sites present.  Returns
// the accepted sites; adds dE = sum 4 (ND - k) and dM = sum -2 s of the flips.
template <int ND>
__device__ __forceinline__ uint32_t decide_word(uint32_t b, uint32_t s0, uint32_t s1, uint32_t s2, uint32_t valid,
                                                const DevThr& T, const PhiloxKeys& K, uint32_t c0, uint32_t sweep,
                                                uint32_t c2, uint32_t stream_id, int& de, int& dm) {
  uint32_t acc, cls[ND];
  if constexpr (ND == 2) {
    // k = 0 -> dE = 8 (class 2), k = 1 -> dE = 4 (class 1), k >= 2 -> dE <= 0
    const uint32_t hi = s1 | s2;
    cls[0] = s0 & ~hi & valid;
    cls[1] = ~s0 & ~hi & valid;
    acc = hi & valid;
  } else {
    // k = 0 -> class 3, 1 -> class 2, 2 -> class 1, k >= 3 -> dE <= 0
    cls[0] = ~s0 & s1 & ~s2 & valid;
    cls[1] = s0 & ~s1 & ~s2 & valid;
    cls[2] = ~s0 & ~s1 & ~s2 & valid;
    acc = (s2 | (s0 & s1)) & valid;
  }
  acc = lazy_accept<ND>(acc, cls, T, K, c0, sweep, c2, stream_id);
  const int nf = __popc(acc);
  de += 4 * (ND * nf - (__popc(acc & s0) + 2 * __popc(acc & s1) + 4 * __popc(acc & s2)));
  dm += 2 * (2 * __popc(acc & b) - nf);
  return acc;
}


static constexpr unsigned kWaitLimit = 1u << 22;

static __device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

static __device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

static __device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

static __device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bulk asynchronous copy global -> shared (TMA engine, non-tensor form); both
// addresses 16-byte aligned, bytes a multiple of 16.
static __device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

static __device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
static __device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Four int8 spins (0x01 / 0xFF) -> four bits (1 = -1) at bits 0..3 in byte
// order: bit 1 of byte k moves to bit 28 + k in one multiply (no carries).
static __device__ __forceinline__ uint32_t sign_bits4(uint32_t w) { return ((w & 0x02020202u) * 0x08102040u) >> 28; }


// 64 int8 spins (16 little-endian words, 4 consecutive sites each) -> the E word
// (even sites) and O word (odd sites).  Bits 1..7 of a spin byte are its sign,
// so site k of a group of 8 same-parity sites is taken at a distinct bit of x
// and one multiply by two shifts moves the 8 sign bits, in order and without
// carries, into bits 24..31.
static __device__ __forceinline__ uint32_t gather_e(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3) {
  const uint32_t x = (w0 & 0x00020002u) | (w1 & 0x00080008u) | (w2 & 0x00200020u) | (w3 & 0x00800080u);
  return x * ((1u << 23) + (1u << 8));
}
static __device__ __forceinline__ uint32_t gather_o(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3) {
  const uint32_t x = (w0 & 0x02000200u) | (w1 & 0x08000800u) | (w2 & 0x20002000u) | (w3 & 0x80008000u);
  return x * ((1u << 15) + 1u);
}

// Top bytes of four products -> one word, product v in byte v.
static __device__ __forceinline__ uint32_t top_bytes(uint32_t p0, uint32_t p1, uint32_t p2, uint32_t p3) {
  return __byte_perm(__byte_perm(p0, p1, 0x0073), __byte_perm(p2, p3, 0x0073), 0x5410);
}

// Planes 4 first_call .. 31 for the sites still tied after a first decision
// stage (tm[q][p]: 0 / ~0 = bit 31 - p of the class-q threshold); whole warps.
template <int NC>
__device__ __noinline__ uint32_t rest_planes(uint32_t (&eq)[NC], const uint32_t (*tm)[32], const PhiloxKeys& K,
                                             uint32_t c0, uint32_t c1, uint32_t c2, uint32_t stream_id,
                                             uint32_t first_call) {
  uint32_t acc = 0;
#pragma unroll 1
  for (uint32_t call = first_call; call < 8u; ++call) {
    uint32_t pend = 0;
#pragma unroll
    for (int k = 0; k < NC; ++k) pend |= eq[k];
    if (!__any_sync(0xffffffffu, pend != 0u)) break;
    const U4 P = philox10(c0 + call, c1, c2, stream_id, K);
    const uint32_t pl[4] = {P.x, P.y, P.z, P.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t u = pl[j];
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        const uint32_t t = tm[k][4 * call + j];
        acc |= eq[k] & ~u & t;
        eq[k] &= ~(u ^ t);
      }
    }
  }
  return acc;
}


// Philox4x32-10 with the rounds in a loop and the round keys formed as it goes
// (k0 + r * 0x9E3779B9, k1 + r * 0xBB67AE85, as philox_keys): the same words as
// philox10 in a handful of registers, for rarely taken paths.
__device__ __forceinline__ U4 philox10_rolled(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                              uint32_t k1) {
#pragma unroll 1
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c0;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return U4{c0, c1, c2, c3};
}

// The decision for the sites still tied after FIRST first-stage calls (whole
// warps).  The next call, which a warp with a tie nearly always needs alone, is
// inlined with constant plane indices and a rolled Philox (few registers, so
// the hot path does not spill); only a tie left after it (about 2^-16 of a
// class's sites) takes the function call for the planes beyond.
template <int NC, int FIRST>
__device__ __forceinline__ uint32_t tail_planes(uint32_t (&eq)[NC], const uint32_t (*tm)[32], const PhiloxKeys& K,
                                                uint32_t c0, uint32_t c1, uint32_t c2, uint32_t stream_id) {
  uint32_t pend = 0;
#pragma unroll
  for (int k = 0; k < NC; ++k) pend |= eq[k];
  if (!__any_sync(0xffffffffu, pend != 0u)) return 0u;
  const U4 P = philox10_rolled(c0 + (uint32_t)FIRST, c1, c2, stream_id, K.k0[0], K.k1[0]);
  const uint32_t pl[4] = {P.x, P.y, P.z, P.w};
  uint32_t acc = 0;
  pend = 0;
#pragma unroll
  for (int k = 0; k < NC; ++k) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t t = tm[k][4 * FIRST + j];
      acc |= eq[k] & ~pl[j] & t;
      eq[k] &= ~(pl[j] ^ t);
    }
    pend |= eq[k];
  }
  if (__any_sync(0xffffffffu, pend != 0u)) acc |= rest_planes<NC>(eq, tm, K, c0, c1, c2, stream_id, FIRST + 1);
  return acc;
}

}  // namespace spn
