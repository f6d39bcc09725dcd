// Division by a run-time constant d < 2^31 as a multiply-high and a shift
// (the round-up method of Granlund and Montgomery, PLDI 1994): the setup of
// FastDiv (host, or once per work item on the device) and the device-side quotient.
#pragma once
#include <cstdint>

#include "spn_internal.h"

namespace spn {

__host__ __device__ inline FastDiv fastdiv(uint32_t d) {
  FastDiv f{d, 0, 0};
  if (d <= 1) return f;
  uint32_t l = 0;
  while ((1ull << l) < d) ++l;  // l = ceil(log2 d) >= 1
  f.m = (uint32_t)((((1ull << 32) * ((1ull << l) - d)) / d) + 1);
  f.s = l - 1;
  return f;
}

__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) {
  if (f.d <= 1) return n;
  const uint32_t t = __umulhi(n, f.m);
  return (t + ((n - t) >> 1)) >> f.s;
}


}  // namespace spn
