// Checkerboard Metropolis kernels for int8 Ising-type lattices (Weigel, Sec. 3,
// Eq. 1-2; Sec. 4 for 3D and +-J couplings).
//
//   k_init_hot        hot start from Philox (purpose 1, most significant plane).
//   k_observables     full reduction of E (Eq. 1) and M.
//   k_sweep_generic   one colour of a sweep in place in global memory; a thread
//                     owns one group of 32 same-colour sites.  Any even extents,
//                     optional +-J bonds.  Two launches per sweep realise the
//                     order colour 0, then colour 1.
// The streaming sweep (both colours in one pass) is in stream.cu.
//
// Bit-sliced Metropolis: bit i of a 32-bit word is one site (1 = spin -1).
// The anti-aligned neighbours of 32 sites are counted with a handful of logic
// operations; every site then belongs to one class q = dE/4 and is accepted iff
// dE <= 0 or u < thr(q).  The 32-bit u of a site is stored across 32 Philox
// planes, most significant first (bit 31 - p of u = lane bit of plane p), so the
// comparison of all 32 sites runs plane by plane and stops as soon as every
// site is decided; planes are drawn four at a time (one Philox call).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>

#include "philox.cuh"
#include "spn_internal.h"
#include "sweep_common.cuh"

namespace spn {

uint64_t boltzmann_threshold(double beta, int dE) {
  if (dE <= 0) return (uint64_t)1 << 32;
  const double a = beta * (double)dE;
  const double x = std::exp(-a) * 4294967296.0;
  return (uint64_t)std::floor(x);
}

DevThr make_thresholds(double beta) {
  DevThr T{};
  for (int q = 1; q < 4; ++q) {
    const uint64_t t = boltzmann_threshold(beta, 4 * q);
    if (t >= ((uint64_t)1 << 32)) {
      T.always |= 1u << q;
      T.t[q] = 0xffffffffu;
    } else {
      T.t[q] = (uint32_t)t;
    }
  }
  return T;
}

namespace {
std::atomic<uint64_t> g_launches{0};
}
void count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
uint64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

int device_sm_count() {
  static const int sms = [] {  // initialised once, safe from several host threads
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
  }();
  return sms;
}

// ---------------------------------------------------------------- init / E, M

// Hot start: one thread per group (row r, 64-site word j, colour c); site
// x = 64 j + 2 i + par of the group takes bit i of plane 0 of its group.
__global__ void k_init_hot(int8_t* __restrict__ s, int Lx, int Ly, int64_t nrow, PhiloxKeys K, uint32_t stream_id) {
  const int W = (Lx + 63) >> 6;
  const int64_t total = 2 * nrow * W;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t & 1);
    const int64_t g = t >> 1;  // j + W r
    const int64_t r = g / W;
    const int j = (int)(g - r * W);
    const int par = (int)((c + r % Ly + r / Ly) & 1);
    const uint32_t plane0 = philox10((uint32_t)(8 * g), 0u, (uint32_t)c | (kInit << 1), stream_id, K).x;
    int8_t* row = s + r * Lx;
    for (int i = 0; i < 32; ++i) {
      const int x = 64 * j + 2 * i + par;
      if (x >= Lx) break;
      row[x] = ((plane0 >> i) & 1u) ? (int8_t)-1 : (int8_t)1;
    }
  }
}

__device__ __forceinline__ int bond_sign(const uint8_t* __restrict__ bonds, int64_t n, int d) {
  return (bonds && ((bonds[n] >> d) & 1)) ? -1 : 1;
}

__global__ void k_observables(const int8_t* __restrict__ s, const uint8_t* __restrict__ bonds, int nd, int Lx,
                              int Ly, int Lz, int64_t N, unsigned long long* out2, int* bad) {
  long long e = 0, m = 0;
  int invalid = 0;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(n % Lx);
    const int64_t r = n / Lx;
    const int y = (int)(r % Ly);
    const int z = (int)(r / Ly);
    const int sn = s[n];
    invalid |= (sn != 1 && sn != -1);
    m += sn;
    const int64_t nx = n - x + (x + 1 == Lx ? 0 : x + 1);
    const int64_t ny = n + (int64_t)((y + 1 == Ly ? 0 : y + 1) - y) * Lx;
    e -= (long long)bond_sign(bonds, n, 0) * sn * s[nx];
    e -= (long long)bond_sign(bonds, n, 1) * sn * s[ny];
    if (nd == 3) {
      const int64_t nz = n + (int64_t)((z + 1 == Lz ? 0 : z + 1) - z) * Lx * Ly;
      e -= (long long)bond_sign(bonds, n, 2) * sn * s[nz];
    }
  }
  if (invalid && bad) atomicExch(bad, 1);
  block_accumulate(e, m, out2);
}

cudaError_t launch_init_hot(const Lattice& g, int8_t* s, uint64_t seed, uint32_t stream_id, cudaStream_t st) {
  const int64_t nrow = g.N / g.Lx;
  const int64_t work = 2 * nrow * ((g.Lx + 63) / 64);
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((work + threads - 1) / threads, (int64_t)device_sm_count() * 32);
  k_init_hot<<<(unsigned)std::max<int64_t>(blocks, 1), threads, 0, st>>>(s, g.Lx, g.Ly, nrow, philox_keys(seed),
                                                                         stream_id);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_observables(const Lattice& g, const int8_t* s, unsigned long long* out2, int* bad,
                               cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out2, 0, 2 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((g.N + threads - 1) / threads, (int64_t)device_sm_count() * 16);
  k_observables<<<(unsigned)std::max<int64_t>(blocks, 1), threads, 0, st>>>(s, g.bonds, g.nd, g.Lx, g.Ly, g.Lz,
                                                                           g.N, out2, bad);
  count_launches(1);
  return cudaGetLastError();
}

// ------------------------------------------------------------ generic sweep

// One colour c of sweep `sweep`, in place: a thread owns the sites of colour c
// in one 64-site word of one row (group g = j + ceil(Lx/64) r, up to 32 sites).
template <int ND>
__global__ void k_sweep_generic(int8_t* __restrict__ s, const uint8_t* __restrict__ bonds, int Lx, int Ly, int Lz,
                                int64_t nrow, int c, DevThr T, PhiloxKeys K, uint32_t stream_id, uint32_t sweep,
                                unsigned long long* acc) {
  const int W = (Lx + 63) >> 6;
  const int64_t ngroups = nrow * W;
  const int64_t LxLy = (int64_t)Lx * Ly;
  int de = 0, dm = 0;
  // warp-uniform trip count: the decision votes across the warp
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31);
  for (int64_t g0 = base; g0 < ngroups; g0 += stride) {
    const int64_t g = g0 + (threadIdx.x & 31);
    uint32_t bits = 0, s0 = 0, s1 = 0, s2 = 0, valid = 0;
    int64_t rowbase = 0;
    int j = 0, par = 0;
    if (g < ngroups) {
      const int64_t r = g / W;
      j = (int)(g - r * W);
      const int y = (int)(r % Ly), z = (int)(r / Ly);
      par = (c + y + z) & 1;
      rowbase = r * Lx;
      const int64_t dym = (int64_t)((y == 0 ? Ly - 1 : y - 1) - y) * Lx;
      const int64_t dyp = (int64_t)((y + 1 == Ly ? 0 : y + 1) - y) * Lx;
      const int64_t dzm = (int64_t)((z == 0 ? Lz - 1 : z - 1) - z) * LxLy;
      const int64_t dzp = (int64_t)((z + 1 == Lz ? 0 : z + 1) - z) * LxLy;
      for (int i = 0; i < 32; ++i) {
        const int x = 64 * j + 2 * i + par;
        if (x >= Lx) break;
        const int64_t n = rowbase + x;
        const int sn = s[n];
        const int64_t xm = rowbase + (x == 0 ? Lx - 1 : x - 1), xp = rowbase + (x + 1 == Lx ? 0 : x + 1);
        const int64_t ym = n + dym, yp = n + dyp;
        int h = bond_sign(bonds, n, 0) * s[xp] + bond_sign(bonds, xm, 0) * s[xm] +
                bond_sign(bonds, n, 1) * s[yp] + bond_sign(bonds, ym, 1) * s[ym];
        if (ND == 3) {
          const int64_t zm = n + dzm, zp = n + dzp;
          h += bond_sign(bonds, n, 2) * s[zp] + bond_sign(bonds, zm, 2) * s[zm];
        }
        const int k = (2 * ND - sn * h) / 2;  // anti-aligned (unsatisfied) bonds
        const uint32_t bit = 1u << i;
        valid |= bit;
        bits |= sn < 0 ? bit : 0u;
        s0 |= (k & 1) ? bit : 0u;
        s1 |= (k & 2) ? bit : 0u;
        s2 |= (k & 4) ? bit : 0u;
      }
    }
    const uint32_t flips = decide_word<ND>(bits, s0, s1, s2, valid, T, K, (uint32_t)(8 * g), sweep,
                                           (uint32_t)c | (kMetropolis << 1), stream_id, de, dm);
    if (flips) {
      for (int i = 0; i < 32; ++i) {
        if ((flips >> i) & 1u) {
          const int64_t n = rowbase + 64 * j + 2 * i + par;
          s[n] = (int8_t)(-s[n]);
        }
      }
    }
  }
  block_accumulate(de, dm, acc);
}

cudaError_t launch_sweep_generic(const Lattice& g, int8_t* s, const DevThr& T, const PhiloxKeys& K,
                                 uint32_t stream_id, uint32_t sweep, unsigned long long* acc, cudaStream_t st) {
  const int64_t nrow = g.N / g.Lx;
  const int64_t ngroups = nrow * ((g.Lx + 63) / 64);
  const int threads = 128;
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((ngroups + threads - 1) / threads,
                                                                (int64_t)device_sm_count() * 16));
  for (int c = 0; c < 2; ++c) {
    if (g.nd == 3)
      k_sweep_generic<3><<<(unsigned)blocks, threads, 0, st>>>(s, g.bonds, g.Lx, g.Ly, g.Lz, nrow, c, T, K,
                                                               stream_id, sweep, acc);
    else
      k_sweep_generic<2><<<(unsigned)blocks, threads, 0, st>>>(s, g.bonds, g.Lx, g.Ly, g.Lz, nrow, c, T, K,
                                                               stream_id, sweep, acc);
  }
  count_launches(2);
  return cudaGetLastError();
}

}  // namespace spn
