// Checkerboard Metropolis kernels for int8 Ising-type lattices (Weigel, Sec. 3,
// Eq. 1-2; Sec. 4 for 3D and +-J couplings).
//
//   k_init_hot        hot start from Philox (purpose 1, most significant plane);
//                     k_init_hot_words for rows of whole 64-site words.
//   k_observables     full reduction of E (Eq. 1) and M; k_observables_chunks
//                     for Ising rows of whole 16-byte chunks.
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

// int8 pattern of 8 sites [e0 o0 e1 o1 e2 o2 e3 o3] for index e | o << 4
// (bit set: spin -1)
__device__ __forceinline__ void fill_pattern_table(uint2* lut) {
  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    uint32_t lo = 0, hi = 0;
    for (int k = 0; k < 4; ++k) {
      const uint32_t pair = (((i >> k) & 1) ? 0xffu : 0x01u) | ((((i >> (4 + k)) & 1) ? 0xffu : 0x01u) << 8);
      if (k < 2) lo |= pair << (16 * k); else hi |= pair << (16 * (k - 2));
    }
    lut[i] = make_uint2(lo, hi);
  }
}

// Hot start of rows of whole 64-site words (the spins of k_init_hot): a thread
// per (row r, word j) draws plane 0 of both colour groups of the word and writes
// its 64 sites with four 16-byte stores.
__global__ void k_init_hot_words(int8_t* __restrict__ s, int Lx, int Ly, uint32_t nword, PhiloxKeys K,
                                 uint32_t stream_id) {
  __shared__ uint2 lut[256];
  fill_pattern_table(lut);
  __syncthreads();
  const uint32_t W = (uint32_t)Lx >> 6;
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < nword; g += gridDim.x * blockDim.x) {
    const uint32_t r = g / W, j = g - r * W;
    const uint32_t z = r / (uint32_t)Ly, y = r - z * (uint32_t)Ly;
    const uint32_t p0 = philox10(8u * g, 0u, 0u | (kInit << 1), stream_id, K).x;
    const uint32_t p1 = philox10(8u * g, 0u, 1u | (kInit << 1), stream_id, K).x;
    // colour c holds the sites of parity (c + y + z) & 1
    const bool c0_even = ((y + z) & 1u) == 0u;
    const uint32_t E = c0_even ? p0 : p1, O = c0_even ? p1 : p0;
    const uint32_t X = (E & 0x0f0f0f0fu) | ((O << 4) & 0xf0f0f0f0u);  // byte v: sites 16v .. 16v + 7
    const uint32_t Y = ((E >> 4) & 0x0f0f0f0fu) | (O & 0xf0f0f0f0u);  // byte v: sites 16v + 8 .. 16v + 15
    uint4* dst = reinterpret_cast<uint4*>(s + (size_t)r * (size_t)Lx + 64u * j);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const uint2 lo = lut[(X >> (8 * v)) & 0xffu];
      const uint2 hi = lut[(Y >> (8 * v)) & 0xffu];
      dst[v] = make_uint4(lo.x, lo.y, hi.x, hi.y);
    }
  }
}

// E and M of an Ising lattice (J = 1) with rows of whole 16-byte chunks: a
// thread per 16 sites compares them with their x + 1, y + 1 (and z + 1)
// neighbours through the sign bits of the int8 spins (+1 = 0x01, -1 = 0xff):
// E = sum over bonds of (2 [unequal] - 1), M = sum of (1 - 2 [negative]).
__global__ void k_observables_chunks(const int8_t* __restrict__ s, int nd, int Lx, int Ly, int Lz, uint32_t nchunk,
                                     unsigned long long* out2, int* bad) {
  const uint32_t C = (uint32_t)Lx >> 4;
  long long e = 0, m = 0;
  bool invalid = false;
  const uint32_t sign = 0x80808080u;
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nchunk; q += gridDim.x * blockDim.x) {
    const uint32_t r = q / C, k = q - r * C;
    const uint32_t z = r / (uint32_t)Ly, y = r - z * (uint32_t)Ly;
    const int8_t* row = s + (size_t)r * (size_t)Lx;
    const uint4 A = *reinterpret_cast<const uint4*>(row + 16u * k);
    const uint32_t next = (uint8_t)row[k + 1u == C ? 0u : 16u * (k + 1u)];  // site after the chunk, periodic in x
    const uint32_t ry = y + 1u == (uint32_t)Ly ? r - y : r + 1u;
    const uint4 B = *reinterpret_cast<const uint4*>(s + (size_t)ry * (size_t)Lx + 16u * k);
    const uint32_t a[5] = {A.x, A.y, A.z, A.w, next};
    const uint32_t b[4] = {B.x, B.y, B.z, B.w};
    uint32_t c[4] = {0u, 0u, 0u, 0u};
    if (nd == 3) {
      const uint32_t plane = (uint32_t)Ly;
      const uint32_t rz = z + 1u == (uint32_t)Lz ? r - z * plane : r + plane;
      const uint4 Cz = *reinterpret_cast<const uint4*>(s + (size_t)rz * (size_t)Lx + 16u * k);
      c[0] = Cz.x;
      c[1] = Cz.y;
      c[2] = Cz.z;
      c[3] = Cz.w;
    }
    int unequal = 0, neg = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint32_t xn = __byte_perm(a[i], a[i + 1], 0x4321);  // sites n + 1 .. n + 4
      unequal += __popc((a[i] ^ xn) & sign) + __popc((a[i] ^ b[i]) & sign);
      if (nd == 3) unequal += __popc((a[i] ^ c[i]) & sign);
      neg += __popc(a[i] & sign);
      invalid |= (__vcmpeq4(a[i], 0x01010101u) | __vcmpeq4(a[i], 0xffffffffu)) != 0xffffffffu;
    }
    e += 2 * unequal - 16 * nd;
    m += 16 - 2 * neg;
  }
  if (invalid && bad) atomicExch(bad, 1);
  block_accumulate(e, m, out2);
}

cudaError_t launch_init_hot(const Lattice& g, int8_t* s, uint64_t seed, uint32_t stream_id, cudaStream_t st) {
  if (g.Lx % 64 == 0 && ((uintptr_t)s & 15) == 0 && g.N / 64 < ((int64_t)1 << 31)) {
    const int64_t nword = g.N / 64;
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((nword + threads - 1) / threads, (int64_t)device_sm_count() * 16);
    k_init_hot_words<<<(unsigned)std::max<int64_t>(blocks, 1), threads, 0, st>>>(s, g.Lx, g.Ly, (uint32_t)nword,
                                                                                philox_keys(seed), stream_id);
    count_launches(1);
    return cudaGetLastError();
  }
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
  if (!g.bonds && g.Lx % 16 == 0 && ((uintptr_t)s & 15) == 0 && g.N / 16 < ((int64_t)1 << 31)) {
    const int64_t nchunk = g.N / 16;
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((nchunk + threads - 1) / threads, (int64_t)device_sm_count() * 16);
    k_observables_chunks<<<(unsigned)std::max<int64_t>(blocks, 1), threads, 0, st>>>(
        s, g.nd, g.Lx, g.Ly, g.Lz, (uint32_t)nchunk, out2, bad);
    count_launches(1);
    return cudaGetLastError();
  }
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
