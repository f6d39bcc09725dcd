// The paper's double-checkerboard sweep with the generalised multi-hit
// (Sec. 3): the lattice is cut into coarse tiles coloured like a
// checkerboard; one launch takes every tile of one parity, a CTA per tile.  The
// CTA stages its tile plus a one-site boundary layer into shared memory as
// colour-separated bit words, updates the tile's colour-0 sites, then its
// colour-1 sites, `hits` times over, and writes the tile back.  The boundary
// layer belongs to tiles of the other parity, which this launch never writes,
// so tiles of one parity are independent and the update is done in place.
//
// Tiles are Tx x Ty (x Tz) sites with Tx a multiple of 64, so the tile's
// 32-site words are the lattice's own row words: the random planes of a word
// are those of its group (j + ceil(Lx/64) r), drawn with purpose 4 at counter
// sweep * hits + hit.  Decisions use the same bit-sliced adders, 12-plane
// compare and warp-lazy remainder as the streaming sweep.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "philox.cuh"
#include "spn_internal.h"
#include "sweep_common.cuh"

namespace spn {
namespace {

constexpr uint32_t kPurposeDc = 4u;
constexpr int kDcFirstCalls = 3;  // planes 0 .. 11 in the first stage

struct DcArgs {
  int8_t* s;  // dense int8 lattice, updated in place
  int Lx, Ly, Lz;
  int Tx, Ty, Tz;  // tile edges (Tz = 1 in 2D)
  int Bx, By, Bz;  // tiles per axis (each even)
  int parity;      // tile parity of this launch
  int hits;
  uint32_t ctr0;   // sweep * hits
  uint32_t stream_id;
  uint32_t always;
  PhiloxKeys K;
  uint32_t tm[3][32];
  unsigned long long* acc;
};

template <int ND>
__global__ void __launch_bounds__(512) k_sweep_dc(const __grid_constant__ DcArgs a) {
  constexpr int NC = ND;
  extern __shared__ __align__(16) uint32_t smd[];
  const int tid = threadIdx.x, nth = blockDim.x;
  const int Lx = a.Lx, W = Lx >> 6, Wt = a.Tx >> 6;
  const int RW = 2 * (Wt + 2);  // words of a staged row: E[0 .. Wt+1], then O[0 .. Wt+1]
  const int TyH = a.Ty + 2, TzH = (ND == 3) ? a.Tz + 2 : 1;
  uint2* lut = reinterpret_cast<uint2*>(smd);  // 256 entries
  uint32_t* rows = smd + 512;                  // TyH * TzH staged rows

  for (int i = tid; i < 256; i += nth) {
    uint32_t lo = 0, hi = 0;
    for (int k = 0; k < 4; ++k) {
      const uint32_t pair = (((i >> k) & 1) ? 0xffu : 0x01u) | ((((i >> (4 + k)) & 1) ? 0xffu : 0x01u) << 8);
      if (k < 2) lo |= pair << (16 * k); else hi |= pair << (16 * (k - 2));
    }
    lut[i] = make_uint2(lo, hi);
  }

  // tile of this CTA: the blockIdx.x-th tile of parity a.parity
  const int half = a.Bx >> 1;
  int rem = blockIdx.x;
  const int bz = (ND == 3) ? rem / (a.By * half) : 0;
  rem -= bz * a.By * half;
  const int by = rem / half;
  const int bx = 2 * (rem - by * half) + ((by + bz + a.parity) & 1);
  const int x0 = bx * a.Tx, y0 = by * a.Ty, z0 = bz * a.Tz;
  auto wrap = [](int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); };
  auto grow = [&](int ly, int lz) {  // global row index of staged row (ly, lz), halo included
    const int y = wrap(y0 + ly, a.Ly), z = (ND == 3) ? wrap(z0 + lz, a.Lz) : 0;
    return (int64_t)y + (int64_t)a.Ly * z;
  };
  auto srow = [&](int ly, int lz) { return rows + (size_t)((ly + 1) + TyH * ((ND == 3) ? lz + 1 : 0)) * RW; };

  // ---- stage the tile and its boundary layer
  {
    const int words = TyH * TzH * Wt;
    for (int i = tid; i < words; i += nth) {
      const int r = i / Wt, j = i - r * Wt;
      const int ly = r % TyH - 1, lz = (ND == 3) ? r / TyH - 1 : 0;
      const uint4* src = reinterpret_cast<const uint4*>(a.s + grow(ly, lz) * Lx + x0 + 64 * j);
      uint32_t pe[4], po[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const uint4 c = src[v];
        pe[v] = gather_e(c.x, c.y, c.z, c.w);
        po[v] = gather_o(c.x, c.y, c.z, c.w);
      }
      uint32_t* row = srow(ly, lz);
      row[1 + j] = top_bytes(pe[0], pe[1], pe[2], pe[3]);
      row[(Wt + 2) + 1 + j] = top_bytes(po[0], po[1], po[2], po[3]);
    }
    // left (x0 - 1, odd x) and right (x0 + Tx, even x) boundary sites of the interior rows
    const int irows = a.Ty * ((ND == 3) ? a.Tz : 1);
    for (int i = tid; i < irows; i += nth) {
      const int ly = i % a.Ty, lz = (ND == 3) ? i / a.Ty : 0;
      const int8_t* g = a.s + grow(ly, lz) * Lx;
      uint32_t* row = srow(ly, lz);
      row[0] = 0;
      row[Wt + 1] = (g[wrap(x0 + a.Tx, Lx)] < 0) ? 1u : 0u;                   // E word right of the tile: bit 0
      row[Wt + 2] = (g[wrap(x0 - 1, Lx)] < 0) ? 0x80000000u : 0u;             // O word left of the tile: bit 31
      row[2 * Wt + 3] = 0;
    }
  }
  __syncthreads();

  int de = 0, dm = 0;
  const int items = a.Ty * ((ND == 3) ? a.Tz : 1) * Wt;
  const int rounds = (items + nth - 1) / nth;
  for (int h = 0; h < a.hits; ++h) {
    const uint32_t c1 = a.ctr0 + (uint32_t)h;
    for (int c = 0; c < 2; ++c) {
      const uint32_t c2 = (uint32_t)c | (kPurposeDc << 1);
      for (int q = 0; q < rounds; ++q) {  // uniform trip count: the remainder stage votes
        const int it = tid + q * nth;
        const bool live = it < items;
        uint32_t acc = 0, eq[NC], b = 0, s0 = 0, s1 = 0, s2 = 0, c0 = 0;
        uint32_t* wp = nullptr;
#pragma unroll
        for (int k = 0; k < NC; ++k) eq[k] = 0;
        if (live) {
          const int r = it / Wt, j = it - r * Wt;
          const int ly = r % a.Ty, lz = (ND == 3) ? r / a.Ty : 0;
          const int y = y0 + ly, z = z0 + lz;
          const int par = (c + y + z) & 1;  // x0 is even: 0 = E words, 1 = O words
          uint32_t* row = srow(ly, lz);
          const uint32_t* same = row + par * (Wt + 2);
          const uint32_t* other = row + (1 - par) * (Wt + 2);
          wp = row + par * (Wt + 2) + 1 + j;
          b = *wp;
          uint32_t left, right;
          if (par == 0) {  // even x: x + 1 is odd lane i, x - 1 odd lane i - 1 (or the word to the left)
            right = other[1 + j];
            left = __funnelshift_l(other[j], other[1 + j], 1);
          } else {  // odd x: x - 1 is even lane i, x + 1 even lane i + 1 (or the word to the right)
            left = other[1 + j];
            right = __funnelshift_r(other[1 + j], other[2 + j], 1);
          }
          const uint32_t ym = srow(ly - 1, lz)[par * (Wt + 2) + 1 + j];
          const uint32_t yp = srow(ly + 1, lz)[par * (Wt + 2) + 1 + j];
          (void)same;
          if constexpr (ND == 3) {
            const uint32_t zm = srow(ly, lz - 1)[par * (Wt + 2) + 1 + j];
            const uint32_t zp = srow(ly, lz + 1)[par * (Wt + 2) + 1 + j];
            count6(b ^ left, b ^ right, b ^ ym, b ^ yp, b ^ zm, b ^ zp, s0, s1, s2);
          } else {
            count4(b ^ left, b ^ right, b ^ ym, b ^ yp, s0, s1, s2);
          }
          uint32_t cls[NC];
          acc = classes<ND>(s0, s1, s2, 0xffffffffu, cls);
#pragma unroll
          for (int k = 0; k < NC; ++k) {
            const bool always = (a.always >> (k + 1)) & 1u;
            acc |= always ? cls[k] : 0u;
            eq[k] = always ? 0u : cls[k];
          }
          c0 = 8u * ((uint32_t)(x0 / 64 + j) + (uint32_t)W * (uint32_t)((int64_t)y + (int64_t)a.Ly * z));
          uint32_t pl[4 * kDcFirstCalls];
#pragma unroll
          for (int call = 0; call < kDcFirstCalls; ++call) {
            const U4 P = philox10(c0 + (uint32_t)call, c1, c2, a.stream_id, a.K);
            pl[4 * call + 0] = P.x;
            pl[4 * call + 1] = P.y;
            pl[4 * call + 2] = P.z;
            pl[4 * call + 3] = P.w;
          }
          compare_top<NC, 4 * kDcFirstCalls>(acc, eq, pl, a.tm);
        }
        acc |= tail_planes<NC, kDcFirstCalls>(eq, a.tm, a.K, c0, c1, c2, a.stream_id);
        if (live) {
          *wp = b ^ acc;  // only this thread touches this colour-c word in this step
          tally<ND>(acc, b, s0, s1, s2, de, dm);
        }
      }
      __syncthreads();
    }
  }

  // ---- write the tile back
  {
    const int words = a.Ty * ((ND == 3) ? a.Tz : 1) * Wt;
    for (int i = tid; i < words; i += nth) {
      const int r = i / Wt, j = i - r * Wt;
      const int ly = r % a.Ty, lz = (ND == 3) ? r / a.Ty : 0;
      const uint32_t* row = srow(ly, lz);
      const uint32_t E = row[1 + j], O = row[(Wt + 2) + 1 + j];
      const uint32_t X = (E & 0x0f0f0f0fu) | ((O << 4) & 0xf0f0f0f0u);
      const uint32_t Y = ((E >> 4) & 0x0f0f0f0fu) | (O & 0xf0f0f0f0u);
      uint4* dst = reinterpret_cast<uint4*>(a.s + grow(ly, lz) * Lx + x0 + 64 * j);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const uint2 lo = lut[(X >> (8 * v)) & 0xffu];
        const uint2 hi = lut[(Y >> (8 * v)) & 0xffu];
        dst[v] = make_uint4(lo.x, lo.y, hi.x, hi.y);
      }
    }
  }
  block_accumulate(de, dm, a.acc);
}

size_t dc_smem(int nd, int Tx, int Ty, int Tz) {
  const int Wt = Tx / 64;
  return 512 * 4 + (size_t)(Ty + 2) * (nd == 3 ? Tz + 2 : 1) * 2 * (Wt + 2) * 4;
}

}  // namespace

bool dc_supported(const Lattice& g, int Tx, int Ty, int Tz) {
  if (g.bonds || g.pitch) return false;
  if (Tx < 64 || Tx % 64 || Ty < 1 || (g.nd == 3 && Tz < 1)) return false;
  const int ext[3] = {g.Lx, g.Ly, g.Lz}, T[3] = {Tx, Ty, g.nd == 3 ? Tz : 1};
  for (int d = 0; d < g.nd; ++d)
    if (ext[d] % T[d] || (ext[d] / T[d]) % 2) return false;
  return dc_smem(g.nd, Tx, Ty, Tz) <= 200 * 1024;
}

cudaError_t launch_sweep_dc(const Lattice& g, int8_t* s, int Tx, int Ty, int Tz, int hits, const DevThr& T,
                            const PhiloxKeys& K, uint32_t stream_id, uint32_t sweep, unsigned long long* acc,
                            cudaStream_t st) {
  if (!dc_supported(g, Tx, Ty, Tz) || hits < 1) return cudaErrorInvalidValue;
  if (((uintptr_t)s & 15)) return cudaErrorMisalignedAddress;
  DcArgs a;
  a.s = s;
  a.Lx = g.Lx;
  a.Ly = g.Ly;
  a.Lz = g.nd == 3 ? g.Lz : 1;
  a.Tx = Tx;
  a.Ty = Ty;
  a.Tz = g.nd == 3 ? Tz : 1;
  a.Bx = g.Lx / Tx;
  a.By = g.Ly / Ty;
  a.Bz = g.nd == 3 ? g.Lz / Tz : 1;
  a.hits = hits;
  a.ctr0 = sweep * (uint32_t)hits;
  a.stream_id = stream_id;
  a.always = T.always;
  a.K = K;
  for (int k = 0; k < 3; ++k)
    for (int p = 0; p < 32; ++p) a.tm[k][p] = ((T.t[k + 1] >> (31 - p)) & 1u) ? 0xffffffffu : 0u;
  a.acc = acc;
  const size_t smem = dc_smem(g.nd, Tx, Ty, a.Tz);
  const int items = Ty * a.Tz * (Tx / 64);
  const int threads = std::min(512, std::max(64, (items + 31) / 32 * 32));
  const int ctas = a.Bx * a.By * a.Bz / 2;
  static std::mutex mu;
  static size_t set[2] = {0, 0};
  {
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = set[g.nd == 3 ? 1 : 0];
    if (smem > cur) {
      if (g.nd == 3)
        cudaFuncSetAttribute(k_sweep_dc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      else
        cudaFuncSetAttribute(k_sweep_dc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      cur = smem;
    }
  }
  for (int p = 0; p < 2; ++p) {
    a.parity = p;
    if (g.nd == 3)
      k_sweep_dc<3><<<ctas, threads, smem, st>>>(a);
    else
      k_sweep_dc<2><<<ctas, threads, smem, st>>>(a);
  }
  count_launches(2);
  return cudaGetLastError();
}

}  // namespace spn
