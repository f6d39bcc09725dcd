// Band-parallel streaming sweep of a large 2D Ising lattice (J = 1): one launch
// is one full sweep in the canonical two-colour order of Sec. 3 (all of colour
// 0, then all of colour 1), each int8 spin read from HBM once and written once.
//
// The lattice is cut into bands of 30 consecutive 64-site words across x and
// segments of rows along y; a warp owns one (band, segment) and walks down its
// rows on its own, with no synchronisation with any other warp:
//
//   * lane i holds word j0 - 1 + i of every row (j0 the band's first word): the
//     30 owned words plus one halo word on each side, brought in as int8 by bulk
//     asynchronous copies (TMA engine) into a private ring of shared-memory
//     slots, completed on the slot's mbarrier;
//   * each lane turns its 64 sites into colour-separated bit words (E: even x,
//     O: odd x, 32 sites per word) in a private ring of four bit rows;
//   * step k converts row k+3, updates colour 0 of row k+2 and colour 1 of row
//     k+1, so that colour 1 of a row sees the final colour-0 spins of its row and
//     of the rows above and below (the tile plus halo of Sec. 3, from shared
//     memory);
//   * colour 0 is updated on all 32 lanes: it reads only colour-1 spins from
//     before the sweep, so the halo lanes compute exactly the new colour-0 spins
//     next to the band that its owned sites need; colour 1 is kept and written
//     on the owned lanes only (a halo lane's colour-1 spins stay those from
//     before the sweep, which its later colour-0 updates need);
//   * a site's move is decided from its 4 neighbours by bit-sliced adders and the
//     uint32 compare u < floor(exp(-beta dE) 2^32) of Eq. 2, with u drawn from
//     Philox4x32-10 bit planes keyed by the site (top 12 planes for every site,
//     further planes for a warp with a tie), so a word computed by two warps
//     gets the same result in both;
//   * each owned row goes back to HBM as int8 (through a 256-entry table) once
//     both of its colours are final;
//   * a colour-1 site still tied after the first 12 planes is not decided at
//     once: nothing else in the sweep reads the new colour-1 spins (colour 0
//     reads those from before the sweep), so it waits in a per-warp queue with
//     its word's spins and class masks until 32 have gathered or the segment
//     ends, and a flip then rewrites its int8 byte after the row went out.  The
//     decision is the same, so the results are too; the warp no longer runs the
//     further planes for one lane in one step out of eight.
//
// Rows next to a segment boundary are loaded (and their colour 0 updated) by both
// neighbouring segments' warps for the same reason.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "philox.cuh"
#include "spn_internal.h"
#include "sweep_common.cuh"

namespace spn {
namespace {

constexpr int kOwned = 30;      // words of a band (plus one halo word on each side = 32 lanes)
// warps per CTA, each an independent (band, segment).  One CTA of 24 warps per
// SM rather than three of 8: with three, the SM's schedulers favoured the warps
// of the first CTA, which finished in 55% of the time of the last, and the last
// third of a sweep ran on 8 warps per SM.
constexpr int kWarps = 24;
constexpr int kRing = 3;        // raw band slots per warp
constexpr int kMinBlocks = 1;   // CTAs per SM the register budget aims at
constexpr int kBitRows = 4;     // bit rows k .. k+3 live at step k
constexpr int kBandBytes = 32 * 64;
constexpr int kFirst = 3;       // Philox calls of the first decision stage (12 planes)
constexpr int kTieQueue = 64;   // deferred colour-1 words per warp: fewer than 32 after a drain, plus one step

struct WaveArgs {
  const int8_t* in;
  int8_t* out;
  int Ly, W;       // rows; 64-site words per row (at least 32)
  int nbands, nseg;
  uint32_t sweep, stream_id;
  uint32_t always;     // bit q + 1: class q (dE = 4 (q + 1)) is always accepted
  PhiloxKeys K;
  uint32_t tm[2][32];  // 0 / ~0: bit 31 - p of the threshold of class q, plane p
  unsigned long long* acc;
  int* err;
  uint32_t wait_limit;  // polls of a bounded wait before it gives up
  uint32_t skip_first;  // test support: row 0's copies are never issued
};

constexpr size_t kWaveSmem = (size_t)kWarps * kRing * kBandBytes  // raw slots
                             + (size_t)kWarps * kBitRows * 64 * 4  // bit rows
                             + 256 * 8                             // int8 output table
                             + (size_t)kWarps * kRing * 8          // mbarriers
                             + (size_t)kWarps * kTieQueue * 24;    // tie queues: (c0, eq0, eq1, b), (row, word)

// FC: Philox calls (4 planes each) of the first decision stage; AL: some class
// with dE > 0 may be always accepted (beta = 0 or tiny), else that test is left out
template <int FC, bool AL>
__global__ void __launch_bounds__(32 * kWarps, kMinBlocks) k_sweep_wave(const __grid_constant__ WaveArgs a) {
  constexpr int NC = 2;  // classes with dE > 0: dE = 4, 8
  extern __shared__ __align__(128) uint8_t smem[];
  const int W = a.W, Ly = a.Ly;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint8_t* raw = smem + (size_t)warp * kRing * kBandBytes;  // this warp's slots
  uint32_t* bits = reinterpret_cast<uint32_t*>(smem + (size_t)kWarps * kRing * kBandBytes) + warp * kBitRows * 64;
  uint2* lut = reinterpret_cast<uint2*>(smem + (size_t)kWarps * kRing * kBandBytes + (size_t)kWarps * kBitRows * 256);
  uint64_t* bars = reinterpret_cast<uint64_t*>(lut + 256) + warp * kRing;
  uint4* tq = reinterpret_cast<uint4*>(reinterpret_cast<uint64_t*>(lut + 256) + kWarps * kRing) + warp * kTieQueue;
  uint2* tq_at = reinterpret_cast<uint2*>(reinterpret_cast<uint4*>(reinterpret_cast<uint64_t*>(lut + 256) +
                                                                   kWarps * kRing) + kWarps * kTieQueue) +
                 warp * kTieQueue;
  const uint4* raw16 = reinterpret_cast<const uint4*>(raw);

  // int8 pattern of 8 sites [e0 o0 e1 o1 e2 o2 e3 o3] for index e | o << 4
  for (int i = tid; i < 256; i += blockDim.x) {
    uint32_t lo = 0, hi = 0;
    for (int k = 0; k < 4; ++k) {
      const uint32_t pair = (((i >> k) & 1) ? 0xffu : 0x01u) | ((((i >> (4 + k)) & 1) ? 0xffu : 0x01u) << 8);
      if (k < 2) lo |= pair << (16 * k); else hi |= pair << (16 * (k - 2));
    }
    lut[i] = make_uint2(lo, hi);
  }
  if (lane == 0) {
    for (int b = 0; b < kRing; ++b) mbar_init(&bars[b], 1);
    fence_mbar_init();
  }
  __syncthreads();  // the table and the barriers; warps are independent from here on

  const int unit = blockIdx.x * kWarps + warp;
  if (unit >= a.nbands * a.nseg) return;
  const int band = unit % a.nbands, seg = unit / a.nbands;
  const int zs = (int)(((int64_t)seg * Ly) / a.nseg);
  const int ze = (int)(((int64_t)(seg + 1) * Ly) / a.nseg);
  const int H = ze - zs;
  const int nload = H + 4;  // local rows li = 0 .. H + 3 <-> global zs - 2 + li
  const int j0 = kOwned * band;
  int jw = j0 - 1 + lane;  // this lane's word (W >= 32: at most one wrap)
  jw = jw < 0 ? jw + W : (jw >= W ? jw - W : jw);
  const bool owned = lane >= 1 && lane <= kOwned && j0 + lane - 1 < W;
  // the band's 32 words in memory: words j0 - 1 .. W - 1 (at most 32), then from word 0
  const int first = j0 == 0 ? W - 1 : j0 - 1;
  const int run1 = min(32, W - first);

  auto grow = [&](int li) {  // global row of local row li
    int r = zs - 2 + li;
    r = r < 0 ? r + Ly : r;
    return r >= Ly ? r - Ly : r;
  };
  // request local row li into slot li % kRing (lane 0; the slot's previous
  // contents were read by the whole warp before this call)
  auto issue = [&](int li) {
    if (lane == 0 && li < nload) {
      uint64_t* bar = &bars[li % kRing];
      uint8_t* dst = raw + (size_t)(li % kRing) * kBandBytes;
      const int8_t* src = a.in + (int64_t)grow(li) * (64 * W);
      fence_proxy_async();  // earlier generic reads of the slot before the async writes
      mbar_arrive_expect_tx(bar, (uint32_t)kBandBytes);
      if (!(a.skip_first && li == 0)) {
        bulk_g2s(dst, src + 64 * first, (uint32_t)(64 * run1), bar);
        if (run1 < 32) bulk_g2s(dst + 64 * run1, src, (uint32_t)(64 * (32 - run1)), bar);
      }
    }
  };
  int issued = 0;
  for (; issued < kRing && issued < nload; ++issued) issue(issued);

  // chunk order of the 64-byte span rotated by lane pair: a quarter warp reads 8
  // distinct 4-bank groups; rot_sel undoes the rotation on the gathered bytes
  const int rot = (lane >> 1) & 3;
  const uint32_t rot_sel = (uint32_t)(((0 - rot) & 3) | (((1 - rot) & 3) << 4) | (((2 - rot) & 3) << 8) |
                                      (((3 - rot) & 3) << 12));
  auto row_bits = [&](int li) { return bits + (li & (kBitRows - 1)) * 64; };  // E words 0..31, O words 32..63

  // wait (bounded) for local row li and turn this lane's 64 sites into bit words
  auto convert = [&](int li) -> bool {
    unsigned n = 0;
    while (!mbar_try_wait(&bars[li % kRing], (uint32_t)((li / kRing) & 1))) {
      if (++n > a.wait_limit) return false;
    }
    const uint32_t span = (uint32_t)(li % kRing) * (kBandBytes >> 4) + 4u * (uint32_t)lane;
    uint32_t pe[4], po[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const uint4 c = raw16[span + (uint32_t)((v + rot) & 3)];
      pe[v] = gather_e(c.x, c.y, c.z, c.w);
      po[v] = gather_o(c.x, c.y, c.z, c.w);
    }
    uint32_t* row = row_bits(li);
    row[lane] = __byte_perm(top_bytes(pe[0], pe[1], pe[2], pe[3]), 0u, rot_sel);
    row[32 + lane] = __byte_perm(top_bytes(po[0], po[1], po[2], po[3]), 0u, rot_sel);
    return true;
  };

  int de = 0, dm = 0;
  const uint32_t below = (1u << lane) - 1u;
  uint32_t tn = 0;  // queued colour-1 words (warp-uniform)
  // colour c of local row li (global gr): the lane's colour-c word is recomputed
  // from the other colour's words of its row and the rows above and below;
  // colour 1 also sends the finished row out as int8
  auto update = [&](int li, int c) {
    const int gr = grow(li);
    const int par = (gr + c) & 1;  // 0: the E word holds colour c, 1: the O word (warp-uniform)
    const uint32_t* rm = row_bits(li - 1);
    uint32_t* r0 = row_bits(li);
    const uint32_t* rp = row_bits(li + 1);
    const int ws = par ? 32 + lane : lane;
    const uint32_t b = r0[ws], oj = r0[par ? lane : 32 + lane];
    // x - 1 of an even site 0 is the last odd site of the previous lane's word;
    // x + 1 of the odd site 31 is the first even site of the next lane's word
    // (lanes 0 and 31 get their own word there: the bit it feeds is never used)
    const uint32_t on = par ? __shfl_down_sync(0xffffffffu, oj, 1) : __shfl_up_sync(0xffffffffu, oj, 1);
    const uint32_t left = par ? oj : (oj << 1) | (on >> 31);
    const uint32_t right = par ? (oj >> 1) | (on << 31) : oj;
    const uint32_t zm = rm[ws], zp = rp[ws];
    uint32_t s0, s1, s2, cls[NC];
    count4(b ^ left, b ^ right, b ^ zm, b ^ zp, s0, s1, s2);
    uint32_t acc = classes<2>(s0, s1, s2, 0xffffffffu, cls);
    uint32_t eq[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      const bool always = AL && ((a.always >> (k + 1)) & 1u);  // AL false: no class is (compile time)
      acc |= always ? cls[k] : 0u;
      eq[k] = always ? 0u : cls[k];
    }
    const uint32_t c0 = 8u * ((uint32_t)jw + (uint32_t)W * (uint32_t)gr);
    const uint32_t c2 = (uint32_t)c | (kMetropolis << 1);
    uint32_t pl[4 * FC];
#pragma unroll
    for (int call = 0; call < FC; ++call) {
      const U4 P = philox10(c0 + (uint32_t)call, a.sweep, c2, a.stream_id, a.K);
      pl[4 * call + 0] = P.x;
      pl[4 * call + 1] = P.y;
      pl[4 * call + 2] = P.z;
      pl[4 * call + 3] = P.w;
    }
    compare_top<NC, 4 * FC>(acc, eq, pl, a.tm);
    if (c == 0) {
      acc |= tail_planes<NC, FC>(eq, a.tm, a.K, c0, a.sweep, c2, a.stream_id);
    } else {  // owned ties wait in the queue; a halo lane's colour 1 is not kept
      const bool tie = owned && (eq[0] | eq[1]) != 0u;
      const uint32_t ties = __ballot_sync(0xffffffffu, tie);
      if (tie) {
        const uint32_t q = tn + (uint32_t)__popc(ties & below);
        tq[q] = make_uint4(c0, eq[0], eq[1], b);
        tq_at[q] = make_uint2((uint32_t)gr, (uint32_t)jw);
      }
      tn += (uint32_t)__popc(ties);
    }
    const uint32_t nb = b ^ acc;
    if (c == 0 || owned) r0[ws] = nb;
    if (owned && li >= 2 && li < H + 2) tally<2>(acc, b, s0, s1, s2, de, dm);
    if (c == 1 && owned) {
      const uint32_t E = par ? oj : nb, O = par ? nb : oj;
      const uint32_t X = (E & 0x0f0f0f0fu) | ((O << 4) & 0xf0f0f0f0u);  // byte v: sites 16v .. 16v + 7
      const uint32_t Y = ((E >> 4) & 0x0f0f0f0fu) | (O & 0xf0f0f0f0u);  // byte v: sites 16v + 8 .. 16v + 15
      uint4* dst = reinterpret_cast<uint4*>(a.out + (int64_t)gr * (64 * W) + 64 * jw);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const uint2 lo = lut[(X >> (8 * v)) & 0xffu];
        const uint2 hi = lut[(Y >> (8 * v)) & 0xffu];
        dst[v] = make_uint4(lo.x, lo.y, hi.x, hi.y);
      }
    }
  };

  // the queued colour-1 words [first, first + count), a word per lane: planes
  // 12 .. 31 as far as a site is still tied, then the flipped sites' int8 bytes
  // (after the rows' 16-byte stores of this warp) and their dE, dM
  auto drain = [&](uint32_t first, uint32_t count) {
    __syncwarp();
    uint4 e = make_uint4(0u, 0u, 0u, 0u);
    uint2 at = make_uint2(0u, 0u);
    if (lane < count) {
      e = tq[first + lane];
      at = tq_at[first + lane];
    }
    uint32_t eq[NC] = {e.y, e.z};
    const uint32_t fl = rest_planes<NC>(eq, a.tm, a.K, e.x, a.sweep, 1u | (kMetropolis << 1), a.stream_id, FC);
    if (fl) {
      de += 4 * __popc(fl & e.y) + 8 * __popc(fl & e.z);  // class 0: dE = 4, class 1: dE = 8
      dm += 2 * (2 * __popc(fl & e.w) - __popc(fl));
      const uint32_t par = (at.x + 1u) & 1u;  // colour-1 sites at x = 2 j + par of the word
      int8_t* row = a.out + (int64_t)at.x * (64 * W) + 64 * (int64_t)at.y;
      for (uint32_t f = fl; f; f &= f - 1u) {
        const int j = __ffs((int)f) - 1;
        row[2 * j + (int)par] = ((e.w >> j) & 1u) ? (int8_t)1 : (int8_t)-1;
      }
    }
    __syncwarp();
  };

  // prologue: rows 0, 1, 2 converted, colour 0 of row 1
  bool ok = true;
  for (int li = 0; li < 3 && ok; ++li) {
    ok = __all_sync(0xffffffffu, convert(li));
    __syncwarp();
    if (ok) issue(issued++);
  }
  if (ok) update(1, 0);
  // step k: convert row k + 3, colour 0 of row k + 2, colour 1 of row k + 1
  // (owned rows 2 .. H + 1 only: row 1 is the halo above the segment)
  for (int k = 0; ok && k <= H; ++k) {
    ok = __all_sync(0xffffffffu, convert(k + 3));
    if (!ok) break;
    __syncwarp();
    issue(issued++);
    update(k + 2, 0);
    if (k >= 1) update(k + 1, 1);
    if (tn >= 32u) {
      tn -= 32u;
      drain(tn, 32u);
    }
  }
  if (!ok) {  // this warp gives up
    if (lane == 0) {
      atomicExch(a.err, 1);
      // let the copies still in flight land before the warp exits: every issued
      // row gets the full poll bound, and a row whose copy was never issued is skipped
      const int last = issued < nload ? issued : nload;  // rows actually requested
      for (int li = last > kRing ? last - kRing : 0; li < last; ++li) {
        if (a.skip_first && li == 0) continue;
        unsigned n = 0;
        while (!mbar_try_wait(&bars[li % kRing], (uint32_t)((li / kRing) & 1)) && ++n < kWaitLimit) {
        }
      }
    }
    __syncwarp();
    return;
  }
  if (tn) drain(0u, tn);
  block_accumulate(de, dm, a.acc);
}

// ------------------------------------------------------------------ bit-packed lattices
//
// The same band-parallel sweep for a lattice stored one bit per spin (row r:
// the W words of its even-x sites, then the W words of its odd-x sites; a set
// bit is spin -1).  A lane's E and O words of a row are its two words of the
// packed row, so a row arrives by two 4-byte asynchronous copies per lane
// (cp.async, completed by commit groups) straight into the warp's ring of bit
// rows, and goes back as two 4-byte stores: no conversion and no int8 table.
// A flipped deferred colour-1 site is patched into the written word by an
// atomic XOR.  Nothing here spins on a flag: the copies' groups complete in
// hardware.

constexpr int kPkRing = 8;   // bit rows per warp: rows k .. k+3 in use, four more on their way
constexpr int kPkAhead = 4;  // row k + 3 + kPkAhead is requested at step k
constexpr size_t kWavePkSmem = (size_t)kWarps * kPkRing * 64 * 4  // bit rows
                               + (size_t)kWarps * kTieQueue * 24;  // tie queues

struct WavePkArgs {
  const uint32_t* in;
  uint32_t* out;
  int Ly, W;  // rows; words per colour and row (even, at least 32); a packed row is 2 W words
  int nbands, nseg;
  uint32_t sweep, stream_id;
  uint32_t always;
  PhiloxKeys K;
  uint32_t tm[2][32];
  unsigned long long* acc;
};

__device__ __forceinline__ void cp_async4(uint32_t* dst, const uint32_t* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int FC, bool AL>
__global__ void __launch_bounds__(32 * kWarps, kMinBlocks) k_sweep_wave_packed(const __grid_constant__ WavePkArgs a) {
  constexpr int NC = 2;
  extern __shared__ __align__(128) uint8_t smem[];
  const int W = a.W, Ly = a.Ly, RS = 2 * a.W;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* bits = reinterpret_cast<uint32_t*>(smem) + warp * kPkRing * 64;
  uint4* tq = reinterpret_cast<uint4*>(smem + (size_t)kWarps * kPkRing * 256) + warp * kTieQueue;
  uint2* tq_at =
      reinterpret_cast<uint2*>(smem + (size_t)kWarps * kPkRing * 256 + (size_t)kWarps * kTieQueue * 16) +
      warp * kTieQueue;

  const int unit = blockIdx.x * kWarps + warp;
  if (unit >= a.nbands * a.nseg) return;  // warps are independent: no CTA barrier in this kernel
  const int band = unit % a.nbands, seg = unit / a.nbands;
  const int zs = (int)(((int64_t)seg * Ly) / a.nseg);
  const int ze = (int)(((int64_t)(seg + 1) * Ly) / a.nseg);
  const int H = ze - zs;
  const int nload = H + 4;  // local rows li = 0 .. H + 3 <-> global zs - 2 + li
  const int j0 = kOwned * band;
  int jw = j0 - 1 + lane;
  jw = jw < 0 ? jw + W : (jw >= W ? jw - W : jw);
  const bool owned = lane >= 1 && lane <= kOwned && j0 + lane - 1 < W;

  auto grow = [&](int li) {
    int r = zs - 2 + li;
    r = r < 0 ? r + Ly : r;
    return r >= Ly ? r - Ly : r;
  };
  auto row_bits = [&](int li) { return bits + (li & (kPkRing - 1)) * 64; };  // E words 0..31, O words 32..63
  // request local row li: this lane's E and O words into its ring row; one
  // commit group per call (an empty one past the last row keeps the count)
  auto issue = [&](int li) {
    if (li < nload) {
      const uint32_t* src = a.in + (int64_t)grow(li) * RS;
      uint32_t* dst = row_bits(li);
      cp_async4(dst + lane, src + jw);
      cp_async4(dst + 32 + lane, src + W + jw);
    }
    cp_async_commit();
  };

  int de = 0, dm = 0;
  const uint32_t below = (1u << lane) - 1u;
  uint32_t tn = 0;
  auto update = [&](int li, int c) {
    const int gr = grow(li);
    const int par = (gr + c) & 1;
    const uint32_t* rm = row_bits(li - 1);
    uint32_t* r0 = row_bits(li);
    const uint32_t* rp = row_bits(li + 1);
    const int ws = par ? 32 + lane : lane;
    const uint32_t b = r0[ws], oj = r0[par ? lane : 32 + lane];
    const uint32_t on = par ? __shfl_down_sync(0xffffffffu, oj, 1) : __shfl_up_sync(0xffffffffu, oj, 1);
    const uint32_t left = par ? oj : (oj << 1) | (on >> 31);
    const uint32_t right = par ? (oj >> 1) | (on << 31) : oj;
    const uint32_t zm = rm[ws], zp = rp[ws];
    uint32_t s0, s1, s2, cls[NC];
    count4(b ^ left, b ^ right, b ^ zm, b ^ zp, s0, s1, s2);
    uint32_t acc = classes<2>(s0, s1, s2, 0xffffffffu, cls);
    uint32_t eq[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      const bool always = AL && ((a.always >> (k + 1)) & 1u);  // AL false: no class is (compile time)
      acc |= always ? cls[k] : 0u;
      eq[k] = always ? 0u : cls[k];
    }
    const uint32_t c0 = 8u * ((uint32_t)jw + (uint32_t)W * (uint32_t)gr);
    const uint32_t c2 = (uint32_t)c | (kMetropolis << 1);
    uint32_t pl[4 * FC];
#pragma unroll
    for (int call = 0; call < FC; ++call) {
      const U4 P = philox10(c0 + (uint32_t)call, a.sweep, c2, a.stream_id, a.K);
      pl[4 * call + 0] = P.x;
      pl[4 * call + 1] = P.y;
      pl[4 * call + 2] = P.z;
      pl[4 * call + 3] = P.w;
    }
    compare_top<NC, 4 * FC>(acc, eq, pl, a.tm);
    if (c == 0) {
      acc |= tail_planes<NC, FC>(eq, a.tm, a.K, c0, a.sweep, c2, a.stream_id);
    } else {
      const bool tie = owned && (eq[0] | eq[1]) != 0u;
      const uint32_t ties = __ballot_sync(0xffffffffu, tie);
      if (tie) {
        const uint32_t q = tn + (uint32_t)__popc(ties & below);
        tq[q] = make_uint4(c0, eq[0], eq[1], b);
        tq_at[q] = make_uint2((uint32_t)gr, (uint32_t)jw);
      }
      tn += (uint32_t)__popc(ties);
    }
    const uint32_t nb = b ^ acc;
    if (c == 0 || owned) r0[ws] = nb;
    if (owned && li >= 2 && li < H + 2) tally<2>(acc, b, s0, s1, s2, de, dm);
    if (c == 1 && owned) {
      uint32_t* o = a.out + (int64_t)gr * RS;
      o[jw] = par ? oj : nb;
      o[W + jw] = par ? nb : oj;
    }
  };
  // the queued colour-1 words, a word per lane: planes 12 .. 31 as far as a
  // site is still tied, then the flipped bits XOR-ed into the written word
  auto drain = [&](uint32_t first, uint32_t count) {
    __syncwarp();
    uint4 e = make_uint4(0u, 0u, 0u, 0u);
    uint2 at = make_uint2(0u, 0u);
    if (lane < count) {
      e = tq[first + lane];
      at = tq_at[first + lane];
    }
    uint32_t eq[NC] = {e.y, e.z};
    const uint32_t fl = rest_planes<NC>(eq, a.tm, a.K, e.x, a.sweep, 1u | (kMetropolis << 1), a.stream_id, FC);
    if (fl) {
      de += 4 * __popc(fl & e.y) + 8 * __popc(fl & e.z);
      dm += 2 * (2 * __popc(fl & e.w) - __popc(fl));
      const uint32_t par = (at.x + 1u) & 1u;  // 0: the E word holds colour 1
      atomicXor(a.out + (int64_t)at.x * RS + (par ? W : 0) + (int64_t)at.y, fl);
    }
    __syncwarp();
  };

  // rows 0 .. 2 + kPkAhead requested, then the prologue: colour 0 of row 1
  for (int li = 0; li < 3 + kPkAhead; ++li) issue(li);
  cp_async_wait<kPkAhead>();  // rows 0, 1, 2 have landed
  __syncwarp();
  update(1, 0);
  // step k: row k + 3 has landed; colour 0 of row k + 2, colour 1 of row k + 1
  for (int k = 0; k <= H; ++k) {
    __syncwarp();             // row k - 1 is read no more: its ring row takes row k + 3 + kPkAhead
    issue(k + 3 + kPkAhead);
    cp_async_wait<kPkAhead>();
    __syncwarp();
    update(k + 2, 0);
    if (k >= 1) update(k + 1, 1);
    if (tn >= 32u) {
      tn -= 32u;
      drain(tn, 32u);
    }
  }
  cp_async_wait<0>();
  if (tn) drain(0u, tn);
  block_accumulate(de, dm, a.acc);
}

int nbands_of(const Lattice& g) { return (g.Lx / 64 + kOwned - 1) / kOwned; }

void set_wave_attributes() {
  for (auto k : {k_sweep_wave<kFirst, false>, k_sweep_wave<kFirst, true>}) {
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWaveSmem);
    cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  }
}

}  // namespace

bool wave_supported(const Lattice& g) {
  if (g.nd != 2 || g.bonds) return false;
  if (g.pitch && g.pitch != g.Lx) return false;
  if (g.Lx % 64 || g.Lx < 2048 || g.Lx > (1 << 24)) return false;
  return g.Ly >= 2;
}

bool wave_packed_supported(const Lattice& g) {
  if (g.nd != 2 || g.bonds) return false;
  if (g.Lx % 128 || g.Lx < 2048 || g.Lx > (1 << 24)) return false;  // W even: a packed row is exactly 2 W words
  return g.Ly >= 2;
}

size_t wave_packed_smem_bytes() { return kWavePkSmem; }

size_t wave_smem_bytes(const Lattice&) { return kWaveSmem; }

int wave_cta_threads() { return 32 * kWarps; }

int wave_default_segments(const Lattice& g) {
  static std::mutex mu;
  static int per_sm = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!per_sm) {
      set_wave_attributes();
      int blocks = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_sweep_wave<kFirst, false>, 32 * kWarps, kWaveSmem) !=
          cudaSuccess)
        blocks = 1;
      per_sm = std::max(1, blocks);
    }
  }
  // one resident warp per (band, segment)
  const int64_t units = (int64_t)device_sm_count() * per_sm * kWarps;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g.Ly, units / nbands_of(g)));
}

cudaError_t launch_sweep_wave(const Lattice& g, const int8_t* in, int8_t* out, int nseg, const DevThr& T,
                              const PhiloxKeys& K, uint32_t stream_id, uint32_t sweep, unsigned long long* acc,
                              int* err, cudaStream_t st, uint32_t expire_polls) {
  if (!wave_supported(g) || nseg < 1 || nseg > g.Ly) return cudaErrorInvalidConfiguration;
  if (((uintptr_t)in & 15) || ((uintptr_t)out & 15)) return cudaErrorMisalignedAddress;  // bulk copies, 16-B stores
  WaveArgs a;
  a.in = in;
  a.out = out;
  a.Ly = g.Ly;
  a.W = g.Lx / 64;
  a.nbands = nbands_of(g);
  a.nseg = nseg;
  a.sweep = sweep;
  a.stream_id = stream_id;
  a.always = T.always;
  a.K = K;
  for (int k = 0; k < 2; ++k)
    for (int p = 0; p < 32; ++p) a.tm[k][p] = ((T.t[k + 1] >> (31 - p)) & 1u) ? 0xffffffffu : 0u;
  a.acc = acc;
  a.err = err;
  a.wait_limit = kWaitLimit;
  a.skip_first = 0;
  if (expire_polls) {  // row 0 of every warp is never copied; waits give up after `expire_polls` polls
    a.skip_first = 1;
    a.wait_limit = expire_polls;
  }
  {
    static std::mutex mu;
    static bool set[128] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    if (!set[dev & 127]) {
      set_wave_attributes();
      set[dev & 127] = true;
    }
  }
  const int64_t units = (int64_t)a.nbands * nseg;
  if (T.always & 6u)
    k_sweep_wave<kFirst, true><<<(unsigned)((units + kWarps - 1) / kWarps), 32 * kWarps, kWaveSmem, st>>>(a);
  else
    k_sweep_wave<kFirst, false><<<(unsigned)((units + kWarps - 1) / kWarps), 32 * kWarps, kWaveSmem, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_sweep_wave_packed(const Lattice& g, const uint32_t* in, uint32_t* out, int nseg, const DevThr& T,
                                     const PhiloxKeys& K, uint32_t stream_id, uint32_t sweep,
                                     unsigned long long* acc, cudaStream_t st) {
  if (!wave_packed_supported(g) || nseg < 1 || nseg > g.Ly) return cudaErrorInvalidConfiguration;
  if (((uintptr_t)in & 3) || ((uintptr_t)out & 3)) return cudaErrorMisalignedAddress;
  WavePkArgs a;
  a.in = in;
  a.out = out;
  a.Ly = g.Ly;
  a.W = g.Lx / 64;
  a.nbands = nbands_of(g);
  a.nseg = nseg;
  a.sweep = sweep;
  a.stream_id = stream_id;
  a.always = T.always;
  a.K = K;
  for (int k = 0; k < 2; ++k)
    for (int p = 0; p < 32; ++p) a.tm[k][p] = ((T.t[k + 1] >> (31 - p)) & 1u) ? 0xffffffffu : 0u;
  a.acc = acc;
  {
    static std::mutex mu;
    static bool set[128] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    if (!set[dev & 127]) {
      for (auto k : {k_sweep_wave_packed<kFirst, false>, k_sweep_wave_packed<kFirst, true>}) {
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWavePkSmem);
        cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      }
      set[dev & 127] = true;
    }
  }
  const int64_t units = (int64_t)a.nbands * nseg;
  if (T.always & 6u)
    k_sweep_wave_packed<kFirst, true><<<(unsigned)((units + kWarps - 1) / kWarps), 32 * kWarps, kWavePkSmem, st>>>(a);
  else
    k_sweep_wave_packed<kFirst, false><<<(unsigned)((units + kWarps - 1) / kWarps), 32 * kWarps, kWavePkSmem, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace spn
