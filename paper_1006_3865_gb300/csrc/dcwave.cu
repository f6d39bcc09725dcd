// Band-parallel streaming form of the paper's double-checkerboard sweep with
// multi-hit (Sec. 3) on a large 2D Ising lattice: one launch is one full sweep
// in the order of the tile algorithm (every tile of parity 0: colour 0, colour
// 1, `hits` times over; then every tile of parity 1 the same way), each int8
// spin read from HBM once and written once.
//
// The layout is that of the canonical band-parallel sweep (wave.cu): a warp owns
// a band of 30 64-site words (plus a halo word on each side) and a segment of
// rows, lane i holds word j0 - 1 + i, rows come by bulk copies into a private
// ring and are turned into colour-separated bit words.  A tile is Tx x Ty sites
// with Tx a multiple of 64, so a lane's word lies in one tile per row; its tile
// parity P = (word / (Tx / 64) + row / Ty) & 1 flips every Ty rows.
//
// With Q = 4 hits phases q = 2 hits P + 2 h + c (parity, hit, colour), phase q
// of a row reads the sites of phase q - 1 in that row and the rows above and
// below, so the rows advance as a wavefront: at step k the lanes of parity 0
// take phase s (< 2 hits) at row k + Q - s and the lanes of parity 1 phase
// 2 hits + s at row k + 2 hits - 1 - s, for s = 0 .. 2 hits - 1 in turn.  Every
// phase of parity 0 on a row comes at an earlier step than every phase of
// parity 1 on that row and on the rows above and below it, so a parity-1 site
// sees its parity-0 neighbours final and a parity-0 site sees its parity-1
// neighbours from before the sweep, as the tile order wants.  A lane's
// two rows of a slot have one parity between tile rows; where they straddle one
// the lane has two updates (or none) in that slot, and the warp takes a second
// pass.  Lanes of one slot sit on different rows, so a word's x neighbours come
// from shared memory, not by shuffles.  The halo lanes are recomputed as in
// wave.cu: an error that enters at a halo lane's outer site moves one site per
// phase, and Q phases never reach its inner site (Q < 64).  The kernel is
// written for any number of hits; it is built for one, where it beats the tile
// kernel (from two hits on the tile kernel reuses its staged tile for every hit
// and is faster, and a deeper ring and Q halo rows per segment end slow this
// one down).  The Philox planes are
// those of the tile kernel (purpose 4, counter sweep * hits + hit), so results
// equal the tile kernel's and the oracle's bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "philox.cuh"
#include "spn_internal.h"
#include "fastdiv.cuh"
#include "sweep_common.cuh"

namespace spn {
namespace {

constexpr int kDwOwned = 30;     // words of a band (plus one halo word on each side = 32 lanes)
// warps per CTA, each an independent (band, segment): one CTA per SM, since an
// SM's schedulers favour the warps of its first CTA and with several CTAs the
// last one ran alone at the end of the sweep
constexpr int kDwWarps = 24;
constexpr int kDwRing = 3;       // raw band slots per warp
constexpr int kDwBandBytes = 32 * 64;
constexpr int kDwFirst = 3;      // Philox calls of the first decision stage (12 planes)
constexpr int kDwMaxHits = 1;  // the tile kernel is faster from 2 hits on (its tile stays staged)
constexpr uint32_t kDwPurpose = 4u;  // the tile kernel's purpose bits

struct DwArgs {
  const int8_t* in;
  int8_t* out;
  int Ly, W;      // rows; 64-site words per row (at least 32)
  int Wt, Ty;     // tile width in words, tile height in rows
  int hits;
  int nbands, nseg;
  uint32_t ctr0;  // sweep * hits
  uint32_t stream_id;
  uint32_t always;
  PhiloxKeys K;
  uint32_t tm[2][32];
  unsigned long long* acc;
  int* err;
  uint32_t wait_limit;
  uint32_t skip_first;
};

int dw_ring_rows(int hits) {  // as R in the kernel
  int r = 8;
  while (r < 4 * hits + 3) r *= 2;
  return r;
}

size_t dw_smem(int hits) {
  return (size_t)kDwWarps * kDwRing * kDwBandBytes + (size_t)kDwWarps * dw_ring_rows(hits) * 64 * 4 + 256 * 8 +
         (size_t)kDwWarps * kDwRing * 8;
}

// AL: some class with dE > 0 may be always accepted (beta = 0 or tiny), else that test is left out
template <int HITS, bool AL>
__global__ void __launch_bounds__(32 * kDwWarps, 1) k_sweep_dcwave(const __grid_constant__ DwArgs a) {
  constexpr int NC = 2;  // classes with dE > 0: dE = 4, 8
  extern __shared__ __align__(128) uint8_t smem[];
  constexpr int Q = 4 * HITS, half = 2 * HITS, R = Q + 3 <= 8 ? 8 : (Q + 3 <= 16 ? 16 : 32);
  const int W = a.W, Ly = a.Ly;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint8_t* raw = smem + (size_t)warp * kDwRing * kDwBandBytes;  // this warp's slots
  uint32_t* bits = reinterpret_cast<uint32_t*>(smem + (size_t)kDwWarps * kDwRing * kDwBandBytes) + (size_t)warp * R * 64;
  uint2* lut =
      reinterpret_cast<uint2*>(smem + (size_t)kDwWarps * kDwRing * kDwBandBytes + (size_t)kDwWarps * R * 64 * 4);
  uint64_t* bars = reinterpret_cast<uint64_t*>(lut + 256) + warp * kDwRing;
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
    for (int b = 0; b < kDwRing; ++b) mbar_init(&bars[b], 1);
    fence_mbar_init();
  }
  __syncthreads();  // the table and the barriers; warps are independent from here on

  const int unit = blockIdx.x * kDwWarps + warp;
  if (unit >= a.nbands * a.nseg) return;
  const int band = unit % a.nbands, seg = unit / a.nbands;
  const int zs = (int)(((int64_t)seg * Ly) / a.nseg);
  const int ze = (int)(((int64_t)(seg + 1) * Ly) / a.nseg);
  const int H = ze - zs;
  const int nload = H + 2 * Q;  // local rows li = 0 .. H + 2Q - 1 <-> global zs - Q + li
  const int j0 = kDwOwned * band;
  int jw = j0 - 1 + lane;  // this lane's word (W >= 32: at most one wrap)
  jw = jw < 0 ? jw + W : (jw >= W ? jw - W : jw);
  const bool owned = lane >= 1 && lane <= kDwOwned && j0 + lane - 1 < W;
  const int first = j0 == 0 ? W - 1 : j0 - 1;
  const int run1 = min(32, W - first);
  const uint32_t tx = (uint32_t)(jw / a.Wt);  // tile column of this lane's word
  const FastDiv fTy = fastdiv((uint32_t)a.Ty);

  auto grow = [&](int li) {  // global row of local row li (Ly >= 2Q: one wrap at most)
    int r = zs - Q + li;
    r = r < 0 ? r + Ly : r;
    return r >= Ly ? r - Ly : r;
  };
  auto parity = [&](int gr) { return (int)((tx + fdiv((uint32_t)gr, fTy)) & 1u); };
  auto issue = [&](int li) {
    if (lane == 0 && li < nload) {
      uint64_t* bar = &bars[li % kDwRing];
      uint8_t* dst = raw + (size_t)(li % kDwRing) * kDwBandBytes;
      const int8_t* src = a.in + (int64_t)grow(li) * (64 * W);
      fence_proxy_async();  // earlier generic reads of the slot before the async writes
      mbar_arrive_expect_tx(bar, (uint32_t)kDwBandBytes);
      if (!(a.skip_first && li == 0)) {
        bulk_g2s(dst, src + 64 * first, (uint32_t)(64 * run1), bar);
        if (run1 < 32) bulk_g2s(dst + 64 * run1, src, (uint32_t)(64 * (32 - run1)), bar);
      }
    }
  };
  int issued = 0;
  for (; issued < kDwRing && issued < nload; ++issued) issue(issued);

  const int rot = (lane >> 1) & 3;
  const uint32_t rot_sel = (uint32_t)(((0 - rot) & 3) | (((1 - rot) & 3) << 4) | (((2 - rot) & 3) << 8) |
                                      (((3 - rot) & 3) << 12));
  auto row_bits = [&](int li) { return bits + (li & (R - 1)) * 64; };  // E words 0..31, O words 32..63

  auto convert = [&](int li) -> bool {
    unsigned n = 0;
    while (!mbar_try_wait(&bars[li % kDwRing], (uint32_t)((li / kDwRing) & 1))) {
      if (++n > a.wait_limit) return false;
    }
    const uint32_t span = (uint32_t)(li % kDwRing) * (kDwBandBytes >> 4) + 4u * (uint32_t)lane;
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
  // one update of colour c, hit h at this lane's local row li (rows differ
  // between lanes): the lane's colour-c word from the other colour's words of
  // its row (its own and its neighbours', read from shared memory) and of the
  // rows above and below.  `store` is false on a lane that has no update in
  // this pass (it still takes part in the warp's votes); `last` marks the final
  // phase of the lane's parity, after which its word goes out as int8.
  auto update = [&](int li, int c, int h, bool store, bool last) {
    const int gr = grow(li);
    const int par = (gr + c) & 1;  // 0: the E word holds colour c, 1: the O word
    const uint32_t* rm = row_bits(li - 1);
    uint32_t* r0 = row_bits(li);
    const uint32_t* rp = row_bits(li + 1);
    const int ws = par ? 32 + lane : lane;
    const uint32_t b = r0[ws], oj = r0[par ? lane : 32 + lane];
    // x - 1 of an even site 0 is the last odd site of the previous lane's word;
    // x + 1 of the odd site 31 is the first even site of the next lane's word
    // (lanes 0 and 31 take their own word there: the bit it feeds is never used)
    const uint32_t on = par ? r0[min(lane + 1, 31)] : r0[32 + max(lane - 1, 0)];
    const uint32_t left = par ? oj : (oj << 1) | (on >> 31);
    const uint32_t right = par ? (oj >> 1) | (on << 31) : oj;
    uint32_t s0, s1, s2, cls[NC];
    count4(b ^ left, b ^ right, b ^ rm[ws], b ^ rp[ws], s0, s1, s2);
    uint32_t acc = classes<2>(s0, s1, s2, 0xffffffffu, cls);
    uint32_t eq[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      const bool always = AL && ((a.always >> (k + 1)) & 1u);  // AL false: no class is (compile time)
      acc |= always ? cls[k] : 0u;
      eq[k] = always ? 0u : cls[k];
    }
    const uint32_t c0 = 8u * ((uint32_t)jw + (uint32_t)W * (uint32_t)gr);
    const uint32_t c1 = a.ctr0 + (uint32_t)h;
    const uint32_t c2 = (uint32_t)c | (kDwPurpose << 1);
    uint32_t pl[4 * kDwFirst];
#pragma unroll
    for (int call = 0; call < kDwFirst; ++call) {
      const U4 P = philox10(c0 + (uint32_t)call, c1, c2, a.stream_id, a.K);
      pl[4 * call + 0] = P.x;
      pl[4 * call + 1] = P.y;
      pl[4 * call + 2] = P.z;
      pl[4 * call + 3] = P.w;
    }
    if (!store) eq[0] = eq[1] = 0u;  // a lane without an update asks for no further planes
    compare_top<NC, 4 * kDwFirst>(acc, eq, pl, a.tm);
    acc |= tail_planes<NC, kDwFirst>(eq, a.tm, a.K, c0, c1, c2, a.stream_id);
    if (!store) return;
    const uint32_t nb = b ^ acc;
    r0[ws] = nb;
    const bool mine = owned && li >= Q && li < H + Q;
    if (mine) tally<2>(acc, b, s0, s1, s2, de, dm);
    if (last && mine) {
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

  // Phase q of the tile order is done on local rows q + 1 .. H + 2Q - 2 - q (a
  // row needs its neighbours' phase q - 1); the last phase covers the owned
  // rows Q .. H + Q - 1.  Step k first converts row k + Q + 1, the deepest row
  // that phase 0 at row k + Q reads; the ring holds rows k - 1 .. k + Q + 1.
  bool ok = true;
  for (int li = 0; li < 2 && ok; ++li) {
    ok = __all_sync(0xffffffffu, convert(li));
    __syncwarp();
    if (ok) issue(issued++);
  }
  for (int k = 1 - Q; ok && k <= H + Q - 1; ++k) {
    if (k + Q + 1 < nload) {
      ok = __all_sync(0xffffffffu, convert(k + Q + 1));
      if (!ok) break;
      __syncwarp();
      issue(issued++);
    }
#pragma unroll
    for (int s = 0; s < half; ++s) {
      const int c = s & 1, h = s >> 1;
      const int liA = k + Q - s, liB = k + half - 1 - s;  // phase s (parity 0), phase half + s (parity 1)
      const bool vA = liA >= s + 1 && liA <= H + 2 * Q - 2 - s;
      const bool vB = liB >= half + s + 1 && liB <= H + 2 * Q - 2 - half - s;
      const bool doA = vA && parity(grow(liA)) == 0;
      const bool doB = vB && parity(grow(liB)) == 1;
      const bool last = s == half - 1;
      if (__any_sync(0xffffffffu, doA || doB)) update(doA || !doB ? liA : liB, c, h, doA || doB, last);
      if (__any_sync(0xffffffffu, doA && doB)) update(liB, c, h, doA && doB, last);  // rows straddling a tile row
    }
  }
  if (!ok) {  // this warp gives up
    if (lane == 0) {
      atomicExch(a.err, 1);
      // let the copies still in flight land before the warp exits: every issued
      // row gets the full poll bound, and a row whose copy was never issued is skipped
      const int lastrow = issued < nload ? issued : nload;
      for (int li = lastrow > kDwRing ? lastrow - kDwRing : 0; li < lastrow; ++li) {
        if (a.skip_first && li == 0) continue;
        unsigned n = 0;
        while (!mbar_try_wait(&bars[li % kDwRing], (uint32_t)((li / kDwRing) & 1)) && ++n < kWaitLimit) {
        }
      }
    }
    __syncwarp();
    return;
  }
  block_accumulate(de, dm, a.acc);
}

int dw_nbands(const Lattice& g) { return (g.Lx / 64 + kDwOwned - 1) / kDwOwned; }

using DwKernel = void (*)(DwArgs);
DwKernel dw_kernel(int, bool al) { return al ? k_sweep_dcwave<1, true> : k_sweep_dcwave<1, false>; }

// the shared-memory attributes of the kernel for `hits`, once per device
void dw_prepare(int hits) {
  static std::mutex mu;
  static bool set[128][kDwMaxHits + 1] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  if (!set[dev & 127][hits]) {
    for (bool al : {false, true}) {
      cudaFuncSetAttribute(dw_kernel(hits, al), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dw_smem(hits));
      cudaFuncSetAttribute(dw_kernel(hits, al), cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    }
    set[dev & 127][hits] = true;
  }
}

}  // namespace

bool dcwave_supported(const Lattice& g, int Tx, int Ty, int hits) {
  if (g.nd != 2 || g.bonds) return false;
  if (g.pitch && g.pitch != g.Lx) return false;
  if (g.Lx % 64 || g.Lx < 2048 || g.Lx > (1 << 24)) return false;
  if (hits < 1 || hits > kDwMaxHits || Tx < 64 || Tx % 64 || Ty < 1) return false;
  if (g.Lx % Tx || (g.Lx / Tx) % 2 || g.Ly % Ty || (g.Ly / Ty) % 2) return false;
  return g.Ly >= 8 * hits;  // the Q halo rows on each side of a segment wrap at most once
}

int dcwave_default_segments(const Lattice& g, int hits) {
  static std::mutex mu;
  static int per_sm[kDwMaxHits + 1] = {};
  dw_prepare(hits);
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!per_sm[hits]) {
      int blocks = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, dw_kernel(hits, false), 32 * kDwWarps, dw_smem(hits)) !=
          cudaSuccess)
        blocks = 1;
      per_sm[hits] = std::max(1, blocks);
    }
  }
  // one resident warp per (band, segment)
  const int64_t units = (int64_t)device_sm_count() * per_sm[hits] * kDwWarps;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g.Ly, units / dw_nbands(g)));
}

cudaError_t launch_sweep_dcwave(const Lattice& g, const int8_t* in, int8_t* out, int Tx, int Ty, int hits, int nseg,
                                const DevThr& T, const PhiloxKeys& K, uint32_t stream_id, uint32_t sweep,
                                unsigned long long* acc, int* err, cudaStream_t st, uint32_t expire_polls) {
  if (!dcwave_supported(g, Tx, Ty, hits) || nseg < 1 || nseg > g.Ly) return cudaErrorInvalidConfiguration;
  if (((uintptr_t)in & 15) || ((uintptr_t)out & 15) || in == out) return cudaErrorInvalidValue;
  DwArgs a;
  a.in = in;
  a.out = out;
  a.Ly = g.Ly;
  a.W = g.Lx / 64;
  a.Wt = Tx / 64;
  a.Ty = Ty;
  a.hits = hits;
  a.nbands = dw_nbands(g);
  a.nseg = nseg;
  a.ctr0 = sweep * (uint32_t)hits;
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
  dw_prepare(hits);
  const int64_t units = (int64_t)a.nbands * nseg;
  dw_kernel(hits, (T.always & 6u) != 0)<<<(unsigned)((units + kDwWarps - 1) / kDwWarps), 32 * kDwWarps, dw_smem(hits),
                                          st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace spn
