// Streaming checkerboard sweep of a large 2D / 3D Ising lattice (J = 1).
//
// One launch is one full sweep in the canonical two-colour order of Sec. 3
// (every site of colour 0, then every site of colour 1), with each int8 spin
// read from HBM once and written once.  The lattice is cut along its slowest
// axis (rows in 2D, planes in 3D) into slices; a CTA owns a run of slices of one
// band of rows and walks down it:
//
//   * the raw int8 slices arrive by bulk asynchronous copies (TMA engine) into a
//     ring in shared memory, completed on mbarriers;
//   * each slice is turned into colour-separated bit words (E: even x, O: odd x,
//     32 sites per word) with masks and one multiply per 8 sites;
//   * colour 0 is updated one slice ahead of colour 1, so that colour 1 of slice
//     s sees the final colour-0 spins of slices s-1, s, s+1 (the staged tile plus
//     halo of Sec. 3, re-read from shared memory instead of global memory);
//   * a site's move is decided from its 4 (6) neighbours by bit-sliced adders and
//     the uint32 compare u < floor(exp(-beta dE) 2^32) of Eq. 2, with u drawn
//     from Philox4x32-10 bit planes: three calls give the top 12 bits of u for
//     all 32 sites of a word, which settles every site but about one in 4096
//     of those with dE > 0; a warp with such a tie draws further planes for
//     all its lanes together;
//   * each colour-1 word is written back to HBM as int8 (through a 256-entry
//     table) as soon as it is final, and the energy and magnetisation changes
//     are reduced per CTA.
//
// Slices next to a segment boundary are loaded (and their colour 0 updated) by
// both neighbouring CTAs; the counter-based random numbers make the two copies
// identical, so no CTA ever waits for another.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <atomic>
#include <mutex>

#include "philox.cuh"
#include "spn_internal.h"
#include "sweep_common.cuh"

namespace spn {
namespace {

constexpr int kMaxRounds = 2;  // words a thread handles per phase
// Threads per CTA and the CTAs per SM the register budget aims at (3D keeps
// four CTAs of up to 160 threads resident with 96 registers each, which
// measured faster than three of 256 threads with 80 and spills; 2D uses more
// registers per thread).
constexpr int max_threads(int nd) { return nd == 3 ? 160 : 512; }
constexpr int min_ctas(int nd) { return nd == 3 ? 4 : 1; }
constexpr int kCtasPerSm = 4;                          // CTAs per SM the default geometry aims for
constexpr int kSmemCap = 233472 / kCtasPerSm - 1024;  // 228 KB per SM, 1 KB reserved per CTA
#ifndef SPN_FIRST_CALLS
#define SPN_FIRST_CALLS 3
#endif
constexpr int kFirstCalls = SPN_FIRST_CALLS;  // Philox calls of the first decision stage (4 planes each)

struct StreamArgs {
  const void* in;  // int8 rows of P bytes, or bit-packed rows of RS words
  void* out;
  int Lx, Ly, S;  // S: slices along the slowest axis (Ly in 2D, Lz in 3D)
  int P;          // int8: bytes per row in memory (a multiple of 64, >= Lx); packed: 64 ceil(Lx / 64)
  int RS;         // packed: words per row (E words, O words, zero padding; a multiple of 4)
  int vbl;        // sites per colour in the last 64-site word of a row (1 .. 32)
  int TY, R, nseg, nraw, nbit;
  int roundsC, roundsA, roundsB;
  uint32_t sweep, stream_id;
  uint32_t always;     // bit q + 1: class q (dE = 4 (q + 1)) is always accepted
  PhiloxKeys K;
  uint32_t tm[3][32];  // 0 / ~0: bit 31 - p of the threshold of class q, plane p
  unsigned long long* acc;
  int* err;
  uint32_t wait_limit;  // polls of a bounded mbarrier wait before it gives up
  uint32_t skip_first;  // test support: slice 0's copies are never issued (0)
};

// Per-thread work items, fixed for the launch (item i = thread + q * threads of a
// phase covers slice i / (rows W) of the step, row (i / W) % rows, word i % W).
//   offset word: bits 0..23 word offset within a slice, 24..30 slice of the step,
//                31 live
//   flags:       bit 0 row parity (3D: (y0 + band row) & 1), bit 1 owned row,
//                bit 2 first word of the row, bit 3 last word of the row
__device__ __forceinline__ uint32_t pack_item(int i, int total, int ks, uint32_t off) {
  return off | ((uint32_t)ks << 24) | (i < total ? 0x80000000u : 0u);
}

// PACKED: the lattice lives in HBM as bit words (row r: E words 0 .. W-1, O
// words W .. 2W-1, zero padding to RS words), copied straight into the bit slots
// (one mbarrier per slot) and written back as words; no int8 conversion.
template <int ND, bool PACKED>
__global__ void __launch_bounds__(max_threads(ND), min_ctas(ND)) k_sweep_stream(const __grid_constant__ StreamArgs a) {
  constexpr int NC = ND;  // classes with dE > 0: dE = 4 (q + 1), q < NC
  extern __shared__ __align__(128) uint8_t smem[];
  const int P = a.P, W = P >> 6, W2 = PACKED ? a.RS : 2 * W, vbl = a.vbl;
  const uint32_t vmaskl = vbl == 32 ? 0xffffffffu : ((1u << vbl) - 1u);  // valid lanes of a row's last word
  const int R = a.R, nbit = a.nbit, nraw = a.nraw, S = a.S;
  const int RSL = (ND == 3) ? a.TY + 4 : 1;    // rows per slice: band + 2 halo rows on each side
  const int rowsA = (ND == 3) ? a.TY + 2 : 1;  // colour-0 rows: band + 1 ring row on each side
  const int rowsB = (ND == 3) ? a.TY : 1;      // colour-1 rows: the band
  const int rowBytes = PACKED ? W2 * 4 : P;  // bytes of one row copy
  const int rawBytes = RSL * rowBytes;        // bytes of one slice copy
  const int rawStride = PACKED ? 0 : (rawBytes + 127) & ~127;
  const int sliceWords = RSL * W2;
  uint8_t* raw = smem;
  uint32_t* bits = reinterpret_cast<uint32_t*>(smem + (size_t)nraw * rawStride);
  uint2* lut = reinterpret_cast<uint2*>(bits + (size_t)nbit * sliceWords);
  uint64_t* bars = reinterpret_cast<uint64_t*>(lut + (PACKED ? 0 : 256));
  const uint4* raw16 = reinterpret_cast<const uint4*>(smem);

  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31;
  const int y0 = (ND == 3) ? blockIdx.x * a.TY : 0;
  const int zs = (int)(((int64_t)blockIdx.y * S) / a.nseg);
  const int ze = (int)(((int64_t)(blockIdx.y + 1) * S) / a.nseg);
  const int H = ze - zs;
  const int nload = H + 4;  // local slices li = 0 .. H + 3 <-> global zs - 2 + li
  const int64_t sliceStride = (int64_t)rowBytes * ((ND == 3) ? a.Ly : 1);  // bytes

  // int8 pattern of 8 sites [e0 o0 e1 o1 e2 o2 e3 o3] for index e | o << 4
  for (int i = tid; i < (PACKED ? 0 : 256); i += nth) {
    uint32_t lo = 0, hi = 0;
    for (int k = 0; k < 4; ++k) {
      const uint32_t pair = (((i >> k) & 1) ? 0xffu : 0x01u) | ((((i >> (4 + k)) & 1) ? 0xffu : 0x01u) << 8);
      if (k < 2) lo |= pair << (16 * k); else hi |= pair << (16 * (k - 2));
    }
    lut[i] = make_uint2(lo, hi);
  }
  if (tid == 0) {
    for (int b = 0; b < nraw; ++b) mbar_init(&bars[b], 1);
    fence_mbar_init();
  }

  // ---- per-thread items
  uint32_t cOff[kMaxRounds] = {}, cRaw[kMaxRounds] = {};     // conversion (int8 only)
  uint32_t aOff[kMaxRounds], aC0[kMaxRounds], aFl[kMaxRounds];  // colour 0
  uint32_t bOff[kMaxRounds], bC0[kMaxRounds], bFl[kMaxRounds], bOut[kMaxRounds];  // colour 1
#pragma unroll
  for (int q = 0; q < kMaxRounds; ++q) {
    const int i = tid + q * nth;
    if (!PACKED) {
      const int per = RSL * W, ks = i / per, r = (i - ks * per) / W, j = i - ks * per - r * W;
      cOff[q] = pack_item(i, R * per, ks, (uint32_t)(r * W2 + j));
      cRaw[q] = ((uint32_t)(r * P + 64 * j) >> 4) | (j == W - 1 ? 0x80000000u : 0u);  // bit 31: last word
    }
    {
      const int per = rowsA * W, ks = i / per, r = (i - ks * per) / W, j = i - ks * per - r * W;
      const int rb = (ND == 3) ? r - 1 : 0;  // band row -1 .. TY
      const int gy = (ND == 3) ? (y0 + rb + a.Ly) % a.Ly : 0;
      aOff[q] = pack_item(i, R * per, ks, (uint32_t)(((ND == 3) ? (rb + 2) * W2 : 0) + j));
      aC0[q] = 8u * ((uint32_t)j + (uint32_t)W * (uint32_t)gy);
      aFl[q] = (uint32_t)((y0 + rb) & 1) | ((ND == 2 || (rb >= 0 && rb < a.TY)) ? 2u : 0u) | (j == 0 ? 4u : 0u) |
               (j == W - 1 ? 8u : 0u);
    }
    {
      const int per = rowsB * W, ks = i / per, r = (i - ks * per) / W, j = i - ks * per - r * W;
      const int gy = y0 + r;
      bOff[q] = pack_item(i, R * per, ks, (uint32_t)(((ND == 3) ? (r + 2) * W2 : 0) + j));
      bC0[q] = 8u * ((uint32_t)j + (uint32_t)W * (uint32_t)((ND == 3) ? gy : 0));
      bFl[q] = (uint32_t)((y0 + r) & 1) | 2u | (j == 0 ? 4u : 0u) | (j == W - 1 ? 8u : 0u);
      bOut[q] = PACKED ? (uint32_t)(((ND == 3) ? gy * W2 : 0) + j) : (uint32_t)(((ND == 3) ? gy * P : 0) + 64 * j);
    }
  }
  // chunk order of the 64-byte span rotated by lane pair: a quarter warp reads
  // 8 distinct 4-bank groups; rot_sel undoes the rotation on the gathered bytes
  const int rot = (lane >> 1) & 3;
  const uint32_t rot_sel = (uint32_t)(((0 - rot) & 3) | (((1 - rot) & 3) << 4) | (((2 - rot) & 3) << 8) |
                                      (((3 - rot) & 3) << 12));
  __syncthreads();

  auto wrapS = [&](int z) { return z < 0 ? z + S : (z >= S ? z - S : z); };
  auto wrapY = [&](int y) { return y < 0 ? y + a.Ly : (y >= a.Ly ? y - a.Ly : y); };

  // Copy ring (uniform state): slices [0, conv) converted (packed: arrived),
  // [0, issued) requested, [0, dead) no longer read; cslot / cpar: slot and
  // mbarrier phase of the next slice to convert.  int8 slices go to a ring of
  // nraw raw slots; packed slices straight to their bit slot (nraw = nbit).
  int conv = 0, issued = 0, islot = 0, cslot = 0, dead = 0;
  uint32_t cpar = 0;
  auto issue_upto = [&]() {
    const int free_from = PACKED ? dead : conv;
    const int lim = free_from + nraw < nload ? free_from + nraw : nload;
    for (; issued < lim; ++issued) {
      if (tid < 32) {
        uint8_t* B = PACKED ? reinterpret_cast<uint8_t*>(bits + (size_t)islot * sliceWords)
                            : raw + (size_t)islot * rawStride;
        uint64_t* bar = &bars[islot];
        if (lane == 0) {
          fence_proxy_async();  // earlier generic reads of the slot before the async writes
          mbar_arrive_expect_tx(bar, (uint32_t)rawBytes);
        }
        __syncwarp();
        const int64_t gz = wrapS(zs - 2 + issued);
        const bool skip = a.skip_first && issued == 0;  // its barrier then never completes
        for (int r = lane; r < RSL && !skip; r += 32) {
          const int gy = (ND == 3) ? wrapY(y0 - 2 + r) : 0;
          bulk_g2s(B + (size_t)r * rowBytes,
                   static_cast<const uint8_t*>(a.in) + gz * sliceStride + (int64_t)gy * rowBytes,
                   (uint32_t)rowBytes, bar);
        }
      }
      if (++islot == nraw) islot = 0;
    }
  };

  // Wait (bounded) for raw slices li0 .. li0 + ns - 1 (the next ones in order)
  // and turn them into bit words in slots sfirst ..; false if a wait ran out.
  auto convert = [&](int li0, int ns, int sfirst) -> bool {
    bool ok = true;
    int rs = cslot;
    uint32_t ph = cpar;
    for (int k = 0; k < ns; ++k) {
      unsigned n = 0;
      while (!mbar_try_wait(&bars[rs], ph)) {
        if (++n > a.wait_limit) {
          ok = false;
          break;
        }
      }
      if (++rs == nraw) {
        rs = 0;
        ph ^= 1u;
      }
    }
#pragma unroll
    for (int q = 0; q < kMaxRounds; ++q) {
      const uint32_t x = cOff[q];
      const int ks = (int)((x >> 24) & 0x7fu);
      if (!PACKED && q < a.roundsC && (x >> 31) && ks < ns) {
        int r = cslot + ks;
        r -= r >= nraw ? nraw : 0;
        int sl = sfirst + ks;
        sl -= sl >= nbit ? nbit : 0;
        const uint32_t span = (uint32_t)r * (uint32_t)(rawStride >> 4) + (cRaw[q] & 0x7fffffffu);
        uint32_t pe[4], po[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const uint4 c = raw16[span + (uint32_t)((v + rot) & 3)];
          pe[v] = gather_e(c.x, c.y, c.z, c.w);
          po[v] = gather_o(c.x, c.y, c.z, c.w);
        }
        uint32_t* row = bits + (uint32_t)sl * (uint32_t)sliceWords + (x & 0xffffffu);
        const uint32_t keep = (cRaw[q] >> 31) ? vmaskl : 0xffffffffu;  // padding sites of a row stay 0
        row[0] = __byte_perm(top_bytes(pe[0], pe[1], pe[2], pe[3]), 0u, rot_sel) & keep;
        row[W] = __byte_perm(top_bytes(po[0], po[1], po[2], po[3]), 0u, rot_sel) & keep;
      }
    }
    cslot = rs;
    cpar = ph;
    conv = li0 + ns;
    return ok;
  };

  int de = 0, dm = 0;

  // Colour c on local slices li0 .. li0 + ns - 1 (first one in bit slot sfirst,
  // global slice gz0): every word is rewritten in place (a colour-c word reads
  // only colour 1 - c words); colour-1 words also go out as int8 at once.
  auto phase = [&](const uint32_t (&off)[kMaxRounds], const uint32_t (&c0q)[kMaxRounds],
                   const uint32_t (&flq)[kMaxRounds], int rounds, int li0, int ns, int sfirst, int gz0, int c) {
    const uint32_t c2 = (uint32_t)c | (kMetropolis << 1);
#pragma unroll
    for (int q = 0; q < kMaxRounds; ++q) {
      if (q >= rounds) break;  // uniform
      const uint32_t x = off[q];
      const int ks = (int)((x >> 24) & 0x7fu);
      const bool live = (x >> 31) && ks < ns;
      uint32_t acc = 0, eq[NC], b = 0, oj = 0, s0 = 0, s1 = 0, s2 = 0, c0 = 0, woff = 0;
      int gz = 0;
#pragma unroll
      for (int k = 0; k < NC; ++k) eq[k] = 0;
      if (live) {
        int sl = sfirst + ks;
        sl -= sl >= nbit ? nbit : 0;
        gz = gz0 + ks;
        gz -= gz >= S ? S : 0;
        const uint32_t fl = flq[q];
        const int par = (int)((fl + (uint32_t)gz + (uint32_t)c) & 1u);  // 0: E word, 1: O word
        woff = (uint32_t)sl * (uint32_t)sliceWords + (x & 0xffffffu) + (uint32_t)(par * W);
        b = bits[woff];
        const uint32_t other = par ? woff - (uint32_t)W : woff + (uint32_t)W;
        oj = bits[other];
        const int dj = par ? ((fl & 8u) ? 1 - W : 1) : ((fl & 4u) ? W - 1 : -1);
        const uint32_t on = bits[other + (uint32_t)dj];
        // x - 1 of lane 0 is the last site of the previous word; x + 1 of the
        // last lane is the first site of the next word (periodic in x)
        const uint32_t left = par ? oj : (oj << 1) | ((on >> (((fl & 4u) ? vbl : 32) - 1)) & 1u);
        const uint32_t right = par ? (oj >> 1) | ((on & 1u) << (((fl & 8u) ? vbl : 32) - 1)) : oj;
        const uint32_t zm = bits[sl == 0 ? woff + (uint32_t)((nbit - 1) * sliceWords) : woff - (uint32_t)sliceWords];
        const uint32_t zp = bits[sl == nbit - 1 ? woff - (uint32_t)((nbit - 1) * sliceWords) : woff + (uint32_t)sliceWords];
        if constexpr (ND == 3) {
          count6(b ^ left, b ^ right, b ^ bits[woff - (uint32_t)W2], b ^ bits[woff + (uint32_t)W2], b ^ zm, b ^ zp,
                 s0, s1, s2);
        } else {
          count4(b ^ left, b ^ right, b ^ zm, b ^ zp, s0, s1, s2);
        }
        uint32_t cls[NC];
        acc = classes<ND>(s0, s1, s2, (fl & 8u) ? vmaskl : 0xffffffffu, cls);
#pragma unroll
        for (int k = 0; k < NC; ++k) {
          const bool always = (a.always >> (k + 1)) & 1u;
          acc |= always ? cls[k] : 0u;
          eq[k] = always ? 0u : cls[k];
        }
        c0 = c0q[q] + 8u * (uint32_t)W * (uint32_t)((ND == 3) ? a.Ly * gz : gz);
        uint32_t pl[4 * kFirstCalls];
#pragma unroll
        for (int call = 0; call < kFirstCalls; ++call) {
          const U4 P = philox10(c0 + (uint32_t)call, a.sweep, c2, a.stream_id, a.K);
          pl[4 * call + 0] = P.x;
          pl[4 * call + 1] = P.y;
          pl[4 * call + 2] = P.z;
          pl[4 * call + 3] = P.w;
        }
        compare_top<NC, 4 * kFirstCalls>(acc, eq, pl, a.tm);
      }
      acc |= tail_planes<NC, kFirstCalls>(eq, a.tm, a.K, c0, a.sweep, c2, a.stream_id);
      if (live) {
        const uint32_t nb = b ^ acc;
        bits[woff] = nb;
        const int li = li0 + ks;
        if ((flq[q] & 2u) && li >= 2 && li < H + 2) tally<ND>(acc, b, s0, s1, s2, de, dm);
        if (c == 1) {
          const int par = (int)((flq[q] + (uint32_t)gz + 1u) & 1u);
          const uint32_t E = par ? oj : nb, O = par ? nb : oj;
          if constexpr (PACKED) {
            uint32_t* dst =
                reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(a.out) + (int64_t)gz * sliceStride) + bOut[q];
            dst[0] = E;
            dst[W] = O;
          } else {
            const uint32_t X = (E & 0x0f0f0f0fu) | ((O << 4) & 0xf0f0f0f0u);  // byte v: sites 16v .. 16v + 7
            const uint32_t Y = ((E >> 4) & 0x0f0f0f0fu) | (O & 0xf0f0f0f0u);  // byte v: sites 16v + 8 .. 16v + 15
            uint4* dst =
                reinterpret_cast<uint4*>(static_cast<int8_t*>(a.out) + (int64_t)gz * sliceStride + bOut[q]);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
              const uint2 lo = lut[(X >> (8 * v)) & 0xffu];
              const uint2 hi = lut[(Y >> (8 * v)) & 0xffu];
              dst[v] = make_uint4(lo.x, lo.y, hi.x, hi.y);
            }
          }
        }
      }
    }
  };

  // Schedule: step b0 converts (packed: waits for) slices b0+4 .. b0+3+ns,
  // updates colour 0 on b0+3 .. b0+2+ns and colour 1 (with the output) on
  // b0+2 .. b0+1+ns; 2R+3 bit slots hold every slice a step touches, and a
  // packed slice is requested as soon as the slice two steps back in its slot
  // is no longer read.
  issue_upto();
  bool ok = true;
  const int pro = 4 < nload ? 4 : nload;
  for (int li = 0; li < pro && ok; ++li) {
    const bool mine = convert(li, 1, li);
    ok = __syncthreads_and(mine);
    if (ok) issue_upto();
  }
  if (ok) {
    for (int l = 1; l < 3; l += R) {
      const int ns = (3 - l) < R ? 3 - l : R;
      phase(aOff, aC0, aFl, a.roundsA, l, ns, l, wrapS(zs - 2 + l), 0);
    }
    __syncthreads();
  }
  int sb = 0;  // bit slot of local slice b0
  for (int b0 = 0; ok && b0 < H; b0 += R) {
    const int ns = (b0 + R < H) ? R : H - b0;
    auto slot = [&](int d) { return sb + d >= nbit ? sb + d - nbit : sb + d; };
    const bool mine = convert(b0 + 4, ns, slot(4));
    ok = __syncthreads_and(mine);
    if (!ok) break;
    dead = b0 + 1;  // every thread is past the previous step: slices <= b0 are no longer read
    issue_upto();
    phase(aOff, aC0, aFl, a.roundsA, b0 + 3, ns, slot(3), wrapS(zs + 1 + b0), 0);
    __syncthreads();
    phase(bOff, bC0, bFl, a.roundsB, b0 + 2, ns, slot(2), wrapS(zs + b0), 1);
    sb = slot(R);
  }
  if (!ok) {  // uniform: every thread saw the same barrier result
    if (tid == 0) {
      atomicExch(a.err, 1);
      // let the copies still in flight land before the CTA exits: every issued
      // slice gets the full poll bound (a shortened test bound applies only to
      // the wait that gave up), and a slice whose copy was never issued is skipped
      for (int li = issued > nraw ? issued - nraw : 0; li < issued; ++li) {
        if (a.skip_first && li == 0) continue;
        unsigned n = 0;
        while (!mbar_try_wait(&bars[li % nraw], (uint32_t)((li / nraw) & 1)) && ++n < kWaitLimit) {
        }
      }
    }
    __syncthreads();
    return;
  }
  block_accumulate(de, dm, a.acc);
}

}  // namespace

static int pitch_of(const Lattice& g) { return g.pitch ? g.pitch : g.Lx; }

int packed_row_words(int Lx) { return (2 * ((Lx + 63) / 64) + 3) & ~3; }

namespace {

// Row copy in bytes and the smem row stride in words for a storage form.
int row_bytes(const Lattice& g, bool packed) { return packed ? 4 * packed_row_words(g.Lx) : pitch_of(g); }
int row_stride_words(const Lattice& g, bool packed) {
  return packed ? packed_row_words(g.Lx) : 2 * (pitch_of(g) / 64);
}

}  // namespace

bool stream_path_supported(const Lattice& g, int TY, bool packed) {
  if (g.bonds) return false;
  if (g.Lx < 2 || (g.Lx & 1)) return false;
  if (!packed) {
    const int P = pitch_of(g);
    if (P % 64 || P < g.Lx || P - g.Lx >= 64) return false;
  } else if (g.pitch) {
    return false;  // packed rows carry their own padding
  }
  if (g.nd == 3 && (TY < 2 || TY > 250 || (TY & 1) || g.Ly % TY)) return false;
  if ((g.Lx + 63) / 64 > 65535) return false;
  const int RSL = g.nd == 3 ? TY + 4 : 1;
  if (!packed && (int64_t)RSL * pitch_of(g) * 2 > 96 * 1024) return false;  // two raw slices fit beside the rest
  if (packed && (int64_t)RSL * row_bytes(g, true) * 5 > 160 * 1024) return false;  // five bit slots fit one CTA
  return true;
}

namespace {

size_t smem_bytes(const Lattice& g, int TY, int R, int nraw, bool packed) {
  const int RSL = g.nd == 3 ? TY + 4 : 1;
  const size_t bitsB = (size_t)(2 * R + 3) * RSL * row_stride_words(g, packed) * 4;
  if (packed) return bitsB + (size_t)(2 * R + 3) * 8;
  const size_t rawStride = (size_t)((RSL * pitch_of(g) + 127) & ~127);
  return (size_t)nraw * rawStride + bitsB + 256 * 8 + (size_t)nraw * 8;
}

void phase_counts(const Lattice& g, int TY, int R, bool packed, int& nC, int& nA, int& nB) {
  const int W = (g.Lx + 63) / 64;
  nC = packed ? 0 : R * (g.nd == 3 ? TY + 4 : 1) * W;
  nA = R * (g.nd == 3 ? TY + 2 : 1) * W;
  nB = R * (g.nd == 3 ? TY : 1) * W;
}

}  // namespace

StreamGeom stream_geometry(const Lattice& g, int TY, int R, int nseg, bool packed) {
  StreamGeom s{};
  s.packed = packed ? 1 : 0;
  if (!packed && R <= 1 && g.nd == 3 && wave3_supported(g, TY)) {  // one plane per step: the 3D wavefront kernel
    s.wave = 2;
    s.TY = TY;
    s.R = 1;
    s.threads = wave3_cta_threads(g, TY);
    s.nseg = nseg > 0 ? std::min(nseg, g.Lz) : wave3_default_segments(g, TY);
    s.smem = wave3_smem_bytes(g, TY);
    return s;
  }
  if (packed && R <= 1 && g.nd == 3 && wave3_supported(g, TY)) {  // one plane per step: the 3D wavefront, bit-packed
    s.wave = 4;
    s.TY = TY;
    s.R = 1;
    s.threads = wave3_cta_threads(g, TY, true);
    s.nseg = nseg > 0 ? std::min(nseg, g.Lz) : wave3_default_segments(g, TY, true);
    s.smem = wave3_smem_bytes(g, TY, true);
    return s;
  }
  if (packed && R <= 1 && wave_packed_supported(g)) {  // one row per step: the band-parallel kernel, bit-packed
    s.wave = 3;
    s.TY = 1;
    s.R = 1;
    s.threads = wave_cta_threads();
    s.nseg = nseg > 0 ? std::min(nseg, g.Ly) : wave_default_segments(g);
    s.smem = wave_packed_smem_bytes();
    return s;
  }
  if (!packed && R <= 1 && wave_supported(g)) {  // one row per step: the band-parallel kernel
    s.wave = 1;
    s.TY = 1;
    s.R = 1;
    s.threads = wave_cta_threads();
    s.nseg = nseg > 0 ? std::min(nseg, g.Ly) : wave_default_segments(g);
    s.smem = wave_smem_bytes(g);
    return s;
  }
  s.TY = g.nd == 3 ? TY : 1;
  const int S = g.nd == 3 ? g.Lz : g.Ly;
  const int maxT = max_threads(g.nd);
  auto threads_for = [&](int r) {  // at most kMaxRounds words per thread and phase
    int nC, nA, nB;
    phase_counts(g, s.TY, r, packed, nC, nA, nB);
    const int th = ((std::max(nC, std::max(nA, nB)) + kMaxRounds - 1) / kMaxRounds + 31) / 32 * 32;
    return std::max(64, th);
  };
  const bool automatic = R <= 0;
  if (automatic) {
    // the fewest slices per step that keep at least 128 colour-0 words per step
    // (short steps keep four CTAs per SM within shared memory and registers)
    R = 1;
    for (int r = 1; r <= std::min(S, 64); ++r) {
      int nC, nA, nB;
      phase_counts(g, s.TY, r, packed, nC, nA, nB);
      if (threads_for(r) > maxT || smem_bytes(g, s.TY, r, 2 * r, packed) > (size_t)kSmemCap) break;
      R = r;
      if (nA >= 128) break;
    }
  }
  s.R = R;
  s.nbit = 2 * R + 3;
  s.threads = std::min(maxT, threads_for(R));
  int nC, nA, nB;
  phase_counts(g, s.TY, R, packed, nC, nA, nB);
  s.roundsC = (nC + s.threads - 1) / s.threads;
  s.roundsA = (nA + s.threads - 1) / s.threads;
  s.roundsB = (nB + s.threads - 1) / s.threads;
  s.qcap = 0;
  if (packed) {
    s.nraw = s.nbit;  // copies land in the bit slots
  } else {
    s.nraw = 2 * R;  // a slice is requested about one step before it is converted
    while (s.nraw > R && smem_bytes(g, s.TY, R, s.nraw, false) > (size_t)kSmemCap) --s.nraw;
  }
  s.smem = smem_bytes(g, s.TY, R, s.nraw, packed);
  if (nseg <= 0) {
    const int tiles = g.nd == 3 ? g.Ly / s.TY : 1;
    const int want = device_sm_count() * kCtasPerSm;
    nseg = std::max(1, std::min(S, (want + tiles - 1) / tiles));
  }
  s.nseg = std::min(nseg, S);
  return s;
}

bool stream_geometry_ok(const Lattice& g, const StreamGeom& geo) {
  const bool packed = geo.packed != 0;
  if (geo.wave == 2) return !packed && wave3_supported(g, geo.TY) && geo.nseg >= 1 && geo.nseg <= g.Lz;
  if (geo.wave == 4) return packed && wave3_supported(g, geo.TY) && geo.nseg >= 1 && geo.nseg <= g.Lz;
  if (geo.wave == 3) return packed && wave_packed_supported(g) && geo.nseg >= 1 && geo.nseg <= g.Ly;
  if (geo.wave) return !packed && wave_supported(g) && geo.nseg >= 1 && geo.nseg <= g.Ly;
  if (geo.R < 1 || geo.R > 127 || geo.threads < 32 || geo.threads > max_threads(g.nd) || geo.threads % 32) return false;
  int nC, nA, nB;
  phase_counts(g, geo.TY, geo.R, packed, nC, nA, nB);
  if (geo.roundsC * geo.threads < nC || geo.roundsA * geo.threads < nA || geo.roundsB * geo.threads < nB) return false;
  if (geo.roundsC > kMaxRounds || geo.roundsA > kMaxRounds || geo.roundsB > kMaxRounds) return false;
  if (geo.smem != smem_bytes(g, geo.TY, geo.R, geo.nraw, packed)) return false;
  if (packed ? geo.nraw != geo.nbit : geo.nraw < geo.R) return false;
  return geo.smem <= 227 * 1024 && geo.nbit == 2 * geo.R + 3 && geo.nseg >= 1 &&
         geo.nseg <= (g.nd == 3 ? g.Lz : g.Ly);
}

cudaError_t launch_sweep_stream(const Lattice& g, const void* in, void* out, const StreamGeom& geo,
                                const DevThr& T, const PhiloxKeys& K, uint32_t stream_id, uint32_t sweep,
                                unsigned long long* acc, int* err, cudaStream_t st, uint32_t expire_polls) {
  if (!stream_geometry_ok(g, geo)) return cudaErrorInvalidConfiguration;
  if (geo.wave == 2)
    return launch_sweep_wave3(g, static_cast<const int8_t*>(in), static_cast<int8_t*>(out), geo.TY, geo.nseg, T, K,
                              stream_id, sweep, acc, err, st, expire_polls);
  if (geo.wave == 4) {
    if (expire_polls) {  // test support: armed launches go to the CTA pipeline, as for wave 3
      const StreamGeom alt = stream_geometry(g, geo.TY, 2, 0, true);
      return launch_sweep_stream(g, in, out, alt, T, K, stream_id, sweep, acc, err, st, expire_polls);
    }
    return launch_sweep_wave3_packed(g, static_cast<const uint32_t*>(in), static_cast<uint32_t*>(out), geo.TY, geo.nseg,
                                     T, K, stream_id, sweep, acc, err, st);
  }
  if (geo.wave == 3) {
    if (expire_polls) {  // test support: that kernel has no bounded wait to give up; the CTA pipeline takes the launch
      const StreamGeom alt = stream_geometry(g, 1, 2, 0, true);
      return launch_sweep_stream(g, in, out, alt, T, K, stream_id, sweep, acc, err, st, expire_polls);
    }
    return launch_sweep_wave_packed(g, static_cast<const uint32_t*>(in), static_cast<uint32_t*>(out), geo.nseg, T, K,
                                    stream_id, sweep, acc, st);
  }
  if (geo.wave)
    return launch_sweep_wave(g, static_cast<const int8_t*>(in), static_cast<int8_t*>(out), geo.nseg, T, K, stream_id,
                             sweep, acc, err, st, expire_polls);
  if (((uintptr_t)in & 15) || ((uintptr_t)out & 15)) return cudaErrorMisalignedAddress;  // bulk copies, 16-B stores
  StreamArgs a;
  a.in = in;
  a.out = out;
  a.Lx = g.Lx;
  a.P = geo.packed ? 64 * ((g.Lx + 63) / 64) : pitch_of(g);
  a.RS = geo.packed ? packed_row_words(g.Lx) : 0;
  a.vbl = (g.Lx - (a.P - 64)) / 2;
  a.Ly = g.Ly;
  a.S = g.nd == 3 ? g.Lz : g.Ly;
  a.TY = geo.TY;
  a.R = geo.R;
  a.nseg = geo.nseg;
  a.nraw = geo.nraw;
  a.nbit = geo.nbit;
  a.roundsC = geo.roundsC;
  a.roundsA = geo.roundsA;
  a.roundsB = geo.roundsB;
  a.sweep = sweep;
  a.stream_id = stream_id;
  a.always = T.always;
  a.K = K;
  for (int k = 0; k < 3; ++k)
    for (int p = 0; p < 32; ++p) a.tm[k][p] = ((T.t[k + 1] >> (31 - p)) & 1u) ? 0xffffffffu : 0u;
  a.acc = acc;
  a.err = err;
  a.wait_limit = kWaitLimit;
  a.skip_first = 0;
  if (expire_polls) {  // slice 0 of every CTA is never copied; waits give up after `expire_polls` polls
    a.skip_first = 1;
    a.wait_limit = expire_polls;
  }
  dim3 grid(g.nd == 3 ? g.Ly / geo.TY : 1, geo.nseg);
  // function attributes are set once per device and raised only when a launch needs more
  static std::mutex mu;
  static int smem_set[128][4] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  const int variant = (g.nd == 3 ? 1 : 0) + (geo.packed ? 2 : 0);
  auto kernel = [&]() -> void (*)(StreamArgs) {
    switch (variant) {
      case 0: return k_sweep_stream<2, false>;
      case 1: return k_sweep_stream<3, false>;
      case 2: return k_sweep_stream<2, true>;
      default: return k_sweep_stream<3, true>;
    }
  }();
  {
    std::lock_guard<std::mutex> lock(mu);
    int& cur = smem_set[dev & 127][variant];
    if ((int)geo.smem > cur) {
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)geo.smem);
      cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      cur = (int)geo.smem;
    }
  }
  kernel<<<grid, geo.threads, geo.smem, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

// ---- conversion between int8 rows and bit-packed rows (warp per 64-site word)

namespace {

__global__ void k_pack(const int8_t* __restrict__ s, uint32_t* __restrict__ w, int Lx, int W, int RS, int64_t units) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < units; u += nw) {
    const int64_t row = u / W;
    const int j = (int)(u - row * W);
    const int x = 64 * j + 2 * lane;
    uint32_t pair = 0x0101u;  // padding sites: +1, bit 0
    if (x < Lx) pair = *reinterpret_cast<const uint16_t*>(s + row * Lx + x);
    const uint32_t e = __ballot_sync(0xffffffffu, (pair & 0x80u) != 0u);    // x even: spin -1
    const uint32_t o = __ballot_sync(0xffffffffu, (pair & 0x8000u) != 0u);  // x odd
    uint32_t* dst = w + row * RS;
    if (lane == 0) dst[j] = e;
    if (lane == 1) dst[W + j] = o;
    if (j == W - 1 && lane < RS - 2 * W) dst[2 * W + lane] = 0u;
  }
}

__global__ void k_unpack(const uint32_t* __restrict__ w, int8_t* __restrict__ s, int Lx, int W, int RS, int64_t units) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < units; u += nw) {
    const int64_t row = u / W;
    const int j = (int)(u - row * W);
    const int x = 64 * j + 2 * lane;
    const uint32_t e = w[row * RS + j], o = w[row * RS + W + j];
    if (x < Lx) {
      const uint32_t lo = ((e >> lane) & 1u) ? 0xffu : 0x01u, hi = ((o >> lane) & 1u) ? 0xff00u : 0x0100u;
      *reinterpret_cast<uint16_t*>(s + row * Lx + x) = (uint16_t)(lo | hi);
    }
  }
}

int conv_blocks(int64_t units) {
  const int64_t want = (units + 7) / 8;  // 8 warps per block
  const int64_t cap = (int64_t)device_sm_count() * 16;
  return (int)std::max<int64_t>(1, std::min(want, cap));
}

}  // namespace

cudaError_t launch_pack(const Lattice& g, const int8_t* s, uint32_t* w, cudaStream_t st) {
  if ((g.Lx & 1) || ((uintptr_t)s & 1)) return cudaErrorInvalidValue;
  const int W = (g.Lx + 63) / 64;
  const int64_t units = g.N / g.Lx * W;
  if (units == 0) return cudaSuccess;
  k_pack<<<conv_blocks(units), 256, 0, st>>>(s, w, g.Lx, W, packed_row_words(g.Lx), units);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const Lattice& g, const uint32_t* w, int8_t* s, cudaStream_t st) {
  if ((g.Lx & 1) || ((uintptr_t)s & 1)) return cudaErrorInvalidValue;
  const int W = (g.Lx + 63) / 64;
  const int64_t units = g.N / g.Lx * W;
  if (units == 0) return cudaSuccess;
  k_unpack<<<conv_blocks(units), 256, 0, st>>>(w, s, g.Lx, W, packed_row_words(g.Lx), units);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace spn
