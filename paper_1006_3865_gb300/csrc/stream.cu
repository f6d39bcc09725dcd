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
//     from Philox4x32-10 bit planes (two calls settle a 32-site word except for
//     ties on the top 8 bits, which each warp resolves afterwards);
//   * the finished slice goes back to HBM as int8 through a 256-entry table,
//     and the energy and magnetisation changes are reduced per CTA.
//
// Slices next to a segment boundary are loaded (and their colour 0 updated) by
// both neighbouring CTAs; the counter-based random numbers make the two copies
// identical, so no CTA ever waits for another.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "philox.cuh"
#include "spn_internal.h"
#include "sweep_common.cuh"

namespace spn {
namespace {

constexpr int kMaxRounds = 4;      // words a thread handles per phase
constexpr int kMaxThreads = 320;   // two CTAs per SM: 640 threads at <= 96 registers
constexpr int kSmemCap = 233472 / 2 - 1024;  // two CTAs per SM (228 KB per SM, 1 KB reserved per CTA)

struct StreamArgs {
  const int8_t* in;
  int8_t* out;
  int Lx, Ly, S;            // S: slices along the slowest axis (Ly in 2D, Lz in 3D)
  int TY, R, nseg, nraw, nbit, qcap;
  int roundsC, roundsA, roundsB;
  uint32_t sweep, stream_id;
  PhiloxKeys K;
  DevThr T;
  uint32_t tm[3][8];  // 0 / ~0 masks of threshold bits 31 .. 24, per class
  unsigned long long* acc;
  int* err;
};

// Per-thread work item of one phase, packed: word j (bits 0..15), row of the
// slice (16..23), slice of the step (24..30), live (31).
__device__ __forceinline__ uint32_t item_of(int i, int rows, int W, int total) {
  const int per = rows * W;
  const int ks = i / per;
  const int rem = i - ks * per;
  const int r = rem / W;
  const int j = rem - r * W;
  return (uint32_t)j | ((uint32_t)r << 16) | ((uint32_t)ks << 24) | (i < total ? 0x80000000u : 0u);
}
__device__ __forceinline__ int it_j(uint32_t x) { return (int)(x & 0xffffu); }
__device__ __forceinline__ int it_r(uint32_t x) { return (int)((x >> 16) & 0xffu); }
__device__ __forceinline__ int it_ks(uint32_t x) { return (int)((x >> 24) & 0x7fu); }
__device__ __forceinline__ bool it_live(uint32_t x, int ns) { return (x >> 31) && it_ks(x) < ns; }

// 64 int8 spins (16 little-endian words, 4 consecutive sites each) -> the E word
// (even sites) and O word (odd sites).  Bits 1..7 of a spin byte are its sign,
// so site k of a group of 8 same-parity sites is taken at a distinct bit of x
// and one multiply by two shifts moves the 8 sign bits, in order and without
// carries, into bits 24..31.
__device__ __forceinline__ uint32_t gather_e(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3) {
  const uint32_t x = (w0 & 0x00020002u) | (w1 & 0x00080008u) | (w2 & 0x00200020u) | (w3 & 0x00800080u);
  return x * ((1u << 23) + (1u << 8));
}
__device__ __forceinline__ uint32_t gather_o(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3) {
  const uint32_t x = (w0 & 0x02000200u) | (w1 & 0x08000800u) | (w2 & 0x20002000u) | (w3 & 0x80008000u);
  return x * ((1u << 15) + 1u);
}

// Top bytes of four products -> one word, product v in byte v.
__device__ __forceinline__ uint32_t top_bytes(uint32_t p0, uint32_t p1, uint32_t p2, uint32_t p3) {
  return __byte_perm(__byte_perm(p0, p1, 0x0073), __byte_perm(p2, p3, 0x0073), 0x5410);
}

template <int ND>
__global__ void __launch_bounds__(kMaxThreads, 2) k_sweep_stream(const StreamArgs a) {
  constexpr int NC = ND;  // classes with dE > 0: dE = 4 (q + 1), q < NC
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ int s_cnt[4];  // tie pools: colour 0 of even / odd steps, colour 1 of even / odd steps
  const int Lx = a.Lx, W = Lx >> 6, W2 = 2 * W;
  const int R = a.R, nbit = a.nbit, nraw = a.nraw, qcap = a.qcap;
  const int RSL = (ND == 3) ? a.TY + 4 : 1;    // rows per slice: band + 2 halo rows on each side
  const int rowsA = (ND == 3) ? a.TY + 2 : 1;  // colour-0 rows: band + 1 ring row on each side
  const int rowsB = (ND == 3) ? a.TY : 1;      // colour-1 rows: the band
  const int rowOffA = (ND == 3) ? -1 : 0;
  const int rawBytes = RSL * Lx;
  const int rawStride = (rawBytes + 127) & ~127;
  const int sliceWords = RSL * W2;
  uint8_t* raw = smem;
  uint32_t* bits = reinterpret_cast<uint32_t*>(smem + (size_t)nraw * rawStride);
  uint2* lut = reinterpret_cast<uint2*>(bits + (size_t)nbit * sliceWords);
  uint64_t* bars = reinterpret_cast<uint64_t*>(lut + 256);
  uint32_t* pools = reinterpret_cast<uint32_t*>(bars + nraw);  // 4 x [off | c0 | eq[NC]] x qcap

  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarps = nth >> 5;
  const int y0 = (ND == 3) ? blockIdx.x * a.TY : 0;
  const int zs = (int)(((int64_t)blockIdx.y * a.S) / a.nseg);
  const int ze = (int)(((int64_t)(blockIdx.y + 1) * a.S) / a.nseg);
  const int H = ze - zs;
  const int nload = H + 4;  // local slices li = 0 .. H + 3 <-> global zs - 2 + li
  const int64_t sliceStride = (int64_t)Lx * ((ND == 3) ? a.Ly : 1);

  // int8 pattern of 8 sites [e0 o0 e1 o1 e2 o2 e3 o3] for index e | o << 4
  for (int i = tid; i < 256; i += nth) {
    uint32_t lo = 0, hi = 0;
    for (int k = 0; k < 4; ++k) {
      const uint32_t pair = (((i >> k) & 1) ? 0xffu : 0x01u) | ((((i >> (4 + k)) & 1) ? 0xffu : 0x01u) << 8);
      if (k < 2) lo |= pair << (16 * k); else hi |= pair << (16 * (k - 2));
    }
    lut[i] = make_uint2(lo, hi);
  }
  if (tid < 4) s_cnt[tid] = 0;
  if (tid == 0) {
    for (int b = 0; b < nraw; ++b) mbar_init(&bars[b], 1);
    fence_mbar_init();
  }
  uint32_t ic[kMaxRounds], ia[kMaxRounds], ib[kMaxRounds];
#pragma unroll
  for (int q = 0; q < kMaxRounds; ++q) {
    ic[q] = item_of(tid + q * nth, RSL, W, R * RSL * W);
    ia[q] = item_of(tid + q * nth, rowsA, W, R * rowsA * W);
    ib[q] = item_of(tid + q * nth, rowsB, W, R * rowsB * W);
  }
  // chunk order of the 64-byte span rotated by lane pair: a quarter warp reads
  // 8 distinct 4-bank groups; rot_sel undoes the rotation on the gathered bytes
  const int rot = (lane >> 1) & 3;
  const uint32_t rot_sel = (uint32_t)(((0 - rot) & 3) | (((1 - rot) & 3) << 4) | (((2 - rot) & 3) << 8) |
                                      (((3 - rot) & 3) << 12));
  __syncthreads();

  auto wrapS = [&](int z) { return z < 0 ? z + a.S : (z >= a.S ? z - a.S : z); };
  auto wrapY = [&](int y) { return y < 0 ? y + a.Ly : (y >= a.Ly ? y - a.Ly : y); };
  // bit slot of local slice b0 + d, given sb = b0 mod nbit and -nbit < d < 2 nbit
  auto slot = [&](int sb, int d) {
    int s = sb + d;
    s = s < 0 ? s + nbit : s;
    return s >= nbit ? s - nbit : s;
  };

  // Raw ring (uniform state): slices [0, conv) converted, [0, issued) requested;
  // cslot / cpar: slot and mbarrier phase of the next slice to convert.
  int conv = 0, issued = 0, islot = 0, cslot = 0;
  uint32_t cpar = 0;
  auto issue_upto = [&]() {
    const int lim = conv + nraw < nload ? conv + nraw : nload;
    for (; issued < lim; ++issued) {
      if (tid < 32) {
        uint8_t* B = raw + (size_t)islot * rawStride;
        uint64_t* bar = &bars[islot];
        if (lane == 0) {
          fence_proxy_async();  // earlier generic reads of the slot before the async writes
          mbar_arrive_expect_tx(bar, (uint32_t)rawBytes);
        }
        __syncwarp();
        const int64_t gz = wrapS(zs - 2 + issued);
        for (int r = lane; r < RSL; r += 32) {
          const int gy = (ND == 3) ? wrapY(y0 - 2 + r) : 0;
          bulk_g2s(B + (size_t)r * Lx, a.in + gz * sliceStride + (int64_t)gy * Lx, (uint32_t)Lx, bar);
        }
      }
      if (++islot == nraw) islot = 0;
    }
  };

  // Wait (bounded) for raw slices li0 .. li0 + ns - 1 (the next ones in order)
  // and turn them into bit words; false if a wait ran out.
  auto convert = [&](int li0, int ns, int sb, int b0) -> bool {
    bool ok = true;
    int rs = cslot;
    uint32_t ph = cpar;
    for (int k = 0; k < ns; ++k) {
      unsigned n = 0;
      while (!mbar_try_wait(&bars[rs], ph)) {
        if (++n > kWaitLimit) {
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
      const uint32_t x = ic[q];
      if (q < a.roundsC && it_live(x, ns)) {
        int r = cslot + it_ks(x);
        if (r >= nraw) r -= nraw;
        const int bs = slot(sb, li0 + it_ks(x) - b0);
        const uint8_t* span = raw + (size_t)r * rawStride + (size_t)it_r(x) * Lx + 64 * it_j(x);
        uint32_t pe[4], po[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const uint4 c = *reinterpret_cast<const uint4*>(span + 16 * ((v + rot) & 3));
          pe[v] = gather_e(c.x, c.y, c.z, c.w);
          po[v] = gather_o(c.x, c.y, c.z, c.w);
        }
        uint32_t* row = bits + (size_t)bs * sliceWords + (size_t)it_r(x) * W2 + it_j(x);
        row[0] = __byte_perm(top_bytes(pe[0], pe[1], pe[2], pe[3]), 0u, rot_sel);
        row[W] = __byte_perm(top_bytes(po[0], po[1], po[2], po[3]), 0u, rot_sel);
      }
    }
    cslot = rs;
    cpar = ph;
    conv = li0 + ns;
    return ok;
  };

  int de = 0, dm = 0;

  // Apply the late-accepted sites of a tied word and count them if owned.
  auto settle = [&](uint32_t w, bool own, uint32_t late, const uint32_t (&eq0)[NC]) {
    const uint32_t cur = bits[w];  // the tied sites still hold their old spins
    bits[w] = cur ^ late;
    if (own) {
      int d = 0;
#pragma unroll
      for (int k = 0; k < NC; ++k) d += 4 * (k + 1) * __popc(late & eq0[k]);
      de += d;
      dm += 2 * (2 * __popc(late & cur) - __popc(late));
    }
  };

  // First decision stage of colour c on local slices li0 .. li0 + ns - 1 for the
  // items xs: every word is rewritten in place (a colour-c word reads only
  // colour 1 - c words) with the sites settled by the top 8 bits; words with
  // ties go to tie pool `pool`, which whole warps finish after the next barrier.
  auto phase = [&](const uint32_t (&xs)[kMaxRounds], int rounds, int li0, int ns, int c, int rowOff, int sb, int b0,
                   int pool) {
    uint32_t* P = pools + (size_t)pool * (2 + NC) * qcap;
    const uint32_t c2 = (uint32_t)c | (kMetropolis << 1);
#pragma unroll
    for (int q = 0; q < kMaxRounds; ++q) {
      if (q >= rounds) break;  // uniform
      const uint32_t x = xs[q];
      uint32_t eq[NC];
#pragma unroll
      for (int k = 0; k < NC; ++k) eq[k] = 0;
      uint32_t woff = 0, c0 = 0;
      bool own = false;
      if (it_live(x, ns)) {
        const int li = li0 + it_ks(x);
        const int bs = slot(sb, li - b0);
        const int bm = bs == 0 ? nbit - 1 : bs - 1, bp = bs + 1 == nbit ? 0 : bs + 1;
        const int gz = wrapS(zs - 2 + li);
        const int rb = it_r(x) + rowOff;                           // band row
        const int gy = (ND == 3) ? wrapY(y0 + rb) : 0;
        const int par = (((ND == 3) ? y0 + rb : 0) + gz + c) & 1;  // 0: E word, 1: O word
        const int rr = (ND == 3) ? rb + 2 : 0;                     // row within the slice
        const int j = it_j(x);
        const int rowBase = bs * sliceWords + rr * W2;
        woff = (uint32_t)(rowBase + par * W + j);
        const uint32_t b = bits[woff];
        const uint32_t* other = bits + rowBase + (W - par * W);
        const uint32_t oj = other[j];
        const uint32_t on = other[par ? (j + 1 == W ? 0 : j + 1) : (j == 0 ? W - 1 : j - 1)];
        const uint32_t left = par ? oj : __funnelshift_l(on, oj, 1);   // x - 1
        const uint32_t right = par ? __funnelshift_r(oj, on, 1) : oj;  // x + 1
        const uint32_t zm = bits[woff + (bm - bs) * sliceWords];
        const uint32_t zp = bits[woff + (bp - bs) * sliceWords];
        uint32_t s0, s1, s2;
        if constexpr (ND == 3) {
          count6(b ^ left, b ^ right, b ^ bits[woff - W2], b ^ bits[woff + W2], b ^ zm, b ^ zp, s0, s1, s2);
        } else {
          count4(b ^ left, b ^ right, b ^ zm, b ^ zp, s0, s1, s2);
        }
        uint32_t cls[NC];
        uint32_t acc = classes<ND>(s0, s1, s2, 0xffffffffu, cls);
#pragma unroll
        for (int k = 0; k < NC; ++k) {
          const bool always = (a.T.always >> (k + 1)) & 1u;
          acc |= always ? cls[k] : 0u;
          eq[k] = always ? 0u : cls[k];
        }
        c0 = 8u * ((uint32_t)j + (uint32_t)W * (uint32_t)((ND == 3) ? gy + a.Ly * gz : gz));
        const U4 P0 = philox10(c0, a.sweep, c2, a.stream_id, a.K);
        const U4 P1 = philox10(c0 + 1u, a.sweep, c2, a.stream_id, a.K);
        const uint32_t pl[8] = {P0.x, P0.y, P0.z, P0.w, P1.x, P1.y, P1.z, P1.w};
        // u < t on the top 8 bits, least significant plane first:
        // below' = maj(~u_p, t_p, below), equal &= (u_p == t_p)
#pragma unroll
        for (int k = 0; k < NC; ++k) {
          uint32_t below = 0, equal = 0xffffffffu;
#pragma unroll
          for (int p = 7; p >= 0; --p) {
            const uint32_t tm = a.tm[k][p];
            const uint32_t nu = ~pl[p];
            below = (nu & tm) | (nu & below) | (tm & below);
            equal &= ~(pl[p] ^ tm);
          }
          acc |= eq[k] & below;
          eq[k] &= equal;
        }
        bits[woff] = b ^ acc;
        own = (li >= 2 && li < H + 2) && (ND == 2 || (rb >= 0 && rb < a.TY));
        if (own) tally<ND>(acc, b, s0, s1, s2, de, dm);
      }
      uint32_t any = 0;
#pragma unroll
      for (int k = 0; k < NC; ++k) any |= eq[k];
      const unsigned vote = __ballot_sync(0xffffffffu, any != 0u);
      if (vote) {
        int base = 0;
        if (lane == 0) base = atomicAdd(&s_cnt[pool], __popc(vote));
        base = __shfl_sync(0xffffffffu, base, 0);
        const int e = base + __popc(vote & ((1u << lane) - 1u));
        const bool ovf = any != 0u && e >= qcap;
        if (any != 0u && !ovf) {
          P[e] = woff | ((uint32_t)c << 30) | (own ? 0x80000000u : 0u);
          P[qcap + e] = c0;
#pragma unroll
          for (int k = 0; k < NC; ++k) P[(2 + k) * qcap + e] = eq[k];
        }
        if (__any_sync(0xffffffffu, ovf)) {  // the pool is full: settle these words here
          uint32_t e2[NC], e0[NC];
#pragma unroll
          for (int k = 0; k < NC; ++k) e0[k] = e2[k] = ovf ? eq[k] : 0u;
          const uint32_t late = decide_tail<NC>(e2, a.T, a.K, c0, a.sweep, c2, a.stream_id);
          if (ovf) settle(woff, own, late, e0);
        }
      }
    }
  };

  // Planes 8 .. 31 for the words of two tie pools, one word per lane, packed
  // into as few warps as possible.
  auto tails = [&](int pa, int pb) {
    const int na = s_cnt[pa] < qcap ? s_cnt[pa] : qcap;
    const int nb = s_cnt[pb] < qcap ? s_cnt[pb] : qcap;
    for (int base = warp * 32; base < na + nb; base += nwarps * 32) {
      const int v = base + lane;
      uint32_t eq[NC], eq0[NC];
      uint32_t c0 = 0, off = 0;
#pragma unroll
      for (int k = 0; k < NC; ++k) eq[k] = 0;
      if (v < na + nb) {
        const uint32_t* P = pools + (size_t)(v < na ? pa : pb) * (2 + NC) * qcap;
        const int e = v < na ? v : v - na;
        off = P[e];
        c0 = P[qcap + e];
#pragma unroll
        for (int k = 0; k < NC; ++k) eq[k] = P[(2 + k) * qcap + e];
      }
#pragma unroll
      for (int k = 0; k < NC; ++k) eq0[k] = eq[k];
      const uint32_t c2 = ((off >> 30) & 1u) | (kMetropolis << 1);
      const uint32_t late = decide_tail<NC>(eq, a.T, a.K, c0, a.sweep, c2, a.stream_id);
      if (v < na + nb) settle(off & 0x3fffffffu, (off >> 31) != 0u, late, eq0);
    }
  };

  // Finished colour-1 rows (both colours final) -> int8 rows in global memory.
  auto output = [&](int li0, int ns, int sb, int b0) {
#pragma unroll
    for (int q = 0; q < kMaxRounds; ++q) {
      const uint32_t x = ib[q];
      if (q < a.roundsB && it_live(x, ns)) {
        const int li = li0 + it_ks(x);
        const int bs = slot(sb, li - b0);
        const int rr = (ND == 3) ? it_r(x) + 2 : 0;
        const uint32_t* row = bits + (size_t)bs * sliceWords + (size_t)rr * W2 + it_j(x);
        const uint32_t E = row[0], O = row[W];
        const uint32_t X = (E & 0x0f0f0f0fu) | ((O << 4) & 0xf0f0f0f0u);  // byte v: sites 16v .. 16v + 7
        const uint32_t Y = ((E >> 4) & 0x0f0f0f0fu) | (O & 0xf0f0f0f0u);  // byte v: sites 16v + 8 .. 16v + 15
        const int gz = wrapS(zs - 2 + li);
        const int gy = (ND == 3) ? y0 + it_r(x) : 0;
        uint4* dst = reinterpret_cast<uint4*>(a.out + (int64_t)gz * sliceStride + (int64_t)gy * Lx + 64 * it_j(x));
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const uint2 lo = lut[(X >> (8 * v)) & 0xffu];
          const uint2 hi = lut[(Y >> (8 * v)) & 0xffu];
          dst[v] = make_uint4(lo.x, lo.y, hi.x, hi.y);
        }
      }
    }
  };

  // Schedule.  Step t (b0 = t R) has two windows between barriers:
  //   W1: ties of colour 0 of step t-1 and colour 1 of step t-1;
  //       colour 0, first stage, on slices b0+R+3 .. b0+2R+2;
  //   W2: int8 output of the colour-1 slices of step t-1;
  //       colour 1, first stage, on slices b0+2 .. b0+R+1;
  //       conversion of slices b0+2R+4 .. b0+3R+3.
  // Colour 0 runs a full step ahead, so its ties are settled before colour 1
  // reads it; 4R+2 bit slots hold every slice a window touches.
  issue_upto();
  bool ok = true;
  const int pro = 2 * R + 4 < nload ? 2 * R + 4 : nload;
  for (int li = 0; li < pro && ok; ++li) {
    const bool mine = convert(li, 1, 0, 0);
    ok = __syncthreads_and(mine);
    if (ok) issue_upto();
  }
  if (ok) {
    const int last = R + 2 < H + 2 ? R + 2 : H + 2;  // colour 0 on slices 1 .. R+2 (ties: pool 1, step -1)
    for (int l = 1; l <= last; l += R) phase(ia, a.roundsA, l, (last - l + 1) < R ? last - l + 1 : R, 0, rowOffA, 0, 0, 1);
  }
  ok = __syncthreads_and(ok);
  const int nsteps = (H + R - 1) / R;
  int sb = 0;  // b0 mod nbit
  for (int t = 0; ok && t <= nsteps; ++t) {
    const int b0 = t * R;
    const int pe = t & 1, po = pe ^ 1;
    tails(po, 2 + po);  // pools of step t-1
    if (t < nsteps) {
      const int first = b0 + R + 3, last = b0 + 2 * R + 2 < H + 2 ? b0 + 2 * R + 2 : H + 2;
      if (first <= last) phase(ia, a.roundsA, first, last - first + 1, 0, rowOffA, sb, b0, pe);
    }
    __syncthreads();
    if (tid == 0) {
      s_cnt[po] = 0;
      s_cnt[2 + po] = 0;
    }
    if (t >= 1) {
      const int first = b0 - R + 2, last = b0 + 1 < H + 1 ? b0 + 1 : H + 1;
      output(first, last - first + 1, sb, b0);
    }
    bool mine = true;
    if (t < nsteps) {
      const int first = b0 + 2, last = b0 + R + 1 < H + 1 ? b0 + R + 1 : H + 1;
      phase(ib, a.roundsB, first, last - first + 1, 1, 0, sb, b0, 2 + pe);
      const int cf = b0 + 2 * R + 4, cl = b0 + 3 * R + 3 < nload - 1 ? b0 + 3 * R + 3 : nload - 1;
      if (cf <= cl) mine = convert(cf, cl - cf + 1, sb, b0);
    }
    ok = __syncthreads_and(mine);
    if (ok) issue_upto();
    sb += R;
    if (sb >= nbit) sb -= nbit;
  }
  if (!ok) {  // uniform: every thread saw the same barrier result
    if (tid == 0) {
      atomicExch(a.err, 1);
      // let the copies still in flight land before the CTA exits (bounded)
      for (int li = issued > nraw ? issued - nraw : 0; li < issued; ++li) {
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

bool stream_path_supported(const Lattice& g, int TY) {
  if (g.bonds) return false;
  if (g.Lx % 64) return false;
  if (g.nd == 3 && (TY < 2 || TY > 250 || (TY & 1) || g.Ly % TY)) return false;
  if (g.Lx / 64 > 65535) return false;
  const int RSL = g.nd == 3 ? TY + 4 : 1;
  if ((int64_t)RSL * g.Lx * 2 > 96 * 1024) return false;  // two raw slices must fit beside the rest
  return true;
}

namespace {

size_t smem_bytes(const Lattice& g, int TY, int R, int nraw, int threads, int qcap) {
  const int W = g.Lx / 64;
  const int RSL = g.nd == 3 ? TY + 4 : 1;
  const size_t rawStride = (size_t)((RSL * g.Lx + 127) & ~127);
  const size_t bitsB = (size_t)(4 * R + 2) * RSL * 2 * W * 4;
  const size_t q = (size_t)4 * (2 + g.nd) * qcap * 4;
  return (size_t)nraw * rawStride + bitsB + 256 * 8 + (size_t)nraw * 8 + q;
}

// Entries of one tie pool: a quarter of a phase's words, about twice the
// expected number of ties (one site in 256 of the positive-dE sites).
int pool_cap(int threads, int ra, int rb) { return std::max(64, (threads * std::max(ra, rb) / 4 + 31) / 32 * 32); }

void phase_counts(const Lattice& g, int TY, int R, int& nC, int& nA, int& nB) {
  const int W = g.Lx / 64;
  nC = R * (g.nd == 3 ? TY + 4 : 1) * W;
  nA = R * (g.nd == 3 ? TY + 2 : 1) * W;
  nB = R * (g.nd == 3 ? TY : 1) * W;
}

}  // namespace

StreamGeom stream_geometry(const Lattice& g, int TY, int R, int nseg) {
  StreamGeom s{};
  s.TY = g.nd == 3 ? TY : 1;
  const int S = g.nd == 3 ? g.Lz : g.Ly;
  auto threads_for = [&](int r) {  // about two colour-0 words per thread
    int nC, nA, nB;
    phase_counts(g, s.TY, r, nC, nA, nB);
    int th = ((nA + 1) / 2 + 31) / 32 * 32;
    const int need = ((std::max(nC, std::max(nA, nB)) + kMaxRounds - 1) / kMaxRounds + 31) / 32 * 32;
    th = std::max(th, need);
    return std::max(64, std::min(kMaxThreads, th));
  };
  auto rounds_for = [&](int r, int th, int& rc, int& ra, int& rb) {
    int nC, nA, nB;
    phase_counts(g, s.TY, r, nC, nA, nB);
    rc = (nC + th - 1) / th;
    ra = (nA + th - 1) / th;
    rb = (nB + th - 1) / th;
    return std::max(rc, std::max(ra, rb));
  };
  const bool automatic = R <= 0;
  if (automatic) {
    R = 1;
    for (int r = std::min(S, 64); r >= 1; --r) {
      const int th = threads_for(r);
      int rc, ra, rb;
      if (rounds_for(r, th, rc, ra, rb) > kMaxRounds) continue;
      if (smem_bytes(g, s.TY, r, 2 * r, th, pool_cap(th, ra, rb)) <= (size_t)kSmemCap) {
        R = r;
        break;
      }
    }
  }
  s.R = R;
  s.nbit = 4 * R + 2;
  s.threads = threads_for(R);
  int rc, ra, rb;
  rounds_for(R, s.threads, rc, ra, rb);
  s.roundsC = rc;
  s.roundsA = ra;
  s.roundsB = rb;
  s.qcap = pool_cap(s.threads, ra, rb);
  s.nraw = 2 * R;  // a slice is requested one step before it is converted
  while (s.nraw > R && smem_bytes(g, s.TY, R, s.nraw, s.threads, s.qcap) > (size_t)kSmemCap) --s.nraw;
  s.smem = smem_bytes(g, s.TY, R, s.nraw, s.threads, s.qcap);
  if (nseg <= 0) {
    const int tiles = g.nd == 3 ? g.Ly / s.TY : 1;
    const int want = device_sm_count() * 2;
    nseg = std::max(1, std::min(S, (want + tiles - 1) / tiles));
  }
  s.nseg = std::min(nseg, S);
  return s;
}

bool stream_geometry_ok(const Lattice& g, const StreamGeom& geo) {
  if (geo.R < 1 || geo.threads < 32 || geo.threads > kMaxThreads || geo.threads % 32) return false;
  int nC, nA, nB;
  phase_counts(g, geo.TY, geo.R, nC, nA, nB);
  const int cap = geo.threads * kMaxRounds;
  if (nC > cap || nA > cap || nB > cap) return false;
  if (geo.roundsC * geo.threads < nC || geo.roundsA * geo.threads < nA || geo.roundsB * geo.threads < nB) return false;
  if (geo.roundsC > kMaxRounds || geo.roundsA > kMaxRounds || geo.roundsB > kMaxRounds) return false;
  if (geo.qcap < 32 || geo.qcap % 32) return false;
  if (geo.smem != smem_bytes(g, geo.TY, geo.R, geo.nraw, geo.threads, geo.qcap)) return false;
  return geo.smem <= 227 * 1024 && geo.nraw >= geo.R && geo.nbit == 4 * geo.R + 2 && geo.nseg >= 1 &&
         geo.nseg <= (g.nd == 3 ? g.Lz : g.Ly);
}

cudaError_t launch_sweep_stream(const Lattice& g, const int8_t* in, int8_t* out, const StreamGeom& geo,
                                const DevThr& T, const PhiloxKeys& K, uint32_t stream_id, uint32_t sweep,
                                unsigned long long* acc, int* err, cudaStream_t st) {
  if (!stream_geometry_ok(g, geo)) return cudaErrorInvalidConfiguration;
  if (((uintptr_t)in & 15) || ((uintptr_t)out & 15)) return cudaErrorMisalignedAddress;  // bulk copies, 16-B stores
  StreamArgs a;
  a.in = in;
  a.out = out;
  a.Lx = g.Lx;
  a.Ly = g.Ly;
  a.S = g.nd == 3 ? g.Lz : g.Ly;
  a.TY = geo.TY;
  a.R = geo.R;
  a.nseg = geo.nseg;
  a.nraw = geo.nraw;
  a.nbit = geo.nbit;
  a.qcap = geo.qcap;
  a.roundsC = geo.roundsC;
  a.roundsA = geo.roundsA;
  a.roundsB = geo.roundsB;
  a.sweep = sweep;
  a.stream_id = stream_id;
  a.K = K;
  a.T = T;
  for (int k = 0; k < 3; ++k)
    for (int p = 0; p < 8; ++p) a.tm[k][p] = ((T.t[k + 1] >> (31 - p)) & 1u) ? 0xffffffffu : 0u;
  a.acc = acc;
  a.err = err;
  dim3 grid(g.nd == 3 ? g.Ly / geo.TY : 1, geo.nseg);
  if (g.nd == 3) {
    cudaFuncSetAttribute(k_sweep_stream<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)geo.smem);
    cudaFuncSetAttribute(k_sweep_stream<3>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    k_sweep_stream<3><<<grid, geo.threads, geo.smem, st>>>(a);
  } else {
    cudaFuncSetAttribute(k_sweep_stream<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)geo.smem);
    cudaFuncSetAttribute(k_sweep_stream<2>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    k_sweep_stream<2><<<grid, geo.threads, geo.smem, st>>>(a);
  }
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace spn
