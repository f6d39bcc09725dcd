// Multi-spin coded +-J Edwards-Anderson spin glass with replica exchange
// (Weigel, Sec. 4: many disorder realisations at once with asynchronous
// multi-spin coding; parallel tempering is the batched workload of this
// library, with the standard pair-exchange rule of Hukushima and Nemoto).
//
// Square (2D, 4 bonds per site) and simple cubic (3D, 6 bonds) lattices.
// Storage: a batch of S disorder samples, each with 32 replicas held in the
// 32 temperature slots of one word per site.  In device memory two samples
// share a 64-bit word (bits 0-31 sample 2p, bits 32-63 sample 2p+1), so each
// uint64 carries 64 replicas.  Bonds: one byte per site and sample, bit d set
// iff J(n, d) = -1 (forward bond to n + e_d), bit 3 + d iff J(n - e_d, d) = -1.
//
// k_ea_resident: one CTA per sample keeps the sample's whole word lattice and
// bonds in shared memory (colour-separated: even-x and odd-x words per row) for
// all sweeps of a launch.  Per site: the 2 ND neighbour words XOR the bond masks
// give the unsatisfied bonds of all 32 replicas; a bit-sliced adder counts them;
// replicas with dE = 4 (ND - k) > 0 accept iff u < thr(beta of their
// temperature, dE).  The thresholds of one dE level grow with the temperature index, so the
// accepting temperatures form a suffix: the number of thresholds <= u gives its
// start and a 33-entry table, kept in step with the slot permutation, turns it
// into the slot mask.  That number comes from a 1024-bucket table over the top
// 10 bits of u, one 32-bit entry per bucket with a byte per level (the count at
// the bucket's start and whether 0, 1 or more thresholds fall inside it), and
// at most one compare per level; only a bucket holding two or more thresholds
// of some level takes the 5-step binary search.  When
// Lx is a multiple of 8 a thread updates four consecutive same-colour words of
// a row at once: 16-byte shared-memory loads and stores, and the one Philox
// call whose four words are the four sites' u.  After every X-th sweep the CTA
// counts unsatisfied bonds per replica, takes the exchange decisions of the
// even or odd temperature pairs with host-built tables of
// floor(exp(dbeta * dE) 2^32), and updates the permutation.
//
// With replica exchange (the default there; k_ea_resident<ND, true>) every slot
// draws its own u, bit 31 - p of slot j's u being bit j of plane p of the
// site's own Philox calls.  A shared u leaves each replica's Metropolis step
// exact but correlates the replicas, and replica exchange then lets the
// temperature marginals drift; with a u per slot the ladder stays exact.  The
// CTA keeps per dE level and plane the mask of slots whose temperature's
// threshold has that bit set (rebuilt after each exchange) and compares planes
// most significant first until no slot ties: planes 0-7 for all four sites of
// a thread at once (their Philox calls interleaved), then the few sites still
// tied one call at a time.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "philox.cuh"
#include "spn.h"
#include "spn_internal.h"
#include "fastdiv.cuh"

namespace spn {

// colour-separated shared-memory word index of site (x, y, z)
__device__ __forceinline__ int ea_slot(int x, int row, int h) { return (row * 2 + (x & 1)) * h + (x >> 1); }

constexpr int kEaBucketShift = 22;                      // bucket of u = u >> 22
constexpr int kEaBuckets = 1 << (32 - kEaBucketShift);  // one 32-bit entry each

// One sample (CTA) of a batch launch, or one served job of a multi-job launch.
template <int ND, bool PS = false>  // PS: every temperature slot draws its own u
__device__ __forceinline__ void ea_run(const EaArgs& a, int sample) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int N = a.N, h = a.Lx >> 1, nrow = a.Ly * a.Lz;
  uint32_t* sp = reinterpret_cast<uint32_t*>(smem);           // N words
  uint8_t* bb = smem + (size_t)N * 4;                         // N bond bytes
  uint32_t* thr = reinterpret_cast<uint32_t*>(smem + (((size_t)N * 5 + 15) & ~(size_t)15));  // 96
  uint32_t* suffix = thr + 96;                                // 33 (+3 pad)
  uint32_t* ucount = suffix + 36;                             // 32 unsatisfied-bond counts
  uint8_t* tos = reinterpret_cast<uint8_t*>(ucount + 32);     // 32 temp_of_slot
  uint8_t* sot = tos + 32;                                    // 32 slot_of_temp
  int* xcount = reinterpret_cast<int*>(sot + 32);             // 32 accepted exchanges this launch
  uint32_t* lut = reinterpret_cast<uint32_t*>(xcount + 32);   // kEaBuckets entries, a byte per dE level
  uint32_t* tmask = lut + kEaBuckets;                          // per-slot u: [level][plane] slot masks

  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31;
  const int pair = sample >> 1, half = sample & 1;
  const uint32_t* gw = reinterpret_cast<const uint32_t*>(a.words + (size_t)pair * N) + half;
  const uint8_t* gb = a.bonds + (size_t)sample * N;

  // load the sample into the colour-separated layout
  for (int n = tid; n < N; n += nth) {
    const int x = n % a.Lx, row = n / a.Lx;
    const int q = ea_slot(x, row, h);
    sp[q] = gw[2 * (size_t)n];
    bb[q] = gb[n];
  }
  for (int i = tid; i < 96; i += nth) thr[i] = a.thr[i / 32][i % 32];
  if (tid < 32) {
    tos[tid] = a.temp_of_slot[sample * 32 + tid];
    xcount[tid] = 0;
  }
  __syncthreads();
  if (tid < 32) sot[tos[tid]] = (uint8_t)tid;
  // per-slot u: bit j of tmask[32 lv + p] is bit 31 - p of the level-lv
  // threshold of slot j's temperature (rebuilt whenever the slot map changes)
  auto build_tmask = [&]() {
    for (int i = tid; i < ND * 32; i += nth) {
      const int lv = i >> 5, p = i & 31;
      uint32_t wv = 0;
      for (int j = 0; j < 32; ++j) wv |= ((thr[32 * lv + tos[j]] >> (31 - p)) & 1u) << j;
      tmask[i] = wv;
    }
  };
  // bucket table: for u in [b 2^22, (b+1) 2^22 - 1], the number of thresholds
  // of a level that are <= u lies between lo = #(thr <= b 2^22) and
  // hi = #(thr <= (b+1) 2^22 - 1).  Byte lv of entry b: lo (bits 0-5) and
  // min(hi - lo, 2) (bits 6-7: 0 settled, 1 one compare, 2 binary search).
  for (int b = tid; b < kEaBuckets; b += nth) {
    const uint32_t u0 = (uint32_t)b << kEaBucketShift, u1 = u0 + ((1u << kEaBucketShift) - 1u);
    uint32_t e = 0;
    for (int lv = 0; lv < ND; ++lv) {
      const uint32_t* tl = thr + 32 * lv;
      int lo = 0, hi = 0;
#pragma unroll 8
      for (int t = 0; t < 32; ++t) {
        lo += tl[t] <= u0 ? 1 : 0;
        hi += tl[t] <= u1 ? 1 : 0;
      }
      e |= (uint32_t)(lo | ((hi - lo < 2 ? hi - lo : 2) << 6)) << (8 * lv);
    }
    lut[b] = e;
  }
  __syncthreads();
  if (tid < 32) {  // suffix[t0] = slots of temperatures t >= t0
    uint32_t v = 1u << sot[tid];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t w = __shfl_down_sync(0xffffffffu, v, o);
      if (tid + o < 32) v |= w;
    }
    suffix[tid] = v;
    if (tid == 0) suffix[32] = 0;
  }
  __syncthreads();
  if constexpr (PS) {
    build_tmask();
    __syncthreads();
  }

  const int halfN = N >> 1;
  // number of thresholds of level lv that are <= u (the accepting temperatures
  // are the ones from there up), by binary search over the 32 sorted ones
  auto search_le = [&](int lv, uint32_t u) -> int {
    const uint32_t* tl = thr + 32 * lv;
    int cnt = 0;
    cnt += (tl[cnt + 15] <= u) ? 16 : 0;
    cnt += (tl[cnt + 7] <= u) ? 8 : 0;
    cnt += (tl[cnt + 3] <= u) ? 4 : 0;
    cnt += (tl[cnt + 1] <= u) ? 2 : 0;
    cnt += (tl[cnt] <= u) ? 1 : 0;
    cnt += (cnt == 31 && tl[31] <= u) ? 1 : 0;  // all 32 thresholds <= u
    return cnt;
  };
  constexpr uint32_t kSearch = ND == 3 ? 0x808080u : 0x8080u;  // some level needs the search
  // bit-sliced count k = s0 + 2 s1 + 4 s2 (0 .. 2 ND) of the unsatisfied bonds of
  // a site's 32 replicas: s its word, bits its bond byte (bits 0..2 forward,
  // 3..5 backward, set iff J = -1), n* the neighbour words (x+, x-, y+, y-, z+, z-)
  auto unsat_count = [&](uint32_t s, uint32_t bits, uint32_t nxp, uint32_t nxm, uint32_t nyp, uint32_t nym,
                         uint32_t nzp, uint32_t nzm, uint32_t& s0, uint32_t& s1, uint32_t& s2) {
    const uint32_t ux = s ^ nxp ^ (0u - (bits & 1u));
    const uint32_t uy = s ^ nyp ^ (0u - ((bits >> 1) & 1u));
    const uint32_t vx = s ^ nxm ^ (0u - ((bits >> 3) & 1u));
    const uint32_t vy = s ^ nym ^ (0u - ((bits >> 4) & 1u));
    uint32_t uz = 0, vz = 0;
    if constexpr (ND == 3) {
      uz = s ^ nzp ^ (0u - ((bits >> 2) & 1u));
      vz = s ^ nzm ^ (0u - ((bits >> 5) & 1u));
    }
    const uint32_t x1 = ux ^ uy ^ uz, y1 = (ux & uy) | (uz & (ux ^ uy));
    const uint32_t x2 = vx ^ vy ^ vz, y2 = (vx & vy) | (vz & (vx ^ vy));
    s0 = x1 ^ x2;
    const uint32_t cc = x1 & x2;
    s1 = y1 ^ y2 ^ cc;
    s2 = (y1 & y2) | (cc & (y1 ^ y2));
  };
  // new word of a site: s its 32 replicas, bits its bond byte, n* the neighbour
  // words, u its uniform deviate (shared u) or m its site index (a u per slot)
  auto update = [&](uint32_t s, uint32_t bits, uint32_t nxp, uint32_t nxm, uint32_t nyp, uint32_t nym, uint32_t nzp,
                    uint32_t nzm, uint32_t u, uint32_t m, uint32_t sw, uint32_t c2) -> uint32_t {
    uint32_t s0, s1, s2;
    unsat_count(s, bits, nxp, nxm, nyp, nym, nzp, nzm, s0, s1, s2);
    if constexpr (PS) {
      // slot j's u has bit 31 - p = bit j of plane p (word p & 3 of the site's
      // Philox call p / 4); planes most significant first against the slots'
      // threshold bits, until no slot ties (strict u < t)
      const uint32_t k2 = ~s0 & s1 & ~s2, k1 = s0 & ~s1 & ~s2, k0 = ~(s0 | s1 | s2);
      const uint32_t l0 = ND == 3 ? k2 : k1, l1 = ND == 3 ? k1 : k0, l2 = ND == 3 ? k0 : 0u;
      uint32_t acc = ND == 3 ? (s2 | (s0 & s1)) : (s1 | s2);
      uint32_t tied = l0 | l1 | l2;
#pragma unroll 1
      for (uint32_t call = 0; call < 8u && tied != 0u; ++call) {
        const U4 P = philox10(m, sw, c2 | ((call + 1u) << 4), (uint32_t)sample, a.K);
        const uint32_t pl[4] = {P.x, P.y, P.z, P.w};
        const uint32_t* t0 = tmask + 4 * call;
#pragma unroll
        for (int jp = 0; jp < 4; ++jp) {
          uint32_t t = (l0 & t0[jp]) | (l1 & t0[32 + jp]);
          if constexpr (ND == 3) t |= l2 & t0[64 + jp];
          acc |= tied & ~pl[jp] & t;
          tied &= ~(pl[jp] ^ t);
        }
      }
      return s ^ acc;
    }
    uint32_t A[ND];
    const uint32_t e = lut[u >> kEaBucketShift];
    if (e & kSearch) {  // a bucket with two or more thresholds of some level (rare)
#pragma unroll
      for (int lv = 0; lv < ND; ++lv) A[lv] = suffix[search_le(lv, u)];
    } else {
#pragma unroll
      for (int lv = 0; lv < ND; ++lv) {
        const uint32_t by = e >> (8 * lv);
        const int lo = (int)(by & 63u);
        A[lv] = suffix[lo + (((by & 64u) && thr[32 * lv + lo] <= u) ? 1 : 0)];
      }
    }
    // dE = 4 (ND - k): k >= ND accepts always; k = ND - 1 - lv takes level lv (dE = 4 (lv + 1))
    const uint32_t k2 = ~s0 & s1 & ~s2, k1 = s0 & ~s1 & ~s2, k0 = ~(s0 | s1 | s2);
    uint32_t acc;
    if constexpr (ND == 3) {
      acc = (s2 | (s0 & s1)) | (k2 & A[0]) | (k1 & A[1]) | (k0 & A[2]);
    } else {
      acc = (s1 | s2) | (k1 & A[0]) | (k0 & A[1]);
    }
    return s ^ acc;
  };
  const bool groups4 = (a.Lx & 7) == 0;  // half-rows of whole 4-word groups
  for (int it = 0; it < a.nsweeps; ++it) {
    const uint32_t sweep = a.sweep0 + (uint32_t)it;
    for (int c = 0; c < 2; ++c) {
      const uint32_t c2 = (uint32_t)c | (3u << 1);
      if (groups4) {
        // sites m0 .. m0 + 3 of this colour: one row, words k0 .. k0 + 3 of its
        // colour-c half; the Philox call of counter m0 / 4 gives their four u
        for (int g = tid; g < (halfN >> 2); g += nth) {
          const uint32_t m0 = 4u * (uint32_t)g;
          const uint32_t row = fdiv(m0, a.div_h);
          const int k0 = (int)m0 - (int)row * h;
          const uint32_t z = ND == 3 ? fdiv(row, a.div_ly) : 0u;
          const int y = (int)row - (int)z * a.Ly;
          const int par = (c ^ (y + (int)z)) & 1;
          const int q0 = ((int)row * 2 + par) * h + k0;
          const int o0 = ((int)row * 2 + (par ^ 1)) * h;  // the row's other-parity words
          const int rym = y == 0 ? (int)row + a.Ly - 1 : (int)row - 1;
          const int ryp = y + 1 == a.Ly ? (int)row - a.Ly + 1 : (int)row + 1;
          const uint4 S = *reinterpret_cast<const uint4*>(sp + q0);
          const uint32_t B = *reinterpret_cast<const uint32_t*>(bb + q0);
          const uint4 O4 = *reinterpret_cast<const uint4*>(sp + o0 + k0);
          // the fifth other-parity word: x - 1 of the first site (even x) or
          // x + 1 of the last site (odd x), periodic in x
          const uint32_t oe = par ? sp[o0 + (k0 + 4 == h ? 0 : k0 + 4)] : sp[o0 + (k0 == 0 ? h - 1 : k0 - 1)];
          const uint4 YP = *reinterpret_cast<const uint4*>(sp + (ryp * 2 + par) * h + k0);
          const uint4 YM = *reinterpret_cast<const uint4*>(sp + (rym * 2 + par) * h + k0);
          uint4 ZP = make_uint4(0, 0, 0, 0), ZM = ZP;
          if constexpr (ND == 3) {
            const int rzm = z == 0 ? (int)row + nrow - a.Ly : (int)row - a.Ly;
            const int rzp = (int)z + 1 == a.Lz ? (int)row - nrow + a.Ly : (int)row + a.Ly;
            ZP = *reinterpret_cast<const uint4*>(sp + (rzp * 2 + par) * h + k0);
            ZM = *reinterpret_cast<const uint4*>(sp + (rzm * 2 + par) * h + k0);
          }
          const uint32_t o[4] = {O4.x, O4.y, O4.z, O4.w};
          // even x: x+1 is other-parity word k, x-1 word k-1; odd x: x-1 word k, x+1 word k+1
          const uint32_t xp0 = par ? o[1] : o[0], xm0 = par ? o[0] : oe;
          const uint32_t xp1 = par ? o[2] : o[1], xm1 = par ? o[1] : o[0];
          const uint32_t xp2 = par ? o[3] : o[2], xm2 = par ? o[2] : o[1];
          const uint32_t xp3 = par ? oe : o[3], xm3 = par ? o[3] : o[2];
          uint4 R;
          if constexpr (PS) {
            // The four sites' own Philox calls run side by side: planes 0-7 (two
            // calls per site) for every site, then, only for sites with a slot
            // still tied (about one in twenty), further calls one at a time.
            const uint32_t sv[4] = {S.x, S.y, S.z, S.w};
            const uint32_t xp[4] = {xp0, xp1, xp2, xp3}, xm[4] = {xm0, xm1, xm2, xm3};
            const uint32_t yp[4] = {YP.x, YP.y, YP.z, YP.w}, ym[4] = {YM.x, YM.y, YM.z, YM.w};
            const uint32_t zp[4] = {ZP.x, ZP.y, ZP.z, ZP.w}, zm[4] = {ZM.x, ZM.y, ZM.z, ZM.w};
            uint32_t acc[4], tied[4], la[4], lb[4];
#pragma unroll
            for (int w = 0; w < 4; ++w) {
              uint32_t s0, s1, s2;
              unsat_count(sv[w], (B >> (8 * w)) & 0xffu, xp[w], xm[w], yp[w], ym[w], zp[w], zm[w], s0, s1, s2);
              const uint32_t k2 = ~s0 & s1 & ~s2, k1 = s0 & ~s1 & ~s2, k0 = ~(s0 | s1 | s2);
              // level 0 (dE = 4) and level 1 (dE = 8) slots select threshold planes
              // 0 and 1; the remaining tied slots (3D: dE = 12) select plane 2
              la[w] = ND == 3 ? k2 : k1;
              lb[w] = ND == 3 ? k1 : k0;
              tied[w] = ND == 3 ? (k2 | k1 | k0) : (k1 | k0);
              acc[w] = ND == 3 ? (s2 | (s0 & s1)) : (s1 | s2);
            }
#pragma unroll
            for (uint32_t call = 0; call < 2u; ++call) {
              U4 P[4];
#pragma unroll
              for (int w = 0; w < 4; ++w)
                P[w] = philox10(m0 + (uint32_t)w, sweep, c2 | ((call + 1u) << 4), (uint32_t)sample, a.K);
              const uint4 T0 = *reinterpret_cast<const uint4*>(tmask + 4 * call);
              const uint4 T1 = *reinterpret_cast<const uint4*>(tmask + 32 + 4 * call);
              const uint4 T2 = ND == 3 ? *reinterpret_cast<const uint4*>(tmask + 64 + 4 * call) : T1;
              const uint32_t t0[4] = {T0.x, T0.y, T0.z, T0.w}, t1[4] = {T1.x, T1.y, T1.z, T1.w},
                             t2[4] = {T2.x, T2.y, T2.z, T2.w};
#pragma unroll
              for (int w = 0; w < 4; ++w) {
                const uint32_t pl[4] = {P[w].x, P[w].y, P[w].z, P[w].w};
#pragma unroll
                for (int jp = 0; jp < 4; ++jp) {
                  const uint32_t t = (la[w] & t0[jp]) | (~la[w] & ((lb[w] & t1[jp]) | (~lb[w] & t2[jp])));
                  acc[w] |= tied[w] & ~pl[jp] & t;
                  tied[w] &= ~(pl[jp] ^ t);
                }
              }
            }
            // Sites still tied after 8 planes (about one in ten): one call at a
            // time for the lane's first tied site, so the warp runs as many calls
            // as its busiest lane needs rather than one per site position.
            uint32_t nxt = 2u | (2u << 4) | (2u << 8) | (2u << 12);  // next call of each site, 4 bits each
#pragma unroll 1
            for (int guard = 0; guard < 24; ++guard) {
              const int w = tied[0] ? 0 : tied[1] ? 1 : tied[2] ? 2 : tied[3] ? 3 : -1;
              if (w < 0) break;
              const uint32_t call = (nxt >> (4 * w)) & 15u;
              const uint32_t lw = w == 0 ? la[0] : w == 1 ? la[1] : w == 2 ? la[2] : la[3];
              const uint32_t mw = w == 0 ? lb[0] : w == 1 ? lb[1] : w == 2 ? lb[2] : lb[3];
              uint32_t tw = w == 0 ? tied[0] : w == 1 ? tied[1] : w == 2 ? tied[2] : tied[3];
              uint32_t aw = 0;
              const U4 P = philox10(m0 + (uint32_t)w, sweep, c2 | ((call + 1u) << 4), (uint32_t)sample, a.K);
              const uint32_t pl[4] = {P.x, P.y, P.z, P.w};
              const uint4 Q0 = *reinterpret_cast<const uint4*>(tmask + 4 * call);
              const uint4 Q1 = *reinterpret_cast<const uint4*>(tmask + 32 + 4 * call);
              const uint4 Q2 = ND == 3 ? *reinterpret_cast<const uint4*>(tmask + 64 + 4 * call) : Q1;
              const uint32_t q0[4] = {Q0.x, Q0.y, Q0.z, Q0.w}, q1[4] = {Q1.x, Q1.y, Q1.z, Q1.w},
                             q2[4] = {Q2.x, Q2.y, Q2.z, Q2.w};
#pragma unroll
              for (int jp = 0; jp < 4; ++jp) {
                const uint32_t t = (lw & q0[jp]) | (~lw & ((mw & q1[jp]) | (~mw & q2[jp])));
                aw |= tw & ~pl[jp] & t;
                tw &= ~(pl[jp] ^ t);
              }
              if (call == 7u) tw = 0;  // all 32 planes compared: a tie is u = t, not below
              nxt += 1u << (4 * w);
#pragma unroll
              for (int v = 0; v < 4; ++v)
                if (v == w) {
                  acc[v] |= aw;
                  tied[v] = tw;
                }
            }
            R = make_uint4(sv[0] ^ acc[0], sv[1] ^ acc[1], sv[2] ^ acc[2], sv[3] ^ acc[3]);
          } else {
            const U4 P = philox10((uint32_t)g, sweep, c2, (uint32_t)sample, a.K);
            R.x = update(S.x, B & 0xffu, xp0, xm0, YP.x, YM.x, ZP.x, ZM.x, P.x, m0, sweep, c2);
            R.y = update(S.y, (B >> 8) & 0xffu, xp1, xm1, YP.y, YM.y, ZP.y, ZM.y, P.y, m0 + 1u, sweep, c2);
            R.z = update(S.z, (B >> 16) & 0xffu, xp2, xm2, YP.z, YM.z, ZP.z, ZM.z, P.z, m0 + 2u, sweep, c2);
            R.w = update(S.w, B >> 24, xp3, xm3, YP.w, YM.w, ZP.w, ZM.w, P.w, m0 + 3u, sweep, c2);
          }
          *reinterpret_cast<uint4*>(sp + q0) = R;
        }
      } else {
        for (int m = tid; m < halfN; m += nth) {
          const uint32_t row = fdiv((uint32_t)m, a.div_h);
          const int k = m - (int)row * h;
          const uint32_t z = ND == 3 ? fdiv(row, a.div_ly) : 0u;
          const int y = (int)row - (int)z * a.Ly;
          const int par = (c ^ (y + (int)z)) & 1;
          const int x = 2 * k + par;
          const int q = ea_slot(x, (int)row, h);
          // neighbours (other parity in the row for x; same parity in rows y +- 1, z +- 1)
          const int xm = x == 0 ? a.Lx - 1 : x - 1, xp = x + 1 == a.Lx ? 0 : x + 1;
          const int rym = y == 0 ? (int)row + a.Ly - 1 : (int)row - 1;
          const int ryp = y + 1 == a.Ly ? (int)row - a.Ly + 1 : (int)row + 1;
          uint32_t nzp = 0, nzm = 0;
          if constexpr (ND == 3) {
            const int rzm = z == 0 ? (int)row + nrow - a.Ly : (int)row - a.Ly;
            const int rzp = (int)z + 1 == a.Lz ? (int)row - nrow + a.Ly : (int)row + a.Ly;
            nzp = sp[ea_slot(x, rzp, h)];
            nzm = sp[ea_slot(x, rzm, h)];
          }
          // u of this site (one word per site, shared by the 32 replicas)
          const U4 P = PS ? U4{0u, 0u, 0u, 0u} : philox10((uint32_t)m >> 2, sweep, c2, (uint32_t)sample, a.K);
          sp[q] = update(sp[q], bb[q], sp[ea_slot(xp, (int)row, h)], sp[ea_slot(xm, (int)row, h)],
                         sp[ea_slot(x, ryp, h)], sp[ea_slot(x, rym, h)], nzp, nzm, u4_word(P, m & 3), (uint32_t)m,
                         sweep, c2);
        }
      }
      __syncthreads();
    }
    const int X = a.exchange_every;
    if (X > 0 && ((int64_t)sweep + 1) % X == 0) {
      const uint32_t e = (uint32_t)(((int64_t)sweep + 1) / X - 1);
      // unsatisfied forward bonds of every replica, bit-sliced per thread
      if (tid < 32) ucount[tid] = 0;
      __syncthreads();
      // chunks of at most 80 sites per thread keep every 8-bit counter <= 240
      for (int n0 = 0; n0 < N; n0 += 80 * nth) {  // block-uniform
        uint32_t cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        const int n1 = N < n0 + 80 * nth ? N : n0 + 80 * nth;
        for (int n = n0 + tid; n < n1; n += nth) {
          const int r = (int)fdiv((uint32_t)n >> 1, a.div_h);  // n / Lx (Lx = 2 h)
          const int x = n - r * a.Lx;
          const int z = ND == 3 ? (int)fdiv((uint32_t)r, a.div_ly) : 0;
          const int y = r - z * a.Ly;
          const int q = ea_slot(x, r, h);
          const uint32_t s = sp[q];
          const uint32_t bits = bb[q];
          const int xp = x + 1 == a.Lx ? 0 : x + 1;
          const int ryp = y + 1 == a.Ly ? r - a.Ly + 1 : r + 1;
          uint32_t w3[ND];
          w3[0] = s ^ sp[ea_slot(xp, r, h)] ^ (0u - (bits & 1u));
          w3[1] = s ^ sp[ea_slot(x, ryp, h)] ^ (0u - ((bits >> 1) & 1u));
          if constexpr (ND == 3) {
            const int rzp = z + 1 == a.Lz ? r - nrow + a.Ly : r + a.Ly;
            w3[2] = s ^ sp[ea_slot(x, rzp, h)] ^ (0u - ((bits >> 2) & 1u));
          }
#pragma unroll
          for (int d = 0; d < ND; ++d) {
            uint32_t carry = w3[d];
#pragma unroll
            for (int b = 0; b < 8; ++b) {
              const uint32_t t = cnt[b] & carry;
              cnt[b] ^= carry;
              carry = t;
            }
          }
        }
        // per-replica totals of the chunk (at most 255 per thread: ND bonds x at
        // most 80 sites).  Bit j of cnt[b] is bit b of replica j's count: byte g of
        // the eight words is an 8 x 8 bit block (row b, column k = replica 8 g + k),
        // whose transpose holds the counts of replicas 8 g .. 8 g + 7 as bytes.
        // Two counts share a word for the warp sum (at most 32 x 255 < 2^16 each).
        uint32_t pk[16];  // pk[i]: replica 2 i in bits 0-15, replica 2 i + 1 in bits 16-31
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          unsigned long long mt = 0;
#pragma unroll
          for (int b = 0; b < 8; ++b) mt |= (unsigned long long)((cnt[b] >> (8 * g)) & 0xffu) << (8 * b);
          unsigned long long t = (mt ^ (mt >> 7)) & 0x00AA00AA00AA00AAull;  // swaps within 2 x 2, 4 x 4, 8 x 8 blocks
          mt = mt ^ t ^ (t << 7);
          t = (mt ^ (mt >> 14)) & 0x0000CCCC0000CCCCull;
          mt = mt ^ t ^ (t << 14);
          t = (mt ^ (mt >> 28)) & 0x00000000F0F0F0F0ull;
          mt = mt ^ t ^ (t << 28);
#pragma unroll
          for (int i = 0; i < 4; ++i)
            pk[4 * g + i] = ((uint32_t)(mt >> (16 * i)) & 0xffu) | (((uint32_t)(mt >> (16 * i + 8)) & 0xffu) << 16);
        }
        uint32_t mine = 0;  // lane j: replica j's warp total
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const uint32_t v = __reduce_add_sync(0xffffffffu, pk[i]);
          if ((lane >> 1) == i) mine = (lane & 1) ? (v >> 16) : (v & 0xffffu);
        }
        if (mine) atomicAdd(&ucount[lane], mine);
      }
      __syncthreads();
      if (tid < 32) {
        // pairs (kk, kk+1) with kk = e mod 2, e mod 2 + 2, ...; lane tid takes kk = tid
        const int kk = tid;
        bool accept = false;
        const bool mine = kk + 1 < 32 && ((kk & 1) == (int)(e & 1));
        if (mine) {
          const int sa = sot[kk], sb = sot[kk + 1];
          const int d = (int)ucount[sb] - (int)ucount[sa];  // (E_k - E_k+1) = -2 d
          if (((a.xalways >> kk) & 1u) || d <= 0) {
            accept = true;
          } else if (d <= a.xlen[kk]) {
            const U4 P = philox10((uint32_t)kk >> 2, e, kExchange << 1, (uint32_t)sample, a.K);
            accept = u4_word(P, kk & 3) < a.xtab[a.xoff[kk] + d - 1];
          }
        }
        // every lane reads the current map before any swap is written
        const int s_self = sot[tid];
        const bool up = __shfl_up_sync(0xffffffffu, accept ? 1 : 0, 1) != 0;  // lane kk+1 learns of kk's swap
        const int s_below = __shfl_up_sync(0xffffffffu, s_self, 1);
        const int s_above = __shfl_down_sync(0xffffffffu, s_self, 1);
        int new_slot = s_self;
        if (mine && accept) new_slot = s_above;
        if (tid > 0 && up) new_slot = s_below;
        __syncwarp();
        sot[tid] = (uint8_t)new_slot;
        __syncwarp();
        tos[new_slot] = (uint8_t)tid;
        if (mine && accept) xcount[kk] += 1;
        uint32_t v = 1u << new_slot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t w = __shfl_down_sync(0xffffffffu, v, o);
          if (tid + o < 32) v |= w;
        }
        suffix[tid] = v;
      }
      __syncthreads();
      if constexpr (PS) {
        build_tmask();
        __syncthreads();
      }
    }
  }

  // write back
  uint32_t* gwo = reinterpret_cast<uint32_t*>(a.words + (size_t)pair * N) + half;
  for (int n = tid; n < N; n += nth) {
    const int x = n % a.Lx, row = n / a.Lx;
    gwo[2 * (size_t)n] = sp[ea_slot(x, row, h)];
  }
  if (tid < 32) {
    a.temp_of_slot[sample * 32 + tid] = tos[tid];
    a.xacc[sample * 32 + tid] += (unsigned long long)xcount[tid];
  }
}

// Threads per CTA: the per-slot variant keeps four sites' Philox states live
// and takes up to 128 registers, so its CTAs have at most 512 threads.
constexpr int ea_max_threads(bool ps) { return ps ? 512 : 1024; }

template <int ND, bool PS>
__global__ void __launch_bounds__(ea_max_threads(PS)) k_ea_resident(EaArgs a) { ea_run<ND, PS>(a, blockIdx.x); }

// Served jobs of one lattice size and random-number mode, one single-sample job per CTA.
template <int ND, bool PS>
__global__ void __launch_bounds__(ea_max_threads(PS)) k_ea_jobs(const EaArgs* __restrict__ list) {
  ea_run<ND, PS>(list[blockIdx.x], 0);
}

// hot start: the replica bits of site n are its 32-bit hot-start word, bit
// 31 - q = bit (m & 31) of plane q = word q & 3 of R(8 (m >> 5) + q / 4, 0, c | 1 << 1, sample)
// for the site key m = 32 (x / 64 + ceil(Lx / 64) r) + (x % 64) / 2 of row r
__global__ void k_ea_init(uint64_t* words, int Lx, int Ly, int N, int nsamples, PhiloxKeys K) {
  const int64_t total = (int64_t)nsamples * N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int sample = (int)(i / N);
    const int n = (int)(i - (int64_t)sample * N);
    const int x = n % Lx, r = n / Lx, y = r % Ly, z = r / Ly;
    const int c = (x + y + z) & 1;
    const uint32_t m = 32u * (uint32_t)((x >> 6) + ((Lx + 63) >> 6) * r) + (uint32_t)((x & 63) >> 1);  // site key
    uint32_t u = 0;
    for (uint32_t call = 0; call < 8; ++call) {
      const U4 P = philox10(8u * (m >> 5) + call, 0u, (uint32_t)c | (kInit << 1), (uint32_t)sample, K);
      const uint32_t pl[4] = {P.x, P.y, P.z, P.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) u |= ((pl[j] >> (m & 31)) & 1u) << (31 - (4 * call + j));
    }
    uint32_t* w = reinterpret_cast<uint32_t*>(words + (size_t)(sample >> 1) * N) + (sample & 1);
    w[2 * (size_t)n] = u;
  }
}

// per-replica E and M by slot: E = 2 U - nd N (U unsatisfied forward bonds), M = N - 2 (#spins -1).
// A thread adds its sites' unsatisfied-bond bits and spin bits of all 32
// replicas into bit-sliced counters (16 planes each), then the per-replica
// totals are read off the planes and reduced over the CTA.  One CTA per sample.
__device__ __forceinline__ void vadd16(uint32_t (&c)[16], uint32_t w) {
#pragma unroll
  for (int b = 0; b < 16; ++b) {
    if (!w) break;
    const uint32_t t = c[b] & w;
    c[b] ^= w;
    w = t;
  }
}

__global__ void __launch_bounds__(256) k_ea_observables(const uint64_t* words, const uint8_t* bonds, int nd, int Lx,
                                                        int Ly, int Lz, int N, long long* E, long long* M) {
  __shared__ unsigned long long su[32], sm[32];
  const int sample = blockIdx.x, tid = threadIdx.x, lane = tid & 31;
  if (tid < 32) su[tid] = sm[tid] = 0;
  __syncthreads();
  const uint32_t* w = reinterpret_cast<const uint32_t*>(words + (size_t)(sample >> 1) * N) + (sample & 1);
  const uint8_t* bb = bonds + (size_t)sample * N;
  uint32_t cu[16], cm[16];
#pragma unroll
  for (int b = 0; b < 16; ++b) cu[b] = cm[b] = 0;
  // at most 16 bits per counter: the threads of a CTA cover N <= 2^20 sites with nd <= 3 bonds each
  for (int n = tid; n < N; n += blockDim.x) {
    const int x = n % Lx, r = n / Lx, y = r % Ly, z = r / Ly;
    const uint32_t s = w[2 * (size_t)n];
    const int np[3] = {n - x + (x + 1 == Lx ? 0 : x + 1), n + ((y + 1 == Ly ? 0 : y + 1) - y) * Lx,
                       n + ((z + 1 == Lz ? 0 : z + 1) - z) * Lx * Ly};
    for (int d = 0; d < nd; ++d) vadd16(cu, s ^ w[2 * (size_t)np[d]] ^ (0u - ((bb[n] >> d) & 1u)));
    vadd16(cm, s);
  }
  for (int j = 0; j < 32; ++j) {
    unsigned int u = 0, m = 0;
#pragma unroll
    for (int b = 0; b < 16; ++b) {
      u |= ((cu[b] >> j) & 1u) << b;
      m |= ((cm[b] >> j) & 1u) << b;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      u += __shfl_xor_sync(0xffffffffu, u, o);
      m += __shfl_xor_sync(0xffffffffu, m, o);
    }
    if (lane == 0) {
      atomicAdd(&su[j], (unsigned long long)u);
      atomicAdd(&sm[j], (unsigned long long)m);
    }
  }
  __syncthreads();
  if (tid < 32) {
    E[sample * 32 + tid] = 2 * (long long)su[tid] - (long long)nd * N;
    M[sample * 32 + tid] = (long long)N - 2 * (long long)sm[tid];
  }
}

// 32 x 32 bit matrix across a warp: lane r holds row r on entry, column r
// (bit i = element (i, r)) on return.  Stage j swaps the off-diagonal j x j
// blocks between lanes r and r ^ j.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t v, int lane) {
  const uint32_t masks[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int k = 0, j = 16; k < 5; ++k, j >>= 1) {
    const uint32_t m = masks[k];
    const uint32_t o = __shfl_xor_sync(0xffffffffu, v, j);
    v = (lane & j) ? (((o >> j) & m) | (v & ~m)) : ((v & m) | ((o << j) & ~m));
  }
  return v;
}

// Overlap of replica pair p (samples 2p and 2p+1 share the 64-bit words of
// pair p): q(t) = N - 2 D(t), D(t) = sites where the two replicas at
// temperature t differ.  A warp takes 32 sites at a time, transposes both
// halves so that lane j holds slot j's bits of the 32 sites, and lane t counts
// the differing bits of the slots its temperature occupies in the two samples.
// q, q^2 and q^4 (128-bit) are accumulated per (pair, t).  One CTA per pair.
__global__ void __launch_bounds__(256) k_ea_overlap(const uint64_t* __restrict__ words,
                                                    const uint8_t* __restrict__ temp_of_slot, int N,
                                                    long long* q_last, unsigned long long* q2_sum,
                                                    unsigned long long* q4_sum) {
  __shared__ int sa[32], sb[32];
  __shared__ unsigned int D[32];
  const int p = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  if (tid < 32) {
    sa[temp_of_slot[(2 * p) * 32 + tid]] = tid;  // slot of each temperature, sample 2p
    sb[temp_of_slot[(2 * p + 1) * 32 + tid]] = tid;
    D[tid] = 0;
  }
  __syncthreads();
  const int ja = sa[lane], jb = sb[lane];  // lane t: the slots of temperature t
  const uint64_t* w = words + (size_t)p * N;
  unsigned int d = 0;
  for (int base = warp * 32; base < N; base += nwarp * 32) {
    const int n = base + lane;
    const uint64_t v = n < N ? w[n] : 0ull;  // absent sites agree
    const uint32_t pa = warp_transpose32((uint32_t)v, lane);
    const uint32_t pb = warp_transpose32((uint32_t)(v >> 32), lane);
    const uint32_t xa = __shfl_sync(0xffffffffu, pa, ja);
    const uint32_t xb = __shfl_sync(0xffffffffu, pb, jb);
    d += (unsigned int)__popc(xa ^ xb);
  }
  atomicAdd(&D[lane], d);
  __syncthreads();
  if (tid < 32) {
    const size_t i = (size_t)p * 32 + tid;
    const long long q = (long long)N - 2 * (long long)D[tid];
    const unsigned long long q2 = (unsigned long long)(q * q);
    q_last[i] = q;
    q2_sum[i] += q2;
    const unsigned long long lo = q2 * q2, hi = __umul64hi(q2, q2);
    const unsigned long long s = q4_sum[2 * i] + lo;
    q4_sum[2 * i + 1] += hi + (s < lo ? 1ull : 0ull);
    q4_sum[2 * i] = s;
  }
}

}  // namespace spn

// ---------------------------------------------------------------- the ABI

struct EaBatch {
  int nd;
  int L[3];
  int N, nsamples, exchange_every;
  bool pairs_share_bonds = false;  // samples 2p, 2p+1 have identical couplings (replica pairs)
  long long* d_qlast = nullptr;    // overlap measurement: [pairs][32] last q
  unsigned long long* d_q2 = nullptr;  // [pairs][32] sum of q^2
  unsigned long long* d_q4 = nullptr;  // [pairs][32][2] sum of q^4 (low, high 64 bits)
  int64_t nmeas = 0;
  long long* d_obs = nullptr;      // [S][64] per-replica E, M of spn_batch_energies
  bool async = false;              // device memory is stream-ordered on astream (server jobs)
  cudaStream_t astream = nullptr;
  uint64_t seed;
  double betas[32];
  uint64_t* d_words = nullptr;
  uint8_t* d_bonds = nullptr;
  uint8_t* d_tos = nullptr;
  unsigned long long* d_xacc = nullptr;
  uint32_t* d_xtab = nullptr;
  int* d_err = nullptr;
  spn::EaArgs args{};
  size_t smem = 0;
  int threads = 0;
  // disorder-parallel layout (spn_create_batch_dp): the word lattices are the
  // state; d_words holds the per-sample words only after a conversion
  bool dp = false;
  int ngroups = 0;
  uint32_t* d_dp = nullptr;   // [32 ngroups][N]
  uint32_t* d_bdp = nullptr;  // [ngroups][nd][N]
  uint32_t* d_U = nullptr;    // [32 ngroups][32]
  uint32_t* d_X = nullptr;    // [ngroups][32]
};

namespace {

int ea_fail(int code, const char* msg) {
  spn::set_last_error(msg);
  return code;
}

size_t ea_smem(int N) {
  return (((size_t)N * 5 + 15) & ~(size_t)15) + (96 + 36 + 32) * 4 + 64 + 32 * 4 + spn::kEaBuckets * 4 + 96 * 4;
}

}  // namespace

namespace {

cudaError_t ea_alloc(EaBatch* b, void* p, size_t bytes) {
  void** q = static_cast<void**>(p);
  return b->async ? cudaMallocAsync(q, bytes, b->astream) : cudaMalloc(q, bytes);
}

void ea_release(EaBatch* b, void* p) {
  if (!p) return;
  if (b->async)
    cudaFreeAsync(p, b->astream);
  else
    cudaFree(p);
}

}  // namespace

void spn_ea_free(EaBatch* b) {
  if (!b) return;
  for (void* p : {(void*)b->d_words, (void*)b->d_bonds, (void*)b->d_tos, (void*)b->d_xacc, (void*)b->d_xtab,
                  (void*)b->d_err, (void*)b->d_qlast, (void*)b->d_q2, (void*)b->d_q4, (void*)b->d_obs,
                  (void*)b->d_dp, (void*)b->d_bdp, (void*)b->d_U, (void*)b->d_X})
    ea_release(b, p);
  delete b;
}

namespace spn {

int ea_window_args(spn_ctx* h, int64_t nsweeps, EaArgs* out, size_t* smem, int* threads) {
  if (!h || !h->ea || h->ea->nsamples != 1) return SPN_E_STATE;
  if (nsweeps < 0 || h->sweeps + (uint64_t)nsweeps > 0xffffffffull) return SPN_E_ARG;
  EaBatch* b = h->ea;
  *out = b->args;
  out->sweep0 = (uint32_t)h->sweeps;
  if (out->u_per_slot) *threads = std::min(b->threads, ea_max_threads(true));
  out->nsweeps = (int)nsweeps;
  *smem = b->smem;
  if (!out->u_per_slot) *threads = b->threads;
  h->sweeps += (uint64_t)nsweeps;
  return SPN_OK;
}

int ea_job_per_sm(spn_ctx* h) {
  if (!h || !h->ea || h->ea->nsamples != 1) return 1;
  const EaBatch* b = h->ea;
  const bool ps = b->args.u_per_slot != 0;
  const int threads = ps ? std::min(b->threads, ea_max_threads(true)) : b->threads;
  auto kern = ps ? (b->nd == 2 ? k_ea_jobs<2, true> : k_ea_jobs<3, true>)
                 : (b->nd == 2 ? k_ea_jobs<2, false> : k_ea_jobs<3, false>);
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem);
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, b->smem) != cudaSuccess) cudaGetLastError();
  return n > 0 ? n : 1;
}

cudaError_t launch_ea_jobs(const EaArgs* d_list, int n, int nd, bool ps, int threads, size_t smem, cudaStream_t st) {
  auto kern = ps ? (nd == 2 ? k_ea_jobs<2, true> : k_ea_jobs<3, true>)
                 : (nd == 2 ? k_ea_jobs<2, false> : k_ea_jobs<3, false>);
  threads = std::min(threads, ea_max_threads(ps));
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<n, threads, smem, st>>>(d_list);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace spn

namespace {

// The host-side part of a batch (validation, bond bytes, exchange tables,
// thresholds): no CUDA call, so the server builds it on worker threads.
int ea_prepare(spn::EaPrep& p, int model, const int32_t* dims, int nsamples, const void* couplings,
               const double* betas, int nbeta, uint64_t seed, int exchange_every) {
  if (!dims || !couplings || !betas) return ea_fail(SPN_E_ARG, "NULL argument");
  if (model != SPN_EA3D_PMJ && model != SPN_EA2D_PMJ)
    return ea_fail(SPN_E_ARG, "batches are multi-spin coded SPN_EA3D_PMJ or SPN_EA2D_PMJ samples");
  const int nd = model == SPN_EA2D_PMJ ? 2 : 3;
  const int ext[3] = {dims[0], dims[1], nd == 3 ? dims[2] : 1};
  if (nsamples < 1) return ea_fail(SPN_E_ARG, "nsamples must be >= 1");
  if (nbeta != 32) return ea_fail(SPN_E_ARG, "the temperature ladder has exactly 32 betas (one per word bit)");
  if (exchange_every < 0) return ea_fail(SPN_E_ARG, "exchange_every must be >= 0");
  for (int d = 0; d < nd; ++d)
    if (ext[d] < 2 || (ext[d] & 1)) return ea_fail(SPN_E_ARG, "every extent must be even and >= 2");
  const int64_t N = (int64_t)ext[0] * ext[1] * ext[2];
  if (ea_smem((int)std::min<int64_t>(N, 1 << 30)) > 227 * 1024 || N > (1 << 20))
    return ea_fail(SPN_E_ARG, "a sample must fit in one CTA's shared memory (about 44,000 sites)");
  for (int t = 0; t < 32; ++t) {
    if (!(betas[t] >= 1e-6) || !std::isfinite(betas[t]))
      return ea_fail(SPN_E_ARG, "ladder betas must be finite and >= 1e-6");
    if (t > 0 && betas[t] > betas[t - 1])
      return ea_fail(SPN_E_ARG, "betas must be non-increasing (temperatures ascending)");
  }
  EaBatch* b = new (std::nothrow) EaBatch;
  if (!b) return ea_fail(SPN_E_NOMEM, "host allocation failed");
  p.b = b;
  p.model = model;
  b->nd = nd;
  for (int d = 0; d < 3; ++d) b->L[d] = ext[d];
  b->N = (int)N;
  b->nsamples = nsamples;
  b->exchange_every = exchange_every;
  b->seed = seed;
  std::memcpy(b->betas, betas, sizeof b->betas);
  // bond bytes: bit d forward J(n,d) = -1, bit 3+d backward J(n - e_d, d) = -1
  p.bb.assign((size_t)nsamples * N, 0);
  const int64_t nw = (N + 63) / 64;
  const int64_t sy = ext[0], sz = (int64_t)ext[0] * ext[1];
  const uint64_t* J = static_cast<const uint64_t*>(couplings);
  auto bit = [](const uint64_t* Jd, int64_t i) { return (uint32_t)((Jd[i >> 6] >> (i & 63)) & 1u); };
  for (int s = 0; s < nsamples; ++s) {
    const uint64_t* Js = J + (int64_t)s * nd * nw;
    uint8_t* out = &p.bb[(size_t)s * N];
    int64_t n = 0;
    for (int z = 0; z < ext[2]; ++z)
      for (int y = 0; y < ext[1]; ++y)
        for (int x = 0; x < ext[0]; ++x, ++n) {
          const int64_t back[3] = {x == 0 ? n + ext[0] - 1 : n - 1, y == 0 ? n + (ext[1] - 1) * sy : n - sy,
                                   z == 0 ? n + (ext[2] - 1) * sz : n - sz};
          uint32_t v = 0;
          for (int d = 0; d < nd; ++d) v |= (bit(Js + d * nw, n) << d) | (bit(Js + d * nw, back[d]) << (3 + d));
          out[n] = (uint8_t)v;
        }
  }
  b->pairs_share_bonds = nsamples % 2 == 0;
  for (int q = 0; b->pairs_share_bonds && q < nsamples / 2; ++q)
    b->pairs_share_bonds = std::memcmp(&p.bb[(size_t)(2 * q) * N], &p.bb[(size_t)(2 * q + 1) * N], (size_t)N) == 0;
  // exchange tables: pair k, d = 1 .. len: floor(exp((b_k - b_k+1) * (-2d)) 2^32)
  spn::EaArgs& A = b->args;
  // with replica exchange every slot draws its own u (the exchange rule needs
  // independent replicas); without it the slots share one u per site
  A.u_per_slot = exchange_every > 0 ? 1 : 0;
  A.xalways = 0;
  for (int k = 0; k < 31; ++k) {
    const double db = betas[k] - betas[k + 1];
    A.xoff[k] = (int)p.tab.size();
    A.xlen[k] = 0;
    if (db == 0.0) {
      A.xalways |= 1u << k;
      continue;
    }
    for (int64_t d = 1;; ++d) {
      const double D = db * (double)(-2 * d);
      const uint64_t t = (uint64_t)std::floor(std::exp(D) * 4294967296.0);
      if (t == 0) break;
      p.tab.push_back((uint32_t)t);
      if (p.tab.size() > (size_t)1 << 22) return ea_fail(SPN_E_ARG, "ladder spacing too small for the exchange tables");
    }
    A.xlen[k] = (int)p.tab.size() - A.xoff[k];
  }
  A.xoff[31] = (int)p.tab.size();
  A.xlen[31] = 0;
  if (p.tab.empty()) p.tab.push_back(0);
  for (int q = 1; q <= 3; ++q)
    for (int t = 0; t < 32; ++t) {
      const uint64_t v = spn::boltzmann_threshold(betas[t], 4 * q);
      A.thr[q - 1][t] = (uint32_t)std::min<uint64_t>(v, 0xffffffffull);  // < 2^32 for beta >= 1e-6
    }
  return SPN_OK;
}

// The device part: memory, copies and the hot start, ordered on st.  async:
// nothing waits for the device (server admissions); otherwise the call
// returns with the batch initialised.  Takes the batch out of p.
int ea_upload(spn_handle* out, spn::EaPrep& p, cudaStream_t st, bool async) {
  *out = nullptr;
  EaBatch* b = p.b;
  p.b = nullptr;
  b->async = async;
  b->astream = st;
  auto bail = [&](int code, const char* msg) {
    spn_ea_free(b);
    return ea_fail(code, msg);
  };
  const int nsamples = b->nsamples, pairs = (nsamples + 1) / 2;
  const int64_t N = b->N;
  spn::EaArgs& A = b->args;
  cudaError_t e;
  if (ea_alloc(b, &b->d_words, (size_t)pairs * N * 8) != cudaSuccess || ea_alloc(b, &b->d_bonds, p.bb.size()) ||
      ea_alloc(b, &b->d_tos, (size_t)nsamples * 32) || ea_alloc(b, &b->d_xacc, (size_t)nsamples * 32 * 8) ||
      ea_alloc(b, &b->d_xtab, p.tab.size() * 4) || ea_alloc(b, &b->d_err, 4) ||
      ea_alloc(b, &b->d_obs, (size_t)nsamples * 64 * 8))
    return bail(SPN_E_NOMEM, "allocating the batch");
  std::vector<uint8_t> tos((size_t)nsamples * 32);
  for (size_t i = 0; i < tos.size(); ++i) tos[i] = (uint8_t)(i % 32);
  // host-to-device copies from pageable memory return once the data is staged
  if (cudaMemcpyAsync(b->d_bonds, p.bb.data(), p.bb.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(b->d_tos, tos.data(), tos.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(b->d_xtab, p.tab.data(), p.tab.size() * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(b->d_xacc, 0, (size_t)nsamples * 32 * 8, st) != cudaSuccess ||
      cudaMemsetAsync(b->d_words, 0, (size_t)pairs * N * 8, st) != cudaSuccess ||
      cudaMemsetAsync(b->d_err, 0, 4, st) != cudaSuccess)
    return bail(SPN_E_CUDA, "copying the batch to the device");
  const spn::PhiloxKeys K = spn::philox_keys(b->seed);
  spn::k_ea_init<<<(int)std::max<int64_t>(1, std::min<int64_t>((int64_t)nsamples * N / 256 + 1, spn::device_sm_count() * 32)), 256, 0, st>>>(
      b->d_words, b->L[0], b->L[1], (int)N, nsamples, K);
  spn::count_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return bail(SPN_E_CUDA, cudaGetErrorString(e));
  if (!async && (e = cudaStreamSynchronize(st)) != cudaSuccess) return bail(SPN_E_CUDA, cudaGetErrorString(e));
  A.words = b->d_words;
  A.bonds = b->d_bonds;
  A.temp_of_slot = b->d_tos;
  A.xacc = b->d_xacc;
  A.xtab = b->d_xtab;
  A.nd = b->nd;
  A.Lx = b->L[0];
  A.Ly = b->L[1];
  A.Lz = b->L[2];
  A.N = (int)N;
  A.div_h = spn::fastdiv((uint32_t)(b->L[0] / 2));
  A.div_ly = spn::fastdiv((uint32_t)b->L[1]);
  A.exchange_every = b->exchange_every;
  A.nsamples = nsamples;
  A.K = K;
  A.err = b->d_err;
  b->smem = ea_smem((int)N);
  b->threads = N >= 16384 ? 1024 : (N >= 4096 ? 512 : 256);
  spn_ctx* h = new (std::nothrow) spn_ctx;
  if (!h) return bail(SPN_E_NOMEM, "host allocation failed");
  h->model = p.model;
  h->seed = b->seed;
  h->ea = b;
  h->st = st;
  *out = h;
  return SPN_OK;
}

int create_batch(spn_handle* out, int model, const int32_t* dims, int nsamples, const void* couplings,
                 const double* betas, int nbeta, uint64_t seed, int exchange_every, cudaStream_t st, bool async) {
  if (!out) return ea_fail(SPN_E_ARG, "NULL argument");
  *out = nullptr;
  spn::EaPrep p;
  const int rc = ea_prepare(p, model, dims, nsamples, couplings, betas, nbeta, seed, exchange_every);
  if (rc) return rc;
  return ea_upload(out, p, st, async);
}

}  // namespace

namespace spn {

EaPrep::~EaPrep() { spn_ea_free(b); }

int ea_prepare_single(EaPrep& p, int model, const int32_t* dims, const void* couplings, const double* betas,
                      uint64_t seed, int exchange_every) {
  return ea_prepare(p, model, dims, 1, couplings, betas, 32, seed, exchange_every);
}

int ea_upload_async(spn_handle* out, EaPrep& p, cudaStream_t st) { return ea_upload(out, p, st, true); }

}  // namespace spn

namespace {

// The per-sample words of a disorder-parallel batch into d_words (bit t =
// temperature t, 2 samples per uint64), ordered on the handle's stream.
cudaError_t dp_to_words(spn_ctx* h) {
  EaBatch* b = h->ea;
  return spn::launch_dp_to_words(b->d_dp, b->d_words, b->L[0], b->N, b->nsamples, b->ngroups, h->st);
}

int dp_sweep(spn_ctx* h, int64_t nsweeps) {
  EaBatch* b = h->ea;
  spn::EaDpArgs A{};
  A.dp = b->d_dp;
  A.bdp = b->d_bdp;
  A.U = b->d_U;
  A.nd = b->nd;
  A.Lx = b->L[0];
  A.Ly = b->L[1];
  A.Lz = b->L[2];
  A.N = b->N;
  A.div_h = spn::fastdiv((uint32_t)(b->L[0] / 2));
  A.div_ly = spn::fastdiv((uint32_t)b->L[1]);
  for (int t = 0; t < 32; ++t)
    for (int lv = 0; lv < 3; ++lv) A.thr[t][lv] = b->args.thr[lv][t];
  A.K = b->args.K;
  spn::EaDpExchangeArgs XA{};
  XA.U = b->d_U;
  XA.X = b->d_X;
  XA.xacc = b->d_xacc;
  XA.xtab = b->d_xtab;
  for (int k = 0; k < 32; ++k) {
    XA.xoff[k] = b->args.xoff[k];
    XA.xlen[k] = b->args.xlen[k];
  }
  XA.xalways = b->args.xalways;
  XA.nsamples = b->nsamples;
  XA.K = b->args.K;
  const int X = b->exchange_every;
  const int threads = b->N >= 16384 ? 1024 : (b->N >= 4096 ? 512 : 256);
  int64_t done = 0;
  while (done < nsweeps) {  // one launch per exchange interval (at most 2000 sweeps)
    const uint64_t sw = h->sweeps + (uint64_t)done;
    int64_t n = nsweeps - done;
    if (X > 0) n = std::min<int64_t>(n, X - (int64_t)(sw % (uint64_t)X));
    n = std::min<int64_t>(n, 2000);
    A.sweep0 = (uint32_t)sw;
    A.nsweeps = (int)n;
    A.need_u = X > 0 && (sw + (uint64_t)n) % (uint64_t)X == 0;
    cudaError_t e = spn::launch_dp_sweep(A, 32 * b->ngroups, threads, h->st);
    if (e == cudaSuccess && A.need_u) {
      XA.e = (uint32_t)((sw + (uint64_t)n) / (uint64_t)X - 1);
      e = spn::launch_dp_exchange(XA, b->ngroups, h->st);
      if (e == cudaSuccess) e = spn::launch_dp_swap(b->d_dp, b->d_X, b->N, b->ngroups, h->st);
    }
    if (e != cudaSuccess) {
      h->sweeps += (uint64_t)done;
      return ea_fail(SPN_E_CUDA, cudaGetErrorString(e));
    }
    done += n;
  }
  h->sweeps += (uint64_t)nsweeps;
  return SPN_OK;
}

}  // namespace

extern "C" {

int spn_create_batch_dp(spn_handle* out, int model, const int32_t* dims, int nsamples, const void* couplings,
                        const double* betas, int nbeta, uint64_t seed, int exchange_every) {
  if (!out) return ea_fail(SPN_E_ARG, "NULL argument");
  *out = nullptr;
  if (dims && dims[0] % 8) return ea_fail(SPN_E_ARG, "the disorder-parallel layout needs Lx a multiple of 8");
  const int rc = create_batch(out, model, dims, nsamples, couplings, betas, nbeta, seed, exchange_every, nullptr, false);
  if (rc) return rc;
  spn_ctx* h = *out;
  EaBatch* b = h->ea;
  b->dp = true;
  b->ngroups = 2 * ((nsamples + 63) / 64);
  b->args.u_per_slot = 0;
  const size_t N = (size_t)b->N, nwl = (size_t)32 * b->ngroups;
  const size_t nw = (N + 63) / 64;
  uint64_t* d_packed = nullptr;
  auto bail = [&](int code, const char* msg) {
    if (d_packed) cudaFree(d_packed);
    spn_destroy(h);
    *out = nullptr;
    return ea_fail(code, msg);
  };
  if (cudaMalloc(&b->d_dp, nwl * N * 4) != cudaSuccess || cudaMalloc(&b->d_bdp, (size_t)b->ngroups * b->nd * N * 4) ||
      cudaMalloc(&b->d_U, nwl * 32 * 4) != cudaSuccess || cudaMalloc(&b->d_X, (size_t)b->ngroups * 32 * 4) ||
      cudaMalloc(&d_packed, (size_t)nsamples * b->nd * nw * 8) != cudaSuccess)
    return bail(SPN_E_NOMEM, "allocating the disorder-parallel batch");
  cudaError_t e = cudaMemcpy(d_packed, couplings, (size_t)nsamples * b->nd * nw * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->d_X, 0, (size_t)b->ngroups * 32 * 4);
  if (e == cudaSuccess) e = spn::launch_dp_bonds(d_packed, b->d_bdp, b->nd, b->L[0], b->N, nsamples, b->ngroups, h->st);
  // the hot start of the per-sample words, in the word lattices
  if (e == cudaSuccess)
    e = spn::launch_dp_from_words(b->d_words, b->d_dp, b->L[0], b->N, nsamples, b->ngroups, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return bail(SPN_E_CUDA, cudaGetErrorString(e));
  cudaFree(d_packed);
  return SPN_OK;
}

int spn_create_batch(spn_handle* out, int model, const int32_t* dims, int nsamples, const void* couplings,
                     const double* betas, int nbeta, uint64_t seed, int exchange_every) {
  return create_batch(out, model, dims, nsamples, couplings, betas, nbeta, seed, exchange_every, nullptr, false);
}

int spn_batch_set_u_per_slot(spn_handle h, int32_t on) {
  if (!h || !h->ea) return ea_fail(SPN_E_STATE, "not a batch handle");
  if (on != 0 && on != 1) return ea_fail(SPN_E_ARG, "on must be 0 or 1");
  if (h->ea->dp) return ea_fail(SPN_E_STATE, "a disorder-parallel batch draws its own random numbers");
  h->ea->args.u_per_slot = on;
  return SPN_OK;
}

int spn_batch_sweep(spn_handle h, int64_t nsweeps) {
  if (!h || !h->ea) return ea_fail(SPN_E_STATE, "not a batch handle");
  if (nsweeps < 0) return ea_fail(SPN_E_ARG, "nsweeps must be >= 0");
  EaBatch* b = h->ea;
  if (h->sweeps + (uint64_t)nsweeps > 0xffffffffull) return ea_fail(SPN_E_ARG, "sweep counter would exceed 2^32");
  if (b->dp) return dp_sweep(h, nsweeps);
  auto kern = b->args.u_per_slot ? (b->nd == 2 ? spn::k_ea_resident<2, true> : spn::k_ea_resident<3, true>)
                                  : (b->nd == 2 ? spn::k_ea_resident<2, false> : spn::k_ea_resident<3, false>);
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem);
  const int threads = std::min(b->threads, spn::ea_max_threads(b->args.u_per_slot != 0));
  int64_t done = 0;
  while (done < nsweeps) {  // bounded launches keep each kernel well under a second
    const int n = (int)std::min<int64_t>(nsweeps - done, 2000);
    spn::EaArgs a = b->args;
    a.sweep0 = (uint32_t)(h->sweeps + done);
    a.nsweeps = n;
    kern<<<b->nsamples, threads, b->smem, h->st>>>(a);
    spn::count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ea_fail(SPN_E_CUDA, cudaGetErrorString(e));
    done += n;
  }
  h->sweeps += (uint64_t)nsweeps;
  return SPN_OK;
}

int spn_batch_get_words(spn_handle h, uint32_t* out, size_t count) {
  if (!h || !h->ea || !out) return ea_fail(SPN_E_ARG, "bad arguments");
  EaBatch* b = h->ea;
  if (count != (size_t)b->nsamples * b->N) return ea_fail(SPN_E_ARG, "count must be nsamples * N");
  const int pairs = (b->nsamples + 1) / 2;
  std::vector<uint64_t> w((size_t)pairs * b->N);
  if (b->dp && dp_to_words(h) != cudaSuccess) return ea_fail(SPN_E_CUDA, "converting the word lattices");
  if (cudaStreamSynchronize(h->st) != cudaSuccess ||
      cudaMemcpy(w.data(), b->d_words, w.size() * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
    return ea_fail(SPN_E_CUDA, "reading the words");
  for (int s = 0; s < b->nsamples; ++s)
    for (int n = 0; n < b->N; ++n)
      out[(size_t)s * b->N + n] = (uint32_t)(w[(size_t)(s >> 1) * b->N + n] >> (32 * (s & 1)));
  return SPN_OK;
}

int spn_batch_set_words(spn_handle h, const uint32_t* in, size_t count) {
  if (!h || !h->ea || !in) return ea_fail(SPN_E_ARG, "bad arguments");
  EaBatch* b = h->ea;
  if (count != (size_t)b->nsamples * b->N) return ea_fail(SPN_E_ARG, "count must be nsamples * N");
  const int pairs = (b->nsamples + 1) / 2;
  std::vector<uint64_t> w((size_t)pairs * b->N, 0);
  for (int s = 0; s < b->nsamples; ++s)
    for (int n = 0; n < b->N; ++n)
      w[(size_t)(s >> 1) * b->N + n] |= (uint64_t)in[(size_t)s * b->N + n] << (32 * (s & 1));
  if (cudaStreamSynchronize(h->st) != cudaSuccess ||
      cudaMemcpy(b->d_words, w.data(), w.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess)
    return ea_fail(SPN_E_CUDA, "writing the words");
  if (b->dp && (spn::launch_dp_from_words(b->d_words, b->d_dp, b->L[0], b->N, b->nsamples, b->ngroups, h->st) !=
                    cudaSuccess ||
                cudaStreamSynchronize(h->st) != cudaSuccess))
    return ea_fail(SPN_E_CUDA, "converting the words to word lattices");
  return SPN_OK;
}

int spn_batch_get_slots(spn_handle h, uint8_t* temp_of_slot, size_t count) {
  if (!h || !h->ea || !temp_of_slot) return ea_fail(SPN_E_ARG, "bad arguments");
  if (count != (size_t)h->ea->nsamples * 32) return ea_fail(SPN_E_ARG, "count must be nsamples * 32");
  if (cudaStreamSynchronize(h->st) != cudaSuccess ||
      cudaMemcpy(temp_of_slot, h->ea->d_tos, count, cudaMemcpyDeviceToHost) != cudaSuccess)
    return ea_fail(SPN_E_CUDA, "reading the slot maps");
  return SPN_OK;
}

int spn_batch_set_slots(spn_handle h, const uint8_t* temp_of_slot, size_t count) {
  if (!h || !h->ea || !temp_of_slot) return ea_fail(SPN_E_ARG, "bad arguments");
  if (count != (size_t)h->ea->nsamples * 32) return ea_fail(SPN_E_ARG, "count must be nsamples * 32");
  for (int s = 0; s < h->ea->nsamples; ++s) {
    uint32_t seen = 0;
    for (int j = 0; j < 32; ++j) {
      const uint8_t t = temp_of_slot[s * 32 + j];
      if (t >= 32 || ((seen >> t) & 1u)) return ea_fail(SPN_E_ARG, "each sample's map must be a permutation of 0..31");
      if (h->ea->dp && t != j)
        return ea_fail(SPN_E_STATE, "a disorder-parallel batch keeps bit t at temperature t (identity maps only)");
      seen |= 1u << t;
    }
  }
  if (cudaStreamSynchronize(h->st) != cudaSuccess ||
      cudaMemcpy(h->ea->d_tos, temp_of_slot, count, cudaMemcpyHostToDevice) != cudaSuccess)
    return ea_fail(SPN_E_CUDA, "writing the slot maps");
  return SPN_OK;
}

int spn_batch_energies(spn_handle h, int64_t* E, int64_t* M, size_t count) {
  if (!h || !h->ea || !E || !M) return ea_fail(SPN_E_ARG, "bad arguments");
  EaBatch* b = h->ea;
  if (count != (size_t)b->nsamples * 32) return ea_fail(SPN_E_ARG, "count must be nsamples * 32");
  long long* dE = b->d_obs;
  long long* dM = b->d_obs + count;
  if (b->dp && dp_to_words(h) != cudaSuccess) return ea_fail(SPN_E_CUDA, "converting the word lattices");
  spn::k_ea_observables<<<b->nsamples, 256, 0, h->st>>>(b->d_words, b->d_bonds, b->nd, b->L[0], b->L[1], b->L[2], b->N, dE,
                                                       dM);
  spn::count_launches(1);
  cudaError_t e = cudaMemcpyAsync(E, dE, count * 8, cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(M, dM, count * 8, cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  return e == cudaSuccess ? SPN_OK : ea_fail(SPN_E_CUDA, cudaGetErrorString(e));
}

int spn_batch_exchange_counts(spn_handle h, int64_t* acc, size_t count) {
  if (!h || !h->ea || !acc) return ea_fail(SPN_E_ARG, "bad arguments");
  if (count != (size_t)h->ea->nsamples * 32) return ea_fail(SPN_E_ARG, "count must be nsamples * 32");
  if (cudaStreamSynchronize(h->st) != cudaSuccess ||
      cudaMemcpy(acc, h->ea->d_xacc, count * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
    return ea_fail(SPN_E_CUDA, "reading the exchange counts");
  return SPN_OK;
}

int spn_batch_measure_overlap(spn_handle h) {
  if (!h || !h->ea) return ea_fail(SPN_E_STATE, "not a batch handle");
  EaBatch* b = h->ea;
  if (!b->pairs_share_bonds)
    return ea_fail(SPN_E_STATE, "overlaps need an even number of samples with samples 2p, 2p+1 sharing couplings");
  const size_t n = (size_t)b->nsamples / 2 * 32;
  if (!b->d_qlast) {
    if (ea_alloc(b, &b->d_qlast, n * 8) != cudaSuccess || ea_alloc(b, &b->d_q2, n * 8) != cudaSuccess ||
        ea_alloc(b, &b->d_q4, n * 16) != cudaSuccess)
      return ea_fail(SPN_E_NOMEM, "cudaMalloc(overlap)");
    if (cudaMemsetAsync(b->d_qlast, 0, n * 8, h->st) != cudaSuccess ||
        cudaMemsetAsync(b->d_q2, 0, n * 8, h->st) != cudaSuccess ||
        cudaMemsetAsync(b->d_q4, 0, n * 16, h->st) != cudaSuccess)
      return ea_fail(SPN_E_CUDA, "clearing the overlap sums");
  }
  if (b->dp && dp_to_words(h) != cudaSuccess) return ea_fail(SPN_E_CUDA, "converting the word lattices");
  spn::k_ea_overlap<<<b->nsamples / 2, 256, 0, h->st>>>(b->d_words, b->d_tos, b->N, b->d_qlast, b->d_q2, b->d_q4);
  spn::count_launches(1);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return ea_fail(SPN_E_CUDA, cudaGetErrorString(e));
  b->nmeas += 1;
  return SPN_OK;
}

int spn_batch_overlap(spn_handle h, int64_t* nmeas, int64_t* q_last, uint64_t* q2_sum, uint64_t* q4_sum,
                      size_t count) {
  if (!h || !h->ea) return ea_fail(SPN_E_STATE, "not a batch handle");
  EaBatch* b = h->ea;
  if (count != (size_t)b->nsamples / 2 * 32) return ea_fail(SPN_E_ARG, "count must be nsamples / 2 * 32");
  if (nmeas) *nmeas = b->nmeas;
  if (cudaStreamSynchronize(h->st) != cudaSuccess) return ea_fail(SPN_E_CUDA, "synchronising");
  if (!b->d_qlast) {  // nothing measured yet
    if (q_last) std::memset(q_last, 0, count * 8);
    if (q2_sum) std::memset(q2_sum, 0, count * 8);
    if (q4_sum) std::memset(q4_sum, 0, count * 16);
    return SPN_OK;
  }
  if ((q_last && cudaMemcpy(q_last, b->d_qlast, count * 8, cudaMemcpyDeviceToHost) != cudaSuccess) ||
      (q2_sum && cudaMemcpy(q2_sum, b->d_q2, count * 8, cudaMemcpyDeviceToHost) != cudaSuccess) ||
      (q4_sum && cudaMemcpy(q4_sum, b->d_q4, count * 16, cudaMemcpyDeviceToHost) != cudaSuccess))
    return ea_fail(SPN_E_CUDA, "reading the overlaps");
  return SPN_OK;
}

int spn_batch_overlap_reset(spn_handle h) {
  if (!h || !h->ea) return ea_fail(SPN_E_STATE, "not a batch handle");
  EaBatch* b = h->ea;
  if (cudaStreamSynchronize(h->st) != cudaSuccess) return ea_fail(SPN_E_CUDA, "synchronising");
  b->nmeas = 0;
  if (b->d_qlast) {
    const size_t n = (size_t)b->nsamples / 2 * 32;
    if (cudaMemset(b->d_qlast, 0, n * 8) != cudaSuccess || cudaMemset(b->d_q2, 0, n * 8) != cudaSuccess ||
        cudaMemset(b->d_q4, 0, n * 16) != cudaSuccess)
      return ea_fail(SPN_E_CUDA, "clearing the overlap sums");
  }
  return SPN_OK;
}

}  // extern "C"
