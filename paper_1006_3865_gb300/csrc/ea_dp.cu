// Disorder-parallel multi-spin coded +-J Edwards-Anderson batches with replica
// exchange (Weigel, Sec. 4: many disorder realisations updated at once with
// asynchronous multi-spin coding, the bits of a word being different systems).
//
// Layout.  A word lattice holds 32 samples (the bits) at one temperature t; the
// samples of group g are s = 64 (g >> 1) + 2 j + (g & 1), j the bit (so the two
// replicas 2p, 2p + 1 of a realisation never share a word).  Word lattice
// 32 g + t is N uint32 words in colour-separated row order (row r = y + Ly z:
// the Lx / 2 even-x words, then the odd-x words), the order a CTA keeps in
// shared memory.  Bonds: per group and direction, one word per site, bit j set
// iff J(n, d) = -1 for sample j (forward bonds only; a site's backward bonds
// are its neighbours' forward bonds).
//
// Sweep.  One CTA per word lattice holds it in shared memory for the sweeps up
// to the next exchange.  A thread updates four consecutive same-colour sites of
// a row: the 2 ND neighbour words XOR the bond words give the unsatisfied
// bonds of the 32 samples, a bit-sliced adder counts them (k), and the one
// Philox call of the four sites gives their u, shared by the 32 samples: a
// sample flips iff k >= ND - c, c = the number of the temperature's thresholds
// floor(exp(-beta dE) 2^32) (dE = 4, 8, 12) above u.  The thresholds of one
// word lattice are three scalars, so the decision costs a few compares.
//
// Exchange.  After the last sweep before an exchange step the CTA counts every
// sample's unsatisfied forward bonds; one warp per group then takes the
// decisions of the step's temperature pairs (the exchange rule of
// Hukushima and Nemoto, with the host-built tables of floor(exp(dbeta dE) 2^32)),
// and a third kernel swaps the accepted samples' configurations between the two
// word lattices of each pair (bit j of every word).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "fastdiv.cuh"
#include "philox.cuh"
#include "spn_internal.h"

namespace spn {
namespace {

__device__ __forceinline__ int dp_sample(int g, int j) { return 64 * (g >> 1) + 2 * j + (g & 1); }

// colour-separated index of site n = x + Lx r (r = y + Ly z)
__device__ __forceinline__ int dp_q(int n, int Lx) {
  const int r = n / Lx, x = n - r * Lx;
  return (r * 2 + (x & 1)) * (Lx >> 1) + (x >> 1);
}

// 32 x 32 bit matrix across a warp: lane r holds row r on entry, column r
// (bit i = element (i, r)) on return.
__device__ __forceinline__ uint32_t dp_transpose32(uint32_t v, int lane) {
  const uint32_t masks[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int k = 0, j = 16; k < 5; ++k, j >>= 1) {
    const uint32_t m = masks[k];
    const uint32_t o = __shfl_xor_sync(0xffffffffu, v, j);
    v = (lane & j) ? (((o >> j) & m) | (v & ~m)) : ((v & m) | ((o << j) & ~m));
  }
  return v;
}

// Per-sample words (uint32 halves of the [pair][N] uint64 array, bit t =
// temperature t, site order) to and from the word lattices.
__global__ void k_dp_from_words(const uint32_t* __restrict__ pairs, uint32_t* __restrict__ dp, int Lx, int N,
                                int nsamples, int ngroups) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < (int64_t)ngroups * N; u += nwarps) {
    const int g = (int)(u / N), n = (int)(u - (int64_t)g * N);
    const int s = dp_sample(g, lane);
    const uint32_t w = s < nsamples ? pairs[2 * ((size_t)(s >> 1) * N + n) + (s & 1)] : 0u;
    dp[(size_t)(32 * g + lane) * N + dp_q(n, Lx)] = dp_transpose32(w, lane);
  }
}

__global__ void k_dp_to_words(const uint32_t* __restrict__ dp, uint32_t* __restrict__ pairs, int Lx, int N,
                              int nsamples, int ngroups) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < (int64_t)ngroups * N; u += nwarps) {
    const int g = (int)(u / N), n = (int)(u - (int64_t)g * N);
    const uint32_t w = dp_transpose32(dp[(size_t)(32 * g + lane) * N + dp_q(n, Lx)], lane);  // lane j: sample j
    const int s = dp_sample(g, lane);
    if (s < nsamples) pairs[2 * ((size_t)(s >> 1) * N + n) + (s & 1)] = w;
  }
}

// Bond words from the per-sample bit-packed couplings [sample][d][ceil(N/64)].
__global__ void k_dp_bonds(const uint64_t* __restrict__ packed, uint32_t* __restrict__ bdp, int nd, int Lx, int N,
                           int nsamples, int ngroups) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (N + 63) / 64;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < (int64_t)ngroups * nd * N;
       u += nwarps) {
    const int gd = (int)(u / N), n = (int)(u - (int64_t)gd * N);
    const int g = gd / nd, d = gd - g * nd;
    const int s = dp_sample(g, lane);
    const bool neg = s < nsamples && ((packed[((int64_t)s * nd + d) * nw + (n >> 6)] >> (n & 63)) & 1ull);
    const uint32_t w = __ballot_sync(0xffffffffu, neg);
    if (lane == 0) bdp[(size_t)gd * N + dp_q(n, Lx)] = w;
  }
}

__device__ __forceinline__ uint4 ldg4(const uint32_t* p) { return __ldg(reinterpret_cast<const uint4*>(p)); }

template <int ND>
__global__ void __launch_bounds__(1024) k_dp_sweep(const __grid_constant__ EaDpArgs a) {
  extern __shared__ __align__(16) uint32_t sp[];  // the word lattice, N words
  __shared__ unsigned int ucount[32];
  const int N = a.N, h = a.Lx >> 1, nrow = a.Ly * a.Lz, halfN = N >> 1;
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31;
  const int wl = blockIdx.x, g = wl >> 5, t = wl & 31;
  uint32_t* gw = a.dp + (size_t)wl * N;
  const uint32_t* bx = a.bdp + (size_t)g * ND * N;
  const uint32_t* by = bx + N;
  const uint32_t* bz = bx + (ND == 3 ? 2 * N : N);
  for (int i = tid; i < (N >> 2); i += nth) reinterpret_cast<uint4*>(sp)[i] = reinterpret_cast<const uint4*>(gw)[i];
  if (tid < 32) ucount[tid] = 0;
  __syncthreads();
  const uint32_t t0 = a.thr[t][0], t1 = a.thr[t][1], t2 = a.thr[t][2];
  const uint32_t stream = (uint32_t)(32 * g + t);

  // new word of one site: s its 32 samples, n* the neighbour words (x+, x-,
  // y+, y-, z+, z-), f* its forward and b* its backward bond words, u its number
  auto update = [&](uint32_t s, uint32_t nxp, uint32_t nxm, uint32_t nyp, uint32_t nym, uint32_t nzp, uint32_t nzm,
                    uint32_t fx, uint32_t bxw, uint32_t fy, uint32_t byw, uint32_t fz, uint32_t bzw,
                    uint32_t u) -> uint32_t {
    const uint32_t ux = s ^ nxp ^ fx, vx = s ^ nxm ^ bxw, uy = s ^ nyp ^ fy, vy = s ^ nym ^ byw;
    uint32_t uz = 0, vz = 0;
    if constexpr (ND == 3) {
      uz = s ^ nzp ^ fz;
      vz = s ^ nzm ^ bzw;
    }
    // bit-sliced count of unsatisfied bonds k = s0 + 2 s1 + 4 s2 (0 .. 2 ND)
    const uint32_t x1 = ux ^ uy ^ uz, y1 = (ux & uy) | (uz & (ux ^ uy));
    const uint32_t x2 = vx ^ vy ^ vz, y2 = (vx & vy) | (vz & (vx ^ vy));
    const uint32_t s0 = x1 ^ x2, cc = x1 & x2;
    const uint32_t s1 = y1 ^ y2 ^ cc, s2 = (y1 & y2) | (cc & (y1 ^ y2));
    // dE = 4 (ND - k): accepted iff k >= ND - c, c = thresholds above u (a prefix: t0 >= t1 >= t2)
    const int c = (u < t0 ? 1 : 0) + (u < t1 ? 1 : 0) + (ND == 3 && u < t2 ? 1 : 0);
    const uint32_t ge1 = s0 | s1 | s2, ge2 = s1 | s2, ge3 = s2 | (s1 & s0);
    uint32_t acc;
    if constexpr (ND == 3) {
      acc = c == 0 ? ge3 : c == 1 ? ge2 : c == 2 ? ge1 : 0xffffffffu;
    } else {
      acc = c == 0 ? ge2 : c == 1 ? ge1 : 0xffffffffu;
    }
    return s ^ acc;
  };

  for (int it = 0; it < a.nsweeps; ++it) {
    const uint32_t sweep = a.sweep0 + (uint32_t)it;
    for (int c = 0; c < 2; ++c) {
      const uint32_t c2 = (uint32_t)c | (3u << 1);
      // sites m0 .. m0 + 3 of this colour: one row, words k0 .. k0 + 3 of its
      // colour-c half; the Philox call of counter m0 / 4 gives their four u
      for (int gq = tid; gq < (halfN >> 2); gq += nth) {
        const uint32_t m0 = 4u * (uint32_t)gq;
        const uint32_t row = fdiv(m0, a.div_h);
        const int k0 = (int)m0 - (int)row * h;
        const uint32_t z = ND == 3 ? fdiv(row, a.div_ly) : 0u;
        const int y = (int)row - (int)z * a.Ly;
        const int par = (c ^ (y + (int)z)) & 1;
        const int q0 = ((int)row * 2 + par) * h + k0;
        const int o0 = ((int)row * 2 + (par ^ 1)) * h;  // the row's other-parity words
        const int rym = y == 0 ? (int)row + a.Ly - 1 : (int)row - 1;
        const int ryp = y + 1 == a.Ly ? (int)row - a.Ly + 1 : (int)row + 1;
        const int ke = par ? (k0 + 4 == h ? 0 : k0 + 4) : (k0 == 0 ? h - 1 : k0 - 1);  // the fifth other-parity word
        const uint4 S = *reinterpret_cast<const uint4*>(sp + q0);
        const uint4 O4 = *reinterpret_cast<const uint4*>(sp + o0 + k0);
        const uint32_t oe = sp[o0 + ke];
        const int qym = (rym * 2 + par) * h + k0;
        const uint4 YP = *reinterpret_cast<const uint4*>(sp + (ryp * 2 + par) * h + k0);
        const uint4 YM = *reinterpret_cast<const uint4*>(sp + qym);
        const uint4 FX = ldg4(bx + q0), FY = ldg4(by + q0);
        const uint4 BX4 = ldg4(bx + o0 + k0), BY = ldg4(by + qym);
        const uint32_t bxe = par ? 0u : __ldg(bx + o0 + ke);
        uint4 ZP = make_uint4(0, 0, 0, 0), ZM = ZP, FZ = ZP, BZ = ZP;
        if constexpr (ND == 3) {
          const int rzm = z == 0 ? (int)row + nrow - a.Ly : (int)row - a.Ly;
          const int rzp = (int)z + 1 == a.Lz ? (int)row - nrow + a.Ly : (int)row + a.Ly;
          const int qzm = (rzm * 2 + par) * h + k0;
          ZP = *reinterpret_cast<const uint4*>(sp + (rzp * 2 + par) * h + k0);
          ZM = *reinterpret_cast<const uint4*>(sp + qzm);
          FZ = ldg4(bz + q0);
          BZ = ldg4(bz + qzm);
        }
        const U4 P = philox10((uint32_t)gq, sweep, c2, stream, a.K);
        const uint32_t o[4] = {O4.x, O4.y, O4.z, O4.w}, bo[4] = {BX4.x, BX4.y, BX4.z, BX4.w};
        // even x: x+1 is other-parity word k, x-1 word k-1 (whose forward x bond
        // is the site's backward one); odd x: x-1 word k, x+1 word k+1
        const uint32_t xp0 = par ? o[1] : o[0], xm0 = par ? o[0] : oe, bm0 = par ? bo[0] : bxe;
        const uint32_t xp1 = par ? o[2] : o[1], xm1 = par ? o[1] : o[0], bm1 = par ? bo[1] : bo[0];
        const uint32_t xp2 = par ? o[3] : o[2], xm2 = par ? o[2] : o[1], bm2 = par ? bo[2] : bo[1];
        const uint32_t xp3 = par ? oe : o[3], xm3 = par ? o[3] : o[2], bm3 = par ? bo[3] : bo[2];
        uint4 R;
        R.x = update(S.x, xp0, xm0, YP.x, YM.x, ZP.x, ZM.x, FX.x, bm0, FY.x, BY.x, FZ.x, BZ.x, P.x);
        R.y = update(S.y, xp1, xm1, YP.y, YM.y, ZP.y, ZM.y, FX.y, bm1, FY.y, BY.y, FZ.y, BZ.y, P.y);
        R.z = update(S.z, xp2, xm2, YP.z, YM.z, ZP.z, ZM.z, FX.z, bm2, FY.z, BY.z, FZ.z, BZ.z, P.z);
        R.w = update(S.w, xp3, xm3, YP.w, YM.w, ZP.w, ZM.w, FX.w, bm3, FY.w, BY.w, FZ.w, BZ.w, P.w);
        *reinterpret_cast<uint4*>(sp + q0) = R;
      }
      __syncthreads();
    }
  }
  for (int i = tid; i < (N >> 2); i += nth) reinterpret_cast<uint4*>(gw)[i] = reinterpret_cast<const uint4*>(sp)[i];
  if (!a.need_u) return;

  // unsatisfied forward bonds of every sample: bit-sliced 8-bit counters per
  // thread over chunks of at most 80 sites (ND bonds each, <= 240), then per
  // sample totals from 8 x 8 bit transposes, summed over the warp and the CTA
  for (int n0 = 0; n0 < N; n0 += 80 * nth) {  // block-uniform
    uint32_t cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int n1 = N < n0 + 80 * nth ? N : n0 + 80 * nth;
    for (int n = n0 + tid; n < n1; n += nth) {
      const int r = (int)fdiv((uint32_t)n >> 1, a.div_h);  // n / Lx (Lx = 2 h)
      const int x = n - r * a.Lx;
      const int z = ND == 3 ? (int)fdiv((uint32_t)r, a.div_ly) : 0;
      const int y = r - z * a.Ly;
      const int q = (r * 2 + (x & 1)) * h + (x >> 1);
      const uint32_t s = sp[q];
      const int xp = x + 1 == a.Lx ? 0 : x + 1;
      const int ryp = y + 1 == a.Ly ? r - a.Ly + 1 : r + 1;
      uint32_t w3[ND];
      w3[0] = s ^ sp[(r * 2 + (xp & 1)) * h + (xp >> 1)] ^ __ldg(bx + q);
      w3[1] = s ^ sp[(ryp * 2 + (x & 1)) * h + (x >> 1)] ^ __ldg(by + q);
      if constexpr (ND == 3) {
        const int rzp = z + 1 == a.Lz ? r - nrow + a.Ly : r + a.Ly;
        w3[2] = s ^ sp[(rzp * 2 + (x & 1)) * h + (x >> 1)] ^ __ldg(bz + q);
      }
#pragma unroll
      for (int d = 0; d < ND; ++d) {
        uint32_t carry = w3[d];
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          const uint32_t tt = cnt[b] & carry;
          cnt[b] ^= carry;
          carry = tt;
        }
      }
    }
    // bit j of cnt[b] is bit b of sample j's count: byte gg of the eight words is
    // an 8 x 8 bit block whose transpose holds the counts of samples 8 gg .. 8 gg + 7
    uint32_t pk[16];  // pk[i]: sample 2 i in bits 0-15, sample 2 i + 1 in bits 16-31
#pragma unroll
    for (int gg = 0; gg < 4; ++gg) {
      unsigned long long mt = 0;
#pragma unroll
      for (int b = 0; b < 8; ++b) mt |= (unsigned long long)((cnt[b] >> (8 * gg)) & 0xffu) << (8 * b);
      unsigned long long tt = (mt ^ (mt >> 7)) & 0x00AA00AA00AA00AAull;
      mt = mt ^ tt ^ (tt << 7);
      tt = (mt ^ (mt >> 14)) & 0x0000CCCC0000CCCCull;
      mt = mt ^ tt ^ (tt << 14);
      tt = (mt ^ (mt >> 28)) & 0x00000000F0F0F0F0ull;
      mt = mt ^ tt ^ (tt << 28);
#pragma unroll
      for (int i = 0; i < 4; ++i)
        pk[4 * gg + i] = ((uint32_t)(mt >> (16 * i)) & 0xffu) | (((uint32_t)(mt >> (16 * i + 8)) & 0xffu) << 16);
    }
    uint32_t mine = 0;  // lane j: sample j's warp total
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const uint32_t v = __reduce_add_sync(0xffffffffu, pk[i]);
      if ((lane >> 1) == i) mine = (lane & 1) ? (v >> 16) : (v & 0xffffu);
    }
    if (mine) atomicAdd(&ucount[lane], mine);
  }
  __syncthreads();
  if (tid < 32) a.U[(size_t)wl * 32 + tid] = ucount[tid];
}

// One warp per group: the decisions of exchange step e for every sample of the
// group (lane j), a ballot per pair into the swap masks.
__global__ void k_dp_exchange(const __grid_constant__ EaDpExchangeArgs a) {
  const int g = blockIdx.x, lane = threadIdx.x & 31;
  const int s = dp_sample(g, lane);
  const bool valid = s < a.nsamples;
  const uint32_t e = a.e;
  for (int k = 0; k + 1 < 32; ++k) {
    bool accept = false;
    if (valid && (k & 1) == (int)(e & 1)) {
      const int d = (int)a.U[(size_t)(32 * g + k + 1) * 32 + lane] - (int)a.U[(size_t)(32 * g + k) * 32 + lane];
      if (((a.xalways >> k) & 1u) || d <= 0) {
        accept = true;
      } else if (d <= a.xlen[k]) {  // (E_k - E_k+1) = -2 d
        const U4 P = philox10((uint32_t)k >> 2, e, kExchange << 1, (uint32_t)s, a.K);
        accept = u4_word(P, k & 3) < a.xtab[a.xoff[k] + d - 1];
      }
    }
    const uint32_t m = __ballot_sync(0xffffffffu, accept);
    if (lane == 0) a.X[32 * g + k] = m;
    if (accept) a.xacc[(size_t)s * 32 + k] += 1ull;
  }
  if (lane == 0) a.X[32 * g + 31] = 0;
}

// Swap the accepted samples' configurations between the two word lattices of
// every pair: bit j of each word, for the pairs whose mask has bit j.
__global__ void k_dp_swap(uint32_t* __restrict__ dp, const uint32_t* __restrict__ X, int N, int ngroups) {
  const int64_t quads = (int64_t)N >> 2;
  const int64_t total = (int64_t)ngroups * 32 * quads;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t wk = i / quads;  // word lattice 32 g + k of the lower temperature of the pair
    const uint32_t m = X[wk];
    if (!m) continue;
    uint4* pa = reinterpret_cast<uint4*>(dp + (size_t)wk * N) + (i - wk * quads);
    uint4* pb = pa + quads;  // word lattice 32 g + k + 1
    uint4 A = *pa, B = *pb;
    const uint32_t dx = (A.x ^ B.x) & m, dy = (A.y ^ B.y) & m, dz = (A.z ^ B.z) & m, dw = (A.w ^ B.w) & m;
    *pa = make_uint4(A.x ^ dx, A.y ^ dy, A.z ^ dz, A.w ^ dw);
    *pb = make_uint4(B.x ^ dx, B.y ^ dy, B.z ^ dz, B.w ^ dw);
  }
}

int grid_for(int64_t work, int per_block) {
  const int64_t want = (work + per_block - 1) / per_block;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)device_sm_count() * 16));
}

}  // namespace

size_t dp_smem(int N) { return (size_t)N * 4; }

cudaError_t launch_dp_from_words(const uint64_t* pairs, uint32_t* dp, int Lx, int N, int nsamples, int ngroups,
                                 cudaStream_t st) {
  k_dp_from_words<<<grid_for((int64_t)ngroups * N * 32, 256), 256, 0, st>>>(reinterpret_cast<const uint32_t*>(pairs),
                                                                            dp, Lx, N, nsamples, ngroups);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_dp_to_words(const uint32_t* dp, uint64_t* pairs, int Lx, int N, int nsamples, int ngroups,
                               cudaStream_t st) {
  k_dp_to_words<<<grid_for((int64_t)ngroups * N * 32, 256), 256, 0, st>>>(dp, reinterpret_cast<uint32_t*>(pairs), Lx,
                                                                          N, nsamples, ngroups);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_dp_bonds(const uint64_t* packed, uint32_t* bdp, int nd, int Lx, int N, int nsamples, int ngroups,
                            cudaStream_t st) {
  k_dp_bonds<<<grid_for((int64_t)ngroups * nd * N * 32, 256), 256, 0, st>>>(packed, bdp, nd, Lx, N, nsamples,
                                                                           ngroups);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_dp_sweep(const EaDpArgs& a, int nwl, int threads, cudaStream_t st) {
  const size_t sm = dp_smem(a.N);
  auto kern = a.nd == 2 ? k_dp_sweep<2> : k_dp_sweep<3>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  kern<<<nwl, threads, sm, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_dp_exchange(const EaDpExchangeArgs& a, int ngroups, cudaStream_t st) {
  k_dp_exchange<<<ngroups, 32, 0, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_dp_swap(uint32_t* dp, const uint32_t* X, int N, int ngroups, cudaStream_t st) {
  k_dp_swap<<<grid_for((int64_t)ngroups * 32 * (N >> 2), 256), 256, 0, st>>>(dp, X, N, ngroups);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace spn
