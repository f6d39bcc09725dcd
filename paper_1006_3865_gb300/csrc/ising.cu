// Checkerboard Metropolis kernels for int8 Ising-type lattices (Weigel, Sec. 3,
// Eq. 1-2; Sec. 4 for 3D and +-J couplings).
//
//   k_init_hot        hot start from Philox (purpose 1, most significant plane).
//   k_observables     full reduction of E (Eq. 1) and M.
//   k_sweep_generic   one colour of a sweep in place in global memory; a thread
//                     owns one group of 32 same-colour sites.  Any even extents,
//                     optional +-J bonds.  Two launches per sweep realise the
//                     order colour 0, then colour 1.
//   k_sweep_stream    both colours of one sweep in one pass (Lx % 64 == 0, no
//                     bonds).  A CTA owns full-width rows (3D: a band of rows)
//                     and a segment of slices along the slowest axis (2D: rows,
//                     3D: z planes).  Raw int8 slices stream into a ring of
//                     shared-memory buffers through bulk asynchronous copies
//                     (cp.async.bulk, completion on mbarriers); each slice is
//                     converted once into colour-separated bit words, colour 0
//                     is updated on the slices plus a one-slice / one-row ring
//                     (repeating a neighbour's work with the same counters, so
//                     it is bit-identical), colour 1 on the owned part, and the
//                     result is expanded back to int8 into the other buffer.
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
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

// ---------------------------------------------------------------- init / E, M

__global__ void k_init_hot(int8_t* __restrict__ s, int Lx, int Ly, int64_t N, PhiloxKeys K, uint32_t stream_id) {
  const int64_t half = N >> 1;
  const int64_t ngroups = (half + 31) >> 5;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < 2 * ngroups;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t & 1);
    const int64_t g = t >> 1;
    const uint32_t plane0 = philox10((uint32_t)(8 * g), 0u, (uint32_t)c | (kInit << 1), stream_id, K).x;
    for (int i = 0; i < 32; ++i) {
      const int64_t m = g * 32 + i;
      if (m >= half) break;
      s[site_of(m, c, Lx, Ly)] = ((plane0 >> i) & 1u) ? (int8_t)-1 : (int8_t)1;
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
  const int64_t work = 2 * (((g.N >> 1) + 31) >> 5);
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((work + threads - 1) / threads, (int64_t)device_sm_count() * 32);
  k_init_hot<<<(unsigned)std::max<int64_t>(blocks, 1), threads, 0, st>>>(s, g.Lx, g.Ly, g.N, philox_keys(seed),
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

// One colour c of sweep `sweep`, in place: a thread owns the group of 32 sites
// with within-colour indices 32 g .. 32 g + 31.
template <int ND>
__global__ void k_sweep_generic(int8_t* __restrict__ s, const uint8_t* __restrict__ bonds, int Lx, int Ly, int Lz,
                                int64_t N, int c, DevThr T, PhiloxKeys K, uint32_t stream_id, uint32_t sweep,
                                unsigned long long* acc) {
  const int64_t half = N >> 1;
  const int64_t ngroups = (half + 31) >> 5;
  int de = 0, dm = 0;
  // warp-uniform trip count: the decision votes across the warp
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31);
  for (int64_t g0 = base; g0 < ngroups; g0 += stride) {
    const int64_t g = g0 + (threadIdx.x & 31);
    uint32_t bits = 0, s0 = 0, s1 = 0, s2 = 0, valid = 0;
    if (g < ngroups) {
      for (int i = 0; i < 32; ++i) {
        const int64_t m = g * 32 + i;
        if (m >= half) break;
        const int64_t n = site_of(m, c, Lx, Ly);
        const int x = (int)(n % Lx);
        const int64_t r = n / Lx;
        const int y = (int)(r % Ly);
        const int z = (int)(r / Ly);
        const int sn = s[n];
        const int64_t xm = n - x + (x == 0 ? Lx - 1 : x - 1), xp = n - x + (x + 1 == Lx ? 0 : x + 1);
        const int64_t ym = n + (int64_t)((y == 0 ? Ly - 1 : y - 1) - y) * Lx;
        const int64_t yp = n + (int64_t)((y + 1 == Ly ? 0 : y + 1) - y) * Lx;
        int h = bond_sign(bonds, n, 0) * s[xp] + bond_sign(bonds, xm, 0) * s[xm] +
                bond_sign(bonds, n, 1) * s[yp] + bond_sign(bonds, ym, 1) * s[ym];
        if (ND == 3) {
          const int64_t LxLy = (int64_t)Lx * Ly;
          const int64_t zm = n + (int64_t)((z == 0 ? Lz - 1 : z - 1) - z) * LxLy;
          const int64_t zp = n + (int64_t)((z + 1 == Lz ? 0 : z + 1) - z) * LxLy;
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
          const int64_t n = site_of(g * 32 + i, c, Lx, Ly);
          s[n] = (int8_t)(-s[n]);
        }
      }
    }
  }
  block_accumulate(de, dm, acc);
}

cudaError_t launch_sweep_generic(const Lattice& g, int8_t* s, const DevThr& T, const PhiloxKeys& K,
                                 uint32_t stream_id, uint32_t sweep, unsigned long long* acc, cudaStream_t st) {
  const int64_t ngroups = ((g.N >> 1) + 31) >> 5;
  const int threads = 128;
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((ngroups + threads - 1) / threads,
                                                                (int64_t)device_sm_count() * 16));
  for (int c = 0; c < 2; ++c) {
    if (g.nd == 3)
      k_sweep_generic<3><<<(unsigned)blocks, threads, 0, st>>>(s, g.bonds, g.Lx, g.Ly, g.Lz, g.N, c, T, K,
                                                               stream_id, sweep, acc);
    else
      k_sweep_generic<2><<<(unsigned)blocks, threads, 0, st>>>(s, g.bonds, g.Lx, g.Ly, g.Lz, g.N, c, T, K,
                                                               stream_id, sweep, acc);
  }
  count_launches(2);
  return cudaGetLastError();
}

// ---------------------------------------------------------- streaming sweep

namespace {

struct StreamArgs {
  const int8_t* in;
  int8_t* out;
  int Lx, Ly, Lz;
  int TY;      // rows per band (3D); 1 in 2D
  int R;       // slices per step
  int nseg;    // segments along the streamed axis
  int S;       // slices along the streamed axis (2D: Ly, 3D: Lz)
  int nraw;    // raw slice buffers
  int nbit;    // bit slice buffers
  uint32_t sweep, stream_id;
  PhiloxKeys K;
  DevThr T;
  unsigned long long* acc;
  int* err;
};

constexpr int kRounds = 2;  // items of one kind a thread handles per step

#ifndef SPN_STREAM_MIN_BLOCKS
#define SPN_STREAM_MIN_BLOCKS 2  // resident CTAs the register allocation aims for (512 threads each)
#endif

// A thread's item of one kind (conversion span, colour-0 word, colour-1 word)
// within a step: slice k (0 .. R-1), band row r, word j; fixed for the launch.
struct Item {
  int k, r, j;
  bool live;
};

__device__ __forceinline__ Item item_of(int it, int per, int W, int n, int rowoff) {
  Item x;
  x.live = it < n;
  const int itc = x.live ? it : 0;
  x.k = itc / per;
  const int rem = itc - x.k * per;
  x.r = rem / W + rowoff;
  x.j = rem - (rem / W) * W;
  return x;
}

template <int ND>
__global__ void __launch_bounds__(512, SPN_STREAM_MIN_BLOCKS) k_sweep_stream(StreamArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  constexpr int YH = (ND == 3) ? 2 : 0;
  const int Lx = a.Lx;
  const int W = Lx >> 6;                     // words per parity per row
  const int RSL = (ND == 3) ? a.TY + 4 : 1;  // rows per slice
  const int rowsA = (ND == 3) ? a.TY + 2 : 1;
  const int rowsB = (ND == 3) ? a.TY : 1;
  const int rawBytes = RSL * Lx;
  const int rawStride = (rawBytes + 127) & ~127;
  const int bitWords = RSL * 2 * W;  // bit slice: E then O words per row
  uint8_t* raw = smem;
  uint32_t* bitbuf = reinterpret_cast<uint32_t*>(smem + (size_t)a.nraw * rawStride);
  uint2* lut = reinterpret_cast<uint2*>(bitbuf + (size_t)a.nbit * bitWords);
  uint64_t* bars = reinterpret_cast<uint64_t*>(lut + 256);
  const int qcap = kRounds * blockDim.x;                               // one entry per item at most
  uint4* qe = reinterpret_cast<uint4*>(smem + (((size_t)a.nraw * rawStride + (size_t)a.nbit * bitWords * 4 +
                                                 256 * 8 + (size_t)a.nraw * 8 + 15) & ~(size_t)15));
  int* qslot_of = reinterpret_cast<int*>(qe + qcap);
  uint32_t* late = reinterpret_cast<uint32_t*>(qslot_of + qcap);
  __shared__ int s_abort;
  __shared__ int s_qcount;
  int* qcount = &s_qcount;

  const int tid = threadIdx.x, nth = blockDim.x;
  const int lane = tid & 31;
  const int y0 = (ND == 3) ? blockIdx.x * a.TY : 0;
  const int seg = blockIdx.y;
  const int zs = (int)(((int64_t)seg * a.S) / a.nseg);
  const int ze = (int)(((int64_t)(seg + 1) * a.S) / a.nseg);
  const int H = ze - zs;
  const int nload = H + 4;  // local slices li = 0 .. H + 3 <-> global zs - 2 + li
  const int64_t sliceStride = (int64_t)Lx * ((ND == 3) ? a.Ly : 1);

  // int8 byte patterns of 8 sites [e0 o0 e1 o1 e2 o2 e3 o3] for index e4 | o4 << 4
  for (int i = tid; i < 256; i += nth) {
    uint32_t lo = 0, hi = 0;
    for (int k = 0; k < 4; ++k) {
      const uint32_t eb = ((i >> k) & 1) ? 0xffu : 0x01u;
      const uint32_t ob = ((i >> (4 + k)) & 1) ? 0xffu : 0x01u;
      const uint32_t pair = eb | (ob << 8);
      if (k < 2) lo |= pair << (16 * k); else hi |= pair << (16 * (k - 2));
    }
    lut[i] = make_uint2(lo, hi);
  }
  if (tid == 0) {
    s_abort = 0;
    s_qcount = 0;
    for (int b = 0; b < a.nraw; ++b) mbar_init(&bars[b], 1);
    fence_mbar_init();
  }

  // Static item maps (slice k of the step, row, word) for the three kinds.
  Item ic[kRounds], ia[kRounds], ib[kRounds];
#pragma unroll
  for (int q = 0; q < kRounds; ++q) {
    ic[q] = item_of(tid + q * nth, RSL * W, W, a.R * RSL * W, 0);
    ia[q] = item_of(tid + q * nth, rowsA * W, W, a.R * rowsA * W, ND == 3 ? -1 : 0);
    ib[q] = item_of(tid + q * nth, rowsB * W, W, a.R * rowsB * W, 0);
  }
  const int roundsC = (a.R * RSL * W + nth - 1) / nth;
  const int roundsA = (a.R * rowsA * W + nth - 1) / nth;
  const int roundsB = (a.R * rowsB * W + nth - 1) / nth;
  __syncthreads();

  auto wrapS = [&](int z) { return z < 0 ? z + a.S : (z >= a.S ? z - a.S : z); };
  auto wrapY = [&](int y) { return y < 0 ? y + a.Ly : (y >= a.Ly ? y - a.Ly : y); };
  auto bslot = [&](int li) { return li % a.nbit; };  // per step only (uniform)

  // Issue the bulk copies of local slice li (warp 0).
  auto issue = [&](int li) {
    if (li >= nload || tid >= 32) return;
    uint8_t* B = raw + (size_t)(li % a.nraw) * rawStride;
    uint64_t* bar = &bars[li % a.nraw];
    if (tid == 0) {
      fence_proxy_async();
      mbar_arrive_expect_tx(bar, (uint32_t)rawBytes);
    }
    __syncwarp();
    const int gz = wrapS(zs - 2 + li);
    for (int r = tid; r < RSL; r += 32) {
      const int gy = (ND == 3) ? wrapY(y0 - YH + r) : 0;
      bulk_g2s(B + (size_t)r * Lx, a.in + (int64_t)gz * sliceStride + (int64_t)gy * Lx, (uint32_t)Lx, bar);
    }
  };

  auto wait_raw = [&](int l0, int ns) -> bool {
    for (int li = l0; li < l0 + ns; ++li) {
      const uint32_t parity = (uint32_t)((li / a.nraw) & 1);
      unsigned n = 0;
      while (!mbar_try_wait(&bars[li % a.nraw], parity)) {
        if (++n > kWaitLimit) {
          s_abort = 1;
          break;
        }
      }
    }
    return __syncthreads_or(s_abort) != 0;
  };

  // Raw slices l0 .. l0+ns-1 -> bit words E (even x) and O (odd x) per row.
  auto convert = [&](int l0, int ns) {
    const int rbase = l0 % a.nraw, bbase = bslot(l0);
#pragma unroll
    for (int q = 0; q < kRounds; ++q) {
      const Item x = ic[q];
      if (q < roundsC && x.live && x.k < ns) {
        int rs = rbase + x.k;
        if (rs >= a.nraw) rs -= a.nraw;
        int bs = bbase + x.k;
        if (bs >= a.nbit) bs -= a.nbit;
        const uint8_t* span = raw + (size_t)rs * rawStride + (size_t)x.r * Lx + 64 * x.j;
        uint32_t E = 0, O = 0;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          // rotate the 16-byte chunk order by lane so a quarter warp hits distinct banks
          const int cv = (v + (lane >> 1)) & 3;
          const uint4 qv = *reinterpret_cast<const uint4*>(span + 16 * cv);
          const uint32_t w[4] = {qv.x, qv.y, qv.z, qv.w};
#pragma unroll
          for (int p = 0; p < 2; ++p) {
            const int t = 2 * cv + p;  // sites 8t .. 8t+7 of the span
            const uint32_t ev = __byte_perm(w[2 * p], w[2 * p + 1], 0x6420);
            const uint32_t od = __byte_perm(w[2 * p], w[2 * p + 1], 0x7531);
            E |= sign_bits4(ev) << (4 * t);
            O |= sign_bits4(od) << (4 * t);
          }
        }
        uint32_t* row = bitbuf + (size_t)bs * bitWords + (size_t)x.r * 2 * W;
        row[x.j] = E;
        row[W + x.j] = O;
      }
    }
  };

  int de = 0, dm = 0;

  // Per-word state between the first decision stage and the final write.
  struct WordState {
    uint32_t b, s0, s1, s2, acc;
    int par;
    bool pending;
  };

  auto slot_plus = [&](int s, int d) {
    s += d;
    return s >= a.nbit ? s - a.nbit : s;
  };

  // Neighbour counts, classes and the first 8 planes of the colour-c word of
  // item x in local slice li (bit slot bs); pushes a tie to the CTA queue.
  auto prepare = [&](const Item& x, int li, int bs, int c, int qslot) {
    const int bm = bs == 0 ? a.nbit - 1 : bs - 1, bp = slot_plus(bs, 1);
    const int gz = wrapS(zs - 2 + li);
    const int gy = (ND == 3) ? wrapY(y0 + x.r) : gz;
    const int gzz = (ND == 3) ? gz : 0;
    const int par = (gy + gzz + c) & 1;
    const int ro = (x.r + YH) * 2 * W;
    const uint32_t* row = bitbuf + (size_t)bs * bitWords + ro;
    const uint32_t* same = row + par * W;
    const uint32_t* other = row + (W - par * W);
    const int j = x.j;
    WordState w;
    w.b = same[j];
    const int jm = j == 0 ? W - 1 : j - 1, jp = j + 1 == W ? 0 : j + 1;
    uint32_t left, right;
    if (par == 0) {
      right = other[j];
      left = __funnelshift_l(other[jm], other[j], 1);  // (O_j << 1) | (O_{j-1} >> 31)
    } else {
      left = other[j];
      right = __funnelshift_r(other[j], other[jp], 1);  // (E_j >> 1) | (E_{j+1} << 31)
    }
    const uint32_t zm = bitbuf[(size_t)bm * bitWords + ro + par * W + j];
    const uint32_t zp = bitbuf[(size_t)bp * bitWords + ro + par * W + j];
    const uint32_t b = w.b;
    if constexpr (ND == 3) {
      const uint32_t ym = same[j - 2 * W];
      const uint32_t yp = same[j + 2 * W];
      count6(b ^ left, b ^ right, b ^ ym, b ^ yp, b ^ zm, b ^ zp, w.s0, w.s1, w.s2);
    } else {
      count4(b ^ left, b ^ right, b ^ zm, b ^ zp, w.s0, w.s1, w.s2);
    }
    uint32_t cls[ND], eq[ND];
    w.acc = classes<ND>(w.s0, w.s1, w.s2, 0xffffffffu, cls);
    const uint32_t c0 = 8u * ((uint32_t)j + (uint32_t)W * (uint32_t)(gy + a.Ly * gzz));
    decide_first<ND>(w.acc, eq, cls, a.T, a.K, c0, a.sweep, (uint32_t)c | (kMetropolis << 1), a.stream_id);
    uint32_t any = 0;
#pragma unroll
    for (int q = 0; q < ND; ++q) any |= eq[q];
    w.pending = any != 0;
    if (w.pending) {
      const int e = atomicAdd(qcount, 1);
      qe[e] = make_uint4(c0, eq[0], eq[1], ND == 3 ? eq[ND - 1] : 0u);
      qslot_of[e] = qslot;
    }
    w.par = par;
    return w;
  };

  // Planes 8.. for the queued words, whole warps at a time.
  auto tail = [&](int c) {
    const int n = *qcount;
    for (int base = tid & ~31; base < n; base += nth) {
      const int e = base + lane;
      uint32_t eq[ND];
      uint32_t c0 = 0;
#pragma unroll
      for (int q = 0; q < ND; ++q) eq[q] = 0;
      if (e < n) {
        const uint4 v = qe[e];
        c0 = v.x;
        eq[0] = v.y;
        eq[1] = v.z;
        if constexpr (ND == 3) eq[2] = v.w;
      }
      const uint32_t accepted =
          decide_tail<ND>(eq, a.T, a.K, c0, a.sweep, (uint32_t)c | (kMetropolis << 1), a.stream_id);
      if (e < n) late[qslot_of[e]] = accepted;
    }
  };

  // Colour 0 on local slices l0 .. l0+ns-1: rows -1 .. TY (3D) of each slice.
  auto passA = [&](int l0, int ns) {
    const int base = bslot(l0);
    WordState st[kRounds];
    int where[kRounds];
    bool own[kRounds];
#pragma unroll
    for (int q = 0; q < kRounds; ++q) {
      where[q] = -1;
      own[q] = false;
      const Item x = ia[q];
      if (q < roundsA && x.live && x.k < ns) {
        const int li = l0 + x.k;
        const int bs = slot_plus(base, x.k);
        st[q] = prepare(x, li, bs, 0, q * nth + tid);
        own[q] = li >= 2 && li < H + 2 && (ND == 2 || (x.r >= 0 && x.r < a.TY));
        where[q] = bs * bitWords + (x.r + YH) * 2 * W + st[q].par * W + x.j;
      }
    }
    __syncthreads();
    tail(0);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kRounds; ++q) {
      if (where[q] >= 0) {
        WordState& w = st[q];
        if (w.pending) w.acc |= late[q * nth + tid];
        if (own[q]) tally<ND>(w.acc, w.b, w.s0, w.s1, w.s2, de, dm);
        bitbuf[where[q]] = w.b ^ w.acc;
      }
    }
    if (tid == 0) *qcount = 0;  // no pushes before the next barrier
    __syncthreads();
  };

  // Colour 1 on local slices l0 .. l0+ns-1, owned rows; final rows to global.
  auto passB = [&](int l0, int ns) {
    const int base = bslot(l0);
    WordState st[kRounds];
    int bsq[kRounds];
#pragma unroll
    for (int q = 0; q < kRounds; ++q) {
      bsq[q] = -1;
      const Item x = ib[q];
      if (q < roundsB && x.live && x.k < ns) {
        const int li = l0 + x.k;
        bsq[q] = slot_plus(base, x.k);
        st[q] = prepare(x, li, bsq[q], 1, q * nth + tid);
      }
    }
    __syncthreads();
    tail(1);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kRounds; ++q) {
      if (bsq[q] >= 0) {
        const Item x = ib[q];
        WordState& w = st[q];
        if (w.pending) w.acc |= late[q * nth + tid];
        tally<ND>(w.acc, w.b, w.s0, w.s1, w.s2, de, dm);
        const uint32_t nw = w.b ^ w.acc;
        const uint32_t* row = bitbuf + (size_t)bsq[q] * bitWords + (x.r + YH) * 2 * W;
        const uint32_t E = w.par == 0 ? nw : row[x.j];
        const uint32_t O = w.par == 0 ? row[W + x.j] : nw;
        const int li = l0 + x.k;
        const int gz = wrapS(zs - 2 + li);
        const int gy = (ND == 3) ? y0 + x.r : gz;
        const int gzz = (ND == 3) ? gz : 0;
        uint4* dst = reinterpret_cast<uint4*>(a.out + (int64_t)gzz * sliceStride + (int64_t)gy * Lx + 64 * x.j);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const uint2 lo = lut[((E >> (8 * v)) & 0xfu) | (((O >> (8 * v)) & 0xfu) << 4)];
          const uint2 hi = lut[((E >> (8 * v + 4)) & 0xfu) | (((O >> (8 * v + 4)) & 0xfu) << 4)];
          dst[v] = make_uint4(lo.x, lo.y, hi.x, hi.y);
        }
      }
    }
    if (tid == 0) *qcount = 0;  // the next pushes follow the next step's conversion barrier
  };

  // Prologue: slices zs-2 .. zs+1 (local 0..3), colour 0 on zs-1 and zs.
  const int first = a.nraw < nload ? a.nraw : nload;
  for (int li = 0; li < first; ++li) issue(li);
  int issued = first;
  bool abort = false;
  for (int li = 0; li < 4 && !abort; ++li) {  // one slice at a time: the raw ring may hold fewer than 4
    abort = wait_raw(li, 1);
    if (abort) break;
    convert(li, 1);
    __syncthreads();
    issue(li + a.nraw);
    issued = (li + 1 + a.nraw < nload) ? li + 1 + a.nraw : nload;
  }
  if (!abort) {
    passA(1, 1);
    passA(2, 1);
  }
  // Step: outputs o in [b0, b0 + ns) (local li = o + 2).
  for (int b0 = 0; b0 < H && !abort; b0 += a.R) {
    const int ns = (b0 + a.R < H) ? a.R : H - b0;
    abort = wait_raw(b0 + 4, ns);
    if (abort) break;
    convert(b0 + 4, ns);
    __syncthreads();
    for (int li = b0 + 4; li < b0 + 4 + ns; ++li) issue(li + a.nraw);
    issued = (b0 + 4 + ns + a.nraw < nload) ? b0 + 4 + ns + a.nraw : nload;
    passA(b0 + 3, ns);
    passB(b0 + 2, ns);
  }

  if (abort) {
    if (tid == 0) {
      atomicExch(a.err, 1);
      // let the copies still in flight land before the CTA exits (bounded)
      for (int li = issued > a.nraw ? issued - a.nraw : 0; li < issued; ++li) {
        unsigned n = 0;
        while (!mbar_try_wait(&bars[li % a.nraw], (uint32_t)((li / a.nraw) & 1)) && ++n < kWaitLimit) {
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
  if (g.nd == 3 && (TY <= 0 || g.Ly % TY)) return false;
  const int RSL = g.nd == 3 ? TY + 4 : 1;
  if ((int64_t)RSL * g.Lx * 3 > 200 * 1024) return false;  // a few raw slices must fit in shared memory
  return true;
}

StreamGeom stream_geometry(const Lattice& g, int TY, int R, int nseg) {
  StreamGeom s{};
  s.TY = g.nd == 3 ? TY : 1;
  const int W = g.Lx / 64;
  const int RSL = g.nd == 3 ? TY + 4 : 1;
  const int S = g.nd == 3 ? g.Lz : g.Ly;
  const int perB = (g.nd == 3 ? TY : 1) * W;
  const bool automatic = R <= 0;
  if (automatic) R = std::max(1, std::min(S, 1024 / std::max(1, perB)));  // two colour-1 words per thread
  const size_t rawStride = (size_t)((RSL * g.Lx + 127) & ~127);
  auto smem_of = [&](int r, int nraw) {  // + the tie queue (16 + 4 + 4 bytes per item), sized for 512 threads
    return (((size_t)nraw * rawStride + (size_t)(2 * r + 3) * RSL * 2 * W * 4 + 256 * 8 + (size_t)nraw * 8 + 15) &
            ~(size_t)15) + (size_t)kRounds * 512 * 24;
  };
  const size_t cap = 233472 / 2 - 1024;  // two CTAs per SM (228 KB per SM, 1 KB reserved per CTA)
  while (automatic && R > 1 && smem_of(R, R) > cap) --R;
  s.R = R;
  s.nbit = 2 * R + 3;
  s.nraw = std::max(3, 2 * R);  // a raw slice is issued once the slice nraw before it is converted
  while (smem_of(R, s.nraw) > cap && s.nraw > std::max(1, R)) s.nraw -= 1;
  s.smem = smem_of(R, s.nraw);
  const int nC = R * RSL * W, nA = R * (g.nd == 3 ? TY + 2 : 1) * W, nB = R * perB;
  const int need = (std::max(nC, std::max(nA, nB)) + kRounds - 1) / kRounds;
  int th = std::max(need, std::min(nB, 512));
  th = ((th + 31) / 32) * 32;
  s.threads = std::min(512, std::max(64, th));
  if (nseg <= 0) {
    const int tiles = g.nd == 3 ? g.Ly / TY : 1;
    const int want = device_sm_count() * 2;
    nseg = std::max(1, std::min(S, (want + tiles - 1) / tiles));
  }
  s.nseg = std::min(nseg, S);
  return s;
}

bool stream_geometry_ok(const Lattice& g, const StreamGeom& geo) {
  const int W = g.Lx / 64;
  const int RSL = g.nd == 3 ? geo.TY + 4 : 1;
  const int nC = geo.R * RSL * W, nA = geo.R * (g.nd == 3 ? geo.TY + 2 : 1) * W, nB = geo.R * (g.nd == 3 ? geo.TY : 1) * W;
  const int cap = geo.threads * kRounds;
  return geo.threads <= 512 && geo.threads % 32 == 0 && nC <= cap && nA <= cap && nB <= cap &&
         geo.smem <= 227 * 1024 && geo.nraw >= geo.R && geo.nbit >= 2 * geo.R + 3 && geo.nseg >= 1;
}

cudaError_t launch_sweep_stream(const Lattice& g, const int8_t* in, int8_t* out, const StreamGeom& geo,
                                const DevThr& T, const PhiloxKeys& K, uint32_t stream_id, uint32_t sweep,
                                unsigned long long* acc, int* err, cudaStream_t st) {
  if (!stream_geometry_ok(g, geo)) return cudaErrorInvalidConfiguration;
  StreamArgs a;
  a.in = in;
  a.out = out;
  a.Lx = g.Lx;
  a.Ly = g.Ly;
  a.Lz = g.Lz;
  a.TY = geo.TY;
  a.R = geo.R;
  a.nseg = geo.nseg;
  a.S = g.nd == 3 ? g.Lz : g.Ly;
  a.nraw = geo.nraw;
  a.nbit = geo.nbit;
  a.sweep = sweep;
  a.stream_id = stream_id;
  a.K = K;
  a.T = T;
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
