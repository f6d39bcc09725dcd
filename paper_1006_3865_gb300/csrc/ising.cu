// Checkerboard Metropolis kernels for int8 Ising-type lattices (Weigel, Sec. 3,
// Eq. 1-2; Sec. 4 for 3D and +-J couplings).
//
//   k_init_hot        hot start from Philox (purpose "init").
//   k_observables     full reduction of E (Eq. 1) and M.
//   k_sweep_generic   one colour of the sweep in place in global memory, one
//                     thread per group of 8 same-colour sites; any even extents,
//                     optional +-J bonds.  The reference order of updates
//                     (colour 0 then colour 1) is realised by two launches.
//   k_sweep_stream    both colours of one sweep in a single pass.  A CTA owns an
//                     x-tile (3D: x-y tile) and a segment of slices along the
//                     slowest axis (2D: rows, 3D: z planes).  Slices plus a
//                     two-site halo stream into a ring of shared-memory buffers
//                     with bulk asynchronous copies (cp.async.bulk completing on
//                     an mbarrier).  Colour 0 is updated on the tile plus a
//                     one-site ring (the ring repeats the neighbours' work with
//                     the same counters, so it is bit-identical), colour 1 on the
//                     tile; the result goes to the other ping-pong buffer.
//
// Spins are int8 +-1 (0x01 / 0xFF).  Bit 1 of a byte is set iff the spin is -1,
// so (a ^ b) & 0x02 marks an anti-aligned pair; four bytes are handled per
// 32-bit operation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "philox.cuh"
#include "spn_internal.h"

namespace spn {

uint64_t boltzmann_threshold(double beta, int dE) {
  if (dE <= 0) return (uint64_t)1 << 32;
  const double a = beta * (double)dE;
  const double x = std::exp(-a) * 4294967296.0;
  return (uint64_t)std::floor(x);
}

ThrTab make_thresholds(double beta) {
  ThrTab T{};
  T.hi[0] = 0x10000u;
  T.lo[0] = 0;
  for (int q = 1; q < 4; ++q) {
    uint64_t t = boltzmann_threshold(beta, 4 * q);
    T.hi[q] = (uint32_t)(t >> 16);
    T.lo[q] = (uint32_t)(t & 0xffffu);
  }
  return T;
}

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

// ------------------------------------------------------------------ helpers

// 16-bit high half of the Metropolis u of within-colour index m, from the
// group's Philox output.
__device__ __forceinline__ uint32_t half16(const U4& P, uint32_t i) {
  const uint32_t w = u4_word(P, (int)(i >> 1));
  return (i & 1) ? (w >> 16) : (w & 0xffffu);
}

// Selected 17-bit high threshold for class idx = dE/4 (idx <= 0: always).
__device__ __forceinline__ uint32_t thr_hi(int idx, const ThrTab& T) {
  return idx <= 0 ? 0x10000u : (idx == 1 ? T.hi[1] : (idx == 2 ? T.hi[2] : T.hi[3]));
}
__device__ __forceinline__ uint32_t thr_lo(int idx, const ThrTab& T) {
  return idx == 1 ? T.lo[1] : (idx == 2 ? T.lo[2] : T.lo[3]);
}

__device__ __forceinline__ void warp_reduce_add2(long long& a, long long& b) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
}

// Block-wide sum of (a, b), one atomic per warp.
__device__ __forceinline__ void block_accumulate(long long a, long long b, unsigned long long* out2) {
  warp_reduce_add2(a, b);
  if ((threadIdx.x & 31) == 0 && (a | b)) {
    atomicAdd(out2 + 0, (unsigned long long)a);
    atomicAdd(out2 + 1, (unsigned long long)b);
  }
}

__device__ __forceinline__ int64_t site_of(int64_t m, int c, int Lx, int Ly) {
  // Site of colour c with within-colour index m: n = 2m or 2m + 1 (Lx even,
  // so both share x >> 1, y and z).
  const int64_t n0 = 2 * m;
  const int64_t r = n0 / Lx;  // y + Ly * z
  const int y = (int)(r % Ly);
  const int z = (int)(r / Ly);
  return n0 + ((c ^ (y + z)) & 1);
}

// ---------------------------------------------------------------- init / E, M

__global__ void k_init_hot(int8_t* __restrict__ s, int Lx, int Ly, int64_t N, PhiloxKeys K, uint32_t stream_id) {
  const int64_t half = N >> 1;
  const int64_t ngroups = (half + 7) >> 3;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < 2 * ngroups;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t & 1);
    const int64_t gidx = t >> 1;
    const U4 P = philox10((uint32_t)gidx, 0u, (uint32_t)c | (kInitHi << 1), stream_id, K);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int64_t m = gidx * 8 + i;
      if (m < half) s[site_of(m, c, Lx, Ly)] = (half16(P, i) >> 15) ? (int8_t)-1 : (int8_t)1;
    }
  }
}

__device__ __forceinline__ int bond_sign(const uint8_t* __restrict__ bonds, int64_t n, int d) {
  return (bonds && ((bonds[n] >> d) & 1)) ? -1 : 1;
}

__global__ void k_observables(const int8_t* __restrict__ s, const uint8_t* __restrict__ bonds, int nd, int Lx,
                              int Ly, int Lz, int64_t N, unsigned long long* out2) {
  long long e = 0, m = 0;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(n % Lx);
    const int64_t r = n / Lx;
    const int y = (int)(r % Ly);
    const int z = (int)(r / Ly);
    const int sn = s[n];
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
  block_accumulate(e, m, out2);
}

cudaError_t launch_init_hot(const Lattice& g, int8_t* s, uint64_t seed, uint32_t stream_id, cudaStream_t st) {
  const int64_t work = 2 * (((g.N >> 1) + 7) >> 3);
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((work + threads - 1) / threads, (int64_t)device_sm_count() * 32);
  k_init_hot<<<(unsigned)std::max<int64_t>(blocks, 1), threads, 0, st>>>(s, g.Lx, g.Ly, g.N, philox_keys(seed),
                                                                         stream_id);
  return cudaGetLastError();
}

cudaError_t launch_observables(const Lattice& g, const int8_t* s, unsigned long long* out2, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out2, 0, 2 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((g.N + threads - 1) / threads, (int64_t)device_sm_count() * 16);
  k_observables<<<(unsigned)std::max<int64_t>(blocks, 1), threads, 0, st>>>(s, g.bonds, g.nd, g.Lx, g.Ly, g.Lz,
                                                                           g.N, out2);
  return cudaGetLastError();
}

// ------------------------------------------------------------ generic sweep

// One colour c of sweep `sweep`, in place: a thread decides the 8 sites of one
// Philox group (within-colour indices 8g .. 8g+7).
template <int ND>
__global__ void k_sweep_generic(int8_t* __restrict__ s, const uint8_t* __restrict__ bonds, int Lx, int Ly, int Lz,
                                int64_t N, int c, ThrTab T, PhiloxKeys K, uint32_t stream_id, uint32_t sweep,
                                unsigned long long* acc) {
  const int64_t half = N >> 1;
  const int64_t ngroups = (half + 7) >> 3;
  long long de = 0, dm = 0;
  for (int64_t gidx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gidx < ngroups;
       gidx += (int64_t)gridDim.x * blockDim.x) {
    const U4 P = philox10((uint32_t)gidx, sweep, (uint32_t)c | (kMetroHi << 1), stream_id, K);
    bool have_lo = false;
    U4 Q{0, 0, 0, 0};
#pragma unroll 1
    for (int i = 0; i < 8; ++i) {
      const int64_t m = gidx * 8 + i;
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
      int h = bond_sign(bonds, n, 0) * s[xp] + bond_sign(bonds, xm, 0) * s[xm] + bond_sign(bonds, n, 1) * s[yp] +
              bond_sign(bonds, ym, 1) * s[ym];
      if (ND == 3) {
        const int64_t LxLy = (int64_t)Lx * Ly;
        const int64_t zm = n + (int64_t)((z == 0 ? Lz - 1 : z - 1) - z) * LxLy;
        const int64_t zp = n + (int64_t)((z + 1 == Lz ? 0 : z + 1) - z) * LxLy;
        h += bond_sign(bonds, n, 2) * s[zp] + bond_sign(bonds, zm, 2) * s[zm];
      }
      const int dE = 2 * sn * h;
      const int idx = dE / 4;
      bool accept;
      if (idx <= 0) {
        accept = true;
      } else {
        const uint32_t uh = half16(P, (uint32_t)i);
        const uint32_t th = thr_hi(idx, T);
        if (uh != th) {
          accept = uh < th;
        } else {
          if (!have_lo) {
            Q = philox10((uint32_t)gidx, sweep, (uint32_t)c | (kMetroLo << 1), stream_id, K);
            have_lo = true;
          }
          accept = half16(Q, (uint32_t)i) < thr_lo(idx, T);
        }
      }
      if (accept) {
        s[n] = (int8_t)(-sn);
        de += dE;
        dm -= 2 * sn;
      }
    }
  }
  block_accumulate(de, dm, acc);
}

cudaError_t launch_sweep_generic(const Lattice& g, int8_t* s, const ThrTab& T, const PhiloxKeys& K,
                                 uint32_t stream_id, uint32_t sweep, unsigned long long* acc, cudaStream_t st) {
  const int64_t ngroups = ((g.N >> 1) + 7) >> 3;
  const int threads = 256;
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
  return cudaGetLastError();
}

// ---------------------------------------------------------- streaming sweep

namespace {

constexpr int kNbuf = 6;             // slice buffers in the ring (prefetch distance 2)
constexpr int kMaxA = 2;             // colour-0 chunks a thread holds between barriers
constexpr uint32_t kAnti = 0x02020202u;
constexpr unsigned kWaitLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bulk asynchronous copy global -> shared (the TMA engine, non-tensor form);
// both addresses 16-byte aligned and bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

struct StreamArgs {
  const int8_t* in;
  int8_t* out;
  int Lx, Ly, Lz;
  int TX, TY;  // TY = 1 in 2D
  int nseg;
  int S;       // slices along the streamed axis (2D: Ly, 3D: Lz)
  uint32_t sweep, stream_id;
  PhiloxKeys K;
  ThrTab T;
  unsigned long long* acc;
  int* err;
};

// Metropolis update of the colour-c sites of one 16-byte chunk.  C: the chunk,
// V: NV vertical neighbour chunks, lb / rb: the bytes left / right of the
// chunk, par: byte parity of the colour-c sites, P: Philox high-half output of
// the chunk's group.  Returns the new chunk; adds dE, dM of accepted moves.
template <int NV>
__device__ __forceinline__ uint4 chunk_update(uint4 C, const uint4 (&V)[NV], uint32_t lb, uint32_t rb, int par,
                                              const U4& P, uint32_t gidx, uint32_t c, const StreamArgs& a,
                                              int& de, int& dm) {
  constexpr int ND = NV / 2 + 1;
  const uint32_t w[4] = {C.x, C.y, C.z, C.w};
  uint32_t kx[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const uint32_t lw = __funnelshift_l(j == 0 ? (lb << 24) : w[j - 1], w[j], 8);
    const uint32_t rw = __funnelshift_r(w[j], j == 3 ? rb : w[j + 1], 8);
    uint32_t x = ((w[j] ^ lw) & kAnti) + ((w[j] ^ rw) & kAnti);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const uint32_t vw = j == 0 ? V[v].x : j == 1 ? V[v].y : j == 2 ? V[v].z : V[v].w;
      x += (w[j] ^ vw) & kAnti;
    }
    kx[j] = x;  // byte b holds 2 * (number of anti-aligned neighbours of site b)
  }
  uint32_t F[4] = {0, 0, 0, 0};
  uint32_t ties = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int j = i >> 1;
    const int b = par + 2 * (i & 1);
    const int k = (int)((kx[j] >> (8 * b + 1)) & 0xfu);
    const int idx = ND - k;  // dE / 4
    const uint32_t uh = half16(P, (uint32_t)i);
    const uint32_t th = thr_hi(idx, a.T);
    const bool acc = uh < th;
    ties |= (uh == th) ? (1u << i) : 0u;
    if (acc) {
      F[j] |= 0xfeu << (8 * b);
      de += 4 * idx;
      dm += ((w[j] >> (8 * b)) & 0x2u) ? 2 : -2;
    }
  }
  if (ties) {  // rare (probability ~2^-16 per site): draw the low halves
    const U4 Q = philox10(gidx, a.sweep, c | (kMetroLo << 1), a.stream_id, a.K);
#pragma unroll 1
    for (int i = 0; i < 8; ++i) {
      if (!((ties >> i) & 1)) continue;
      const int j = i >> 1;
      const int b = par + 2 * (i & 1);
      const int k = (int)((kx[j] >> (8 * b + 1)) & 0xfu);
      const int idx = ND - k;
      if (half16(Q, (uint32_t)i) < thr_lo(idx, a.T)) {
        F[j] |= 0xfeu << (8 * b);
        de += 4 * idx;
        dm += ((w[j] >> (8 * b)) & 0x2u) ? 2 : -2;
      }
    }
  }
  return make_uint4(w[0] ^ F[0], w[1] ^ F[1], w[2] ^ F[2], w[3] ^ F[3]);
}

__device__ __forceinline__ uint4 lds16(const uint8_t* p) { return *reinterpret_cast<const uint4*>(p); }

// Vertical neighbours of the chunk at p: the same chunk in the previous and
// next slice (pm, pp) and, in 3D, in the rows above and below (p -+ RS).
template <int ND>
__device__ __forceinline__ void load_vertical(uint4 (&V)[ND == 3 ? 4 : 2], const uint8_t* p, const uint8_t* pm,
                                              const uint8_t* pp, int RS) {
  if constexpr (ND == 3) {
    V[0] = lds16(p - RS);
    V[1] = lds16(p + RS);
    V[2] = lds16(pm);
    V[3] = lds16(pp);
  } else {
    V[0] = lds16(pm);
    V[1] = lds16(pp);
  }
}

template <int ND>
__global__ void __launch_bounds__(512) k_sweep_stream(StreamArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  constexpr int YH = (ND == 3) ? 2 : 0;       // y-halo rows on each side
  const int RS = a.TX + 32;                  // bytes per buffered row
  const int R = (ND == 3) ? a.TY + 4 : 1;    // rows per slice buffer
  const int SB = ((R * RS) + 127) & ~127;    // bytes per slice buffer
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kNbuf * SB);
  __shared__ int s_abort;

  const int tid = threadIdx.x, nth = blockDim.x;
  const int x0 = blockIdx.x * a.TX;
  const int y0 = (ND == 3) ? blockIdx.y * a.TY : 0;
  const int seg = blockIdx.z;
  const int zs = (int)(((int64_t)seg * a.S) / a.nseg);
  const int ze = (int)(((int64_t)(seg + 1) * a.S) / a.nseg);
  const int H = ze - zs;
  const int nload = H + 4;                   // slices zs-2 .. ze+1
  const int nck = a.TX >> 4;                 // chunks per row
  const int64_t sliceStride = (int64_t)a.Lx * ((ND == 3) ? a.Ly : 1);
  const uint32_t sliceBytes = (uint32_t)(R * RS);

  if (tid == 0) {
    s_abort = 0;
    for (int b = 0; b < kNbuf; ++b) mbar_init(&bars[b], 1);
    fence_mbar_init();
  }
  __syncthreads();

  auto gslice = [&](int li) { int z = zs - 2 + li; z %= a.S; if (z < 0) z += a.S; return z; };
  auto buf = [&](int li) { return smem + (li % kNbuf) * SB; };

  // Issue the copies of local slice li into its buffer (warp 0).
  auto issue = [&](int li) {
    if (li >= nload || tid >= 32) return;
    uint8_t* B = buf(li);
    uint64_t* bar = &bars[li % kNbuf];
    if (tid == 0) {
      fence_proxy_async();
      mbar_arrive_expect_tx(bar, sliceBytes);
    }
    __syncwarp();
    const int gz = gslice(li);
    const int xl = (x0 - 16 + a.Lx) % a.Lx, xr = (x0 + a.TX) % a.Lx;
    for (int r = tid; r < R; r += 32) {
      int gy;
      if (ND == 3) { gy = (y0 - YH + r) % a.Ly; if (gy < 0) gy += a.Ly; } else { gy = 0; }
      const int8_t* row = a.in + (int64_t)gz * sliceStride + (int64_t)gy * a.Lx;
      uint8_t* d = B + r * RS;
      bulk_g2s(d, row + xl, 16, bar);
      bulk_g2s(d + 16, row + x0, (uint32_t)a.TX, bar);
      bulk_g2s(d + 16 + a.TX, row + xr, 16, bar);
    }
  };

  // Bounded wait for local slice li; on timeout every thread learns it.
  auto wait_slice = [&](int li) -> bool {
    const uint32_t parity = (uint32_t)((li / kNbuf) & 1);
    unsigned n = 0;
    while (!mbar_try_wait(&bars[li % kNbuf], parity)) {
      if (++n > kWaitLimit) { s_abort = 1; break; }
    }
    return __syncthreads_or(s_abort) != 0;
  };

  for (int li = 0; li < kNbuf; ++li) issue(li);

  int de = 0, dm = 0;
  const int rowsA = (ND == 3) ? a.TY + 2 : 1;   // colour-0 rows: -1 .. TY (3D)
  const int nA = rowsA * nck;
  const int nRing = (ND == 3) ? a.TY : 1;       // one colour-0 ring site per owned row
  const int nB = ((ND == 3) ? a.TY : 1) * nck;

  // ---- colour-0 pass on local slice li (reads li-1, li, li+1), two barriers.
  auto passA = [&](int li) {
    const uint8_t* Bm = buf(li - 1);
    uint8_t* B0 = buf(li);
    const uint8_t* Bp = buf(li + 1);
    const int gz = gslice(li);
    const bool owned = (li >= 2 && li < H + 2);
    uint4 res[kMaxA];
    int rr[kMaxA], kk[kMaxA];
#pragma unroll
    for (int q = 0; q < kMaxA; ++q) {
      const int it = tid + q * nth;
      rr[q] = -100;
      if (it < nA) {
        const int r = (ND == 3) ? it / nck - 1 : 0;
        const int k = it - (r + ((ND == 3) ? 1 : 0)) * nck;
        int gy;
        if (ND == 3) { gy = (y0 + r) % a.Ly; if (gy < 0) gy += a.Ly; } else { gy = gz; }
        const int gzz = (ND == 3) ? gz : 0;
        const int par = (gy + gzz) & 1;  // colour 0
        const uint8_t* p = B0 + (r + YH) * RS + 16 + 16 * k;
        uint4 V[ND == 3 ? 4 : 2];
        load_vertical<ND>(V, p, Bm + (p - B0), Bp + (p - B0), RS);
        const uint32_t gidx = (uint32_t)((x0 >> 4) + k + (int64_t)(a.Lx >> 4) * (gy + (int64_t)a.Ly * gzz));
        const U4 P = philox10(gidx, a.sweep, 0u | (kMetroHi << 1), a.stream_id, a.K);
        int lde = 0, ldm = 0;
        res[q] = chunk_update(lds16(p), V, p[-1], p[16], par, P, gidx, 0u, a, lde, ldm);
        const bool own = owned && (ND == 2 || (r >= 0 && r < a.TY));
        if (own) { de += lde; dm += ldm; }
        rr[q] = r;
        kk[q] = k;
      }
    }
    // ring: the colour-0 one of x = x0 - 1 and x = x0 + TX in each owned row
    int ring_pos = -1;
    uint8_t ring_val = 0;
    int ring_r = 0;
    if (tid < nRing) {
      const int r = (ND == 3) ? tid : 0;
      int gy;
      if (ND == 3) { gy = (y0 + r) % a.Ly; } else { gy = gz; }
      const int gzz = (ND == 3) ? gz : 0;
      const int xl = (x0 - 1 + a.Lx) % a.Lx;
      const bool left = ((xl + gy + gzz) & 1) == 0;
      const int gx = left ? xl : (x0 + a.TX) % a.Lx;
      const int pos = left ? 15 : 16 + a.TX;
      const uint8_t* p = B0 + (r + YH) * RS + pos;
      const uint32_t sv = p[0];
      uint32_t k = ((sv ^ p[-1]) & 2u) + ((sv ^ p[1]) & 2u) + ((sv ^ Bm[p - B0]) & 2u) + ((sv ^ Bp[p - B0]) & 2u);
      if (ND == 3) k += ((sv ^ p[-RS]) & 2u) + ((sv ^ p[RS]) & 2u);
      const int idx = ND - (int)(k >> 1);
      const int64_t n = (int64_t)gx + (int64_t)a.Lx * (gy + (int64_t)a.Ly * gzz);
      const int64_t m = n >> 1;
      const uint32_t gidx = (uint32_t)(m >> 3);
      const uint32_t i = (uint32_t)(m & 7);
      const U4 P = philox10(gidx, a.sweep, 0u | (kMetroHi << 1), a.stream_id, a.K);
      const uint32_t uh = half16(P, i), th = thr_hi(idx, a.T);
      bool acc = uh < th;
      if (uh == th) {
        const U4 Q = philox10(gidx, a.sweep, 0u | (kMetroLo << 1), a.stream_id, a.K);
        acc = half16(Q, i) < thr_lo(idx, a.T);
      }
      ring_pos = pos;
      ring_r = r;
      ring_val = acc ? (uint8_t)(sv ^ 0xfeu) : (uint8_t)sv;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kMaxA; ++q)
      if (rr[q] != -100) *reinterpret_cast<uint4*>(B0 + (rr[q] + YH) * RS + 16 + 16 * kk[q]) = res[q];
    if (ring_pos >= 0) B0[(ring_r + YH) * RS + ring_pos] = ring_val;
    __syncthreads();
  };

  // ---- colour-1 pass on local slice li, result to global memory.
  auto passB = [&](int li) {
    const uint8_t* Bm = buf(li - 1);
    const uint8_t* B0 = buf(li);
    const uint8_t* Bp = buf(li + 1);
    const int gz = gslice(li);
    for (int it = tid; it < nB; it += nth) {
      const int r = (ND == 3) ? it / nck : 0;
      const int k = it - r * nck;
      const int gy = (ND == 3) ? y0 + r : gz;
      const int gzz = (ND == 3) ? gz : 0;
      const int par = (gy + gzz + 1) & 1;
      const uint8_t* p = B0 + (r + YH) * RS + 16 + 16 * k;
      uint4 V[ND == 3 ? 4 : 2];
      load_vertical<ND>(V, p, Bm + (p - B0), Bp + (p - B0), RS);
      const uint32_t gidx = (uint32_t)((x0 >> 4) + k + (int64_t)(a.Lx >> 4) * (gy + (int64_t)a.Ly * gzz));
      const U4 P = philox10(gidx, a.sweep, 1u | (kMetroHi << 1), a.stream_id, a.K);
      const uint4 o = chunk_update(lds16(p), V, p[-1], p[16], par, P, gidx, 1u, a, de, dm);
      int8_t* dst = a.out + (int64_t)gzz * sliceStride + (int64_t)gy * a.Lx + x0 + 16 * k;
      *reinterpret_cast<uint4*>(dst) = o;
    }
  };

  // Local slice li (global zs - 2 + li) lives in buffer li % kNbuf.  Step t
  // produces slice zs + t (local t + 2): colour 0 on local t + 3 (it needs old
  // t + 2 .. t + 4), then colour 1 on local t + 2 (mid t + 1 .. t + 3).  After
  // step t local t + 1 is dead and its buffer takes local t + 1 + kNbuf.
  int issued = kNbuf < nload ? kNbuf : nload;
  bool abort = false;
  for (int li = 0; li <= 3 && !abort; ++li) abort = wait_slice(li);
  if (!abort) passA(1);
  if (!abort) passA(2);
  if (!abort) { issue(kNbuf); issued = kNbuf + 1 < nload ? kNbuf + 1 : nload; }
  for (int t = 0; t < H && !abort; ++t) {
    abort = wait_slice(t + 4);
    if (abort) break;
    passA(t + 3);     // colour 0 on slice z+1
    passB(t + 2);     // colour 1 on slice z -> global
    __syncthreads();  // every thread is past passB(t + 2)
    issue(t + 1 + kNbuf);
    issued = t + 2 + kNbuf < nload ? t + 2 + kNbuf : nload;
  }

  if (abort) {
    if (tid == 0) {
      atomicExch(a.err, 1);
      // let the copies still in flight land before the CTA exits (bounded)
      for (int li = issued > kNbuf ? issued - kNbuf : 0; li < issued; ++li) {
        unsigned n = 0;
        while (!mbar_try_wait(&bars[li % kNbuf], (uint32_t)((li / kNbuf) & 1)) && ++n < kWaitLimit) {
        }
      }
    }
    __syncthreads();
    return;
  }
  long long lde = de, ldm = dm;
  block_accumulate(lde, ldm, a.acc);
}

}  // namespace

bool stream_path_supported(const Lattice& g, int TX, int TY) {
  if (g.bonds) return false;
  if (g.Lx % 16 || TX <= 0 || TX % 16 || g.Lx % TX) return false;
  if (g.nd == 3 && (TY <= 0 || g.Ly % TY)) return false;
  return true;
}

StreamGeom stream_geometry(const Lattice& g, int TX, int TY, int nseg) {
  StreamGeom s{};
  s.TX = TX;
  s.TY = g.nd == 3 ? TY : 1;
  const int R = g.nd == 3 ? TY + 4 : 1;
  const int SB = ((R * (TX + 32)) + 127) & ~127;
  s.nbuf = kNbuf;
  s.smem = (size_t)kNbuf * SB + kNbuf * sizeof(uint64_t);
  const int nck = TX / 16;
  const int nA = (g.nd == 3 ? TY + 2 : 1) * nck;
  int th = 32;
  while (th * kMaxA < nA || th < (g.nd == 3 ? TY : 1)) th += 32;
  s.threads = std::min(512, std::max(th, std::min(512, nck * (g.nd == 3 ? TY : 1))));
  const int S = g.nd == 3 ? g.Lz : g.Ly;
  if (nseg <= 0) {
    const int tiles = (g.Lx / TX) * (g.nd == 3 ? g.Ly / TY : 1);
    const int want = device_sm_count() * 4;
    nseg = std::max(1, std::min(S, (want + tiles - 1) / tiles));
  }
  s.nseg = std::min(nseg, S);
  return s;
}

cudaError_t launch_sweep_stream(const Lattice& g, const int8_t* in, int8_t* out, const StreamGeom& geo,
                                const ThrTab& T, const PhiloxKeys& K, uint32_t stream_id, uint32_t sweep,
                                unsigned long long* acc, int* err, cudaStream_t st) {
  StreamArgs a;
  a.in = in;
  a.out = out;
  a.Lx = g.Lx;
  a.Ly = g.Ly;
  a.Lz = g.Lz;
  a.TX = geo.TX;
  a.TY = geo.TY;
  a.nseg = geo.nseg;
  a.S = g.nd == 3 ? g.Lz : g.Ly;
  a.sweep = sweep;
  a.stream_id = stream_id;
  a.K = K;
  a.T = T;
  a.acc = acc;
  a.err = err;
  const int nck = geo.TX / 16;
  const int nA = (g.nd == 3 ? geo.TY + 2 : 1) * nck;
  if (nA > geo.threads * kMaxA || geo.threads > 512) return cudaErrorInvalidConfiguration;
  dim3 grid(g.Lx / geo.TX, g.nd == 3 ? g.Ly / geo.TY : 1, geo.nseg);
  if (g.nd == 3) {
    cudaFuncSetAttribute(k_sweep_stream<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)geo.smem);
    k_sweep_stream<3><<<grid, geo.threads, geo.smem, st>>>(a);
  } else {
    cudaFuncSetAttribute(k_sweep_stream<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)geo.smem);
    k_sweep_stream<2><<<grid, geo.threads, geo.smem, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace spn
