// Batched runs of many independent lattices (uneven sizes, temperatures and
// sweep counts) with one persistent, shared-memory-resident kernel.
//
// k_resident<ND, CLUSTER> pops instances from a queue (longest first).  A CTA,
// or a thread-block cluster of CS CTAs when the lattice is too large for one
// CTA, holds the whole lattice bit-packed in shared memory -- even-x and odd-x
// words per row, the layout of the streaming kernel -- and runs every sweep of
// the instance there: hot start, E/M, colour 0, colour 1, the per-sweep E/M
// trace, and the int8 result at the end.  Each CTA of a cluster owns a band of
// rows and reads its neighbours' boundary rows through distributed shared
// memory; a cluster barrier separates the two colours.  The update order, the
// Philox planes and the thresholds are those of every other path, so results
// are bit-identical to one-instance-at-a-time runs.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "philox.cuh"
#include "spn_internal.h"
#include "fastdiv.cuh"
#include "sweep_common.cuh"

namespace cg = cooperative_groups;

namespace spn {

namespace {

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// AL: an instance may have a class with dE > 0 that is always accepted; else
// that test is left out (ResArgs.no_always)
template <int ND, bool CLUSTER, bool AL>
__global__ void __launch_bounds__(512) k_resident(ResArgs a) {  // every caller launches at most 512 threads
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ int s_idx;
  __shared__ long long s_em[2];
  __shared__ uint32_t s_tm[3][32];  // 0 / ~0: bit 31 - p of the instance's threshold of class q
  const int tid = threadIdx.x, nth = blockDim.x;
  // Extents of the current instance (instances of one launch may differ).  A
  // row is W words per parity; every word holds 32 sites but the last, which
  // holds vbl (its unused high bits stay zero).
  int Lx = 2, Ly = 2, Lz = 1, nrow = 2, W = 1, vbl = 1, rpc = 2, own = 2;
  bool vec_io = false;  // whole 64-byte spans, 16-byte aligned
  auto vbits = [&](int j) { return j == W - 1 ? vbl : 32; };
  auto vmaskj = [&](int j) { return j == W - 1 && vbl < 32 ? ((1u << vbl) - 1u) : 0xffffffffu; };
  int CS = 1, rank = 0;
  if constexpr (CLUSTER) {
    CS = (int)cg::this_cluster().num_blocks();
    rank = (int)cg::this_cluster().block_rank();
  }
  uint2* lut = reinterpret_cast<uint2*>(smem);               // 256 entries
  uint32_t* bits = reinterpret_cast<uint32_t*>(smem + 2048);  // rpc rows x 2W words

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

  auto sync_all = [&]() {
    if constexpr (CLUSTER) cg::this_cluster().sync(); else __syncthreads();
  };
  // divisions by the instance's W, Ly and rows per CTA (set per instance)
  FastDiv fW{1, 0, 0}, fLy{1, 0, 0}, fRpc{1, 0, 0};
  // word pointer of global row r (possibly in another CTA of the cluster)
  auto row_ptr = [&](int r) -> uint32_t* {
    if constexpr (!CLUSTER) {
      return bits + (size_t)r * 2 * W;  // one CTA owns every row
    } else {
      const int owner = (int)fdiv((uint32_t)r, fRpc), lr = r - owner * rpc;
      uint32_t* base = bits + (size_t)lr * 2 * W;
      if (owner != rank) return cg::this_cluster().map_shared_rank(base, owner);
      return base;
    }
  };

  while (true) {
    // the cluster's rank-0 CTA takes the next instance from the queue
    if (rank == 0 && tid == 0) s_idx = atomicAdd(a.counter, 1);
    sync_all();
    int idx;
    if constexpr (CLUSTER) {
      idx = *cg::this_cluster().map_shared_rank(&s_idx, 0);
    } else {
      idx = s_idx;
    }
    sync_all();  // everybody has read s_idx before it is overwritten
    if (idx >= a.ninst) break;
    const ResInst in = a.inst[a.order[idx]];
    if (in.tns && rank == 0 && tid == 0) in.tns[0] = globaltimer_ns();
    const PhiloxKeys K = philox_keys(in.seed);
    Lx = in.Lx;
    Ly = in.Ly;
    Lz = ND == 3 ? in.Lz : 1;
    nrow = Ly * Lz;
    W = (Lx + 63) >> 6;
    vbl = (Lx - 64 * (W - 1)) >> 1;
    vec_io = (Lx & 63) == 0;
    rpc = (nrow + CS - 1) / CS;  // rows per CTA; the last CTA of a cluster may own fewer
    fW = fastdiv((uint32_t)W);
    fLy = fastdiv((uint32_t)Ly);
    fRpc = fastdiv((uint32_t)rpc);
    const int r0 = rank * rpc;
    own = nrow - r0 < rpc ? (nrow - r0 > 0 ? nrow - r0 : 0) : rpc;

    // threshold planes of this instance for the decision (read after the sync below)
    for (int i = tid; i < ND * 32; i += nth) {
      const int q = i >> 5;  // class q: dE = 4 (q + 1); selects keep the instance in registers
      const uint32_t t = q == 0 ? in.T.t[1] : (q == 1 ? in.T.t[2] : in.T.t[3]);
      s_tm[q][i & 31] = 0u - ((t >> (31 - (i & 31))) & 1u);
    }

    // ---- load: hot start from Philox or the int8 lattice
    const int wordsOwn = own * 2 * W;
    for (int it = tid; it < wordsOwn; it += nth) {
      const int lr = it / (2 * W);
      const int rem = it - lr * 2 * W;
      const int p = rem / W, j = rem - p * W;
      const int r = r0 + lr;
      const int y = r % Ly, z = r / Ly;
      uint32_t wv = 0;
      if (in.init_hot) {
        const int c = (y + z + p) & 1;
        const uint32_t plane0 =
            philox10(8u * ((uint32_t)j + (uint32_t)W * (uint32_t)r), 0u, (uint32_t)c | (kInit << 1), in.stream, K).x;
        wv = plane0 & vmaskj(j);
      } else {
        const int8_t* row = in.spins + (int64_t)r * Lx;
        const int vb = vbits(j);
        for (int i = 0; i < vb; ++i) wv |= (row[64 * j + 2 * i + p] < 0 ? 1u : 0u) << i;
      }
      bits[(size_t)lr * 2 * W + p * W + j] = wv;
    }
    if (tid < 2) s_em[tid] = 0;
    sync_all();

    // anti-aligned counts of word j (parity par) of row r
    auto counts = [&](int r, int j, int par, uint32_t b, uint32_t& s0, uint32_t& s1, uint32_t& s2) {
      const uint32_t* row = row_ptr(r);
      const uint32_t* other = row + (1 - par) * W;
      const uint32_t o = other[j];
      uint32_t left, right;
      if (par == 0) {  // even x: x + 1 is odd lane i; x - 1 is odd lane i - 1, or the previous word's last site
        const int jm = j == 0 ? W - 1 : j - 1;
        right = o;
        left = (o << 1) | ((other[jm] >> (vbits(jm) - 1)) & 1u);
      } else {  // odd x: x - 1 is even lane i; x + 1 is even lane i + 1, or the next word's first site
        const int jp = j + 1 == W ? 0 : j + 1;
        left = o;
        right = (o >> 1) | ((other[jp] & 1u) << (vbits(j) - 1));
      }
      const int z = (int)fdiv((uint32_t)r, fLy), y = r - z * Ly;
      const int rym = y == 0 ? r + Ly - 1 : r - 1, ryp = y + 1 == Ly ? r - Ly + 1 : r + 1;
      const uint32_t ym = row_ptr(rym)[par * W + j], yp = row_ptr(ryp)[par * W + j];
      if constexpr (ND == 3) {
        const int rzm = z == 0 ? r + nrow - Ly : r - Ly, rzp = z + 1 == Lz ? r - nrow + Ly : r + Ly;
        const uint32_t zm = row_ptr(rzm)[par * W + j], zp = row_ptr(rzp)[par * W + j];
        count6(b ^ left, b ^ right, b ^ ym, b ^ yp, b ^ zm, b ^ zp, s0, s1, s2);
      } else {
        count4(b ^ left, b ^ right, b ^ ym, b ^ yp, s0, s1, s2);
      }
    };

    // ---- E and M of the start (E = -sum over colour-1 sites of (2ND - 2k))
    {
      long long e = 0, m = 0;
      const int items = own * W;
      for (int it = tid; it < items; it += nth) {
        const int lr = it / W, j = it - lr * W;
        const int r = r0 + lr;
        const int y = r % Ly, z = r / Ly;
        const int vb = vbits(j);
        const uint32_t vmask = vmaskj(j);
        for (int p = 0; p < 2; ++p) {
          const uint32_t b = bits[(size_t)lr * 2 * W + p * W + j];
          m += vb - 2 * __popc(b & vmask);
          if (((y + z + p) & 1) == 1) {  // colour 1
            uint32_t s0, s1, s2;
            counts(r, j, p, b, s0, s1, s2);
            e += -2LL * ND * vb + 2LL * (__popc(s0 & vmask) + 2 * __popc(s1 & vmask) + 4 * __popc(s2 & vmask));
          }
        }
      }
      warp_reduce_add2(e, m);
      if ((tid & 31) == 0) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&s_em[0]), (unsigned long long)e);
        atomicAdd(reinterpret_cast<unsigned long long*>(&s_em[1]), (unsigned long long)m);
      }
      __syncthreads();
      if (tid == 0 && in.em0) {
        atomicAdd(in.em0 + 0, (unsigned long long)s_em[0]);
        atomicAdd(in.em0 + 1, (unsigned long long)s_em[1]);
      }
    }

    // ---- sweeps
    const int items = own * W;
    const int rounds = (items + nth - 1) / nth;
    for (int t = 0; t < in.nsweeps; ++t) {
      const uint32_t sweep = in.sweep0 + (uint32_t)t;
      int de = 0, dm = 0;
      for (int c = 0; c < 2; ++c) {
        for (int q = 0; q < rounds; ++q) {  // warp-uniform trip count (votes in the decision)
          const int it = tid + q * nth;
          const bool live = it < items;
          const int itc = live ? it : 0;
          const int lr = (int)fdiv((uint32_t)itc, fW), j = itc - lr * W;
          const int r = r0 + lr;
          const int z = (int)fdiv((uint32_t)r, fLy), y = r - z * Ly;
          const int par = (y + z + c) & 1;
          uint32_t* wp = bits + (size_t)lr * 2 * W + par * W + j;
          const uint32_t b = *wp;
          uint32_t s0, s1, s2;
          counts(r, j, par, b, s0, s1, s2);
          const uint32_t valid = live ? vmaskj(j) : 0u;
          uint32_t cls[ND];
          uint32_t flips = classes<ND>(s0, s1, s2, valid, cls);
          const uint32_t c0 = 8u * ((uint32_t)j + (uint32_t)W * (uint32_t)r), c2 = (uint32_t)c | (kMetropolis << 1);
          uint32_t eq[ND];
#pragma unroll
          for (int k = 0; k < ND; ++k) {
            const bool always = AL && ((in.T.always >> (k + 1)) & 1u);
            flips |= always ? cls[k] : 0u;
            eq[k] = always ? 0u : cls[k];
          }
          // u < t on the top 12 planes of u (three Philox calls, drawn together
          // so their rounds interleave) with the threshold plane of each site's
          // class, then the planes beyond for a warp with a tie
          uint32_t pl[12];
#pragma unroll
          for (int call = 0; call < 3; ++call) {
            const U4 P = philox10(c0 + (uint32_t)call, sweep, c2, in.stream, K);
            pl[4 * call + 0] = P.x;
            pl[4 * call + 1] = P.y;
            pl[4 * call + 2] = P.z;
            pl[4 * call + 3] = P.w;
          }
          compare_top<ND, 12>(flips, eq, pl, s_tm);
          flips |= tail_planes<ND, 3>(eq, s_tm, K, c0, sweep, c2, in.stream);
          if (live) {
            tally<ND>(flips, b, s0, s1, s2, de, dm);
            *wp = b ^ flips;  // only this thread reads or writes this colour-c word in this phase
          }
        }
        sync_all();
      }
      long long lde = de, ldm = dm;
      warp_reduce_add2(lde, ldm);
      if ((tid & 31) == 0 && (lde | ldm) && in.trace) {
        atomicAdd(in.trace + 2 * t + 0, (unsigned long long)lde);
        atomicAdd(in.trace + 2 * t + 1, (unsigned long long)ldm);
      }
    }

    // ---- result: int8 lattice of the own rows
    for (int it = tid; it < own * W; it += nth) {
      const int lr = it / W, j = it - lr * W;
      const int r = r0 + lr;
      const uint32_t E = bits[(size_t)lr * 2 * W + j], O = bits[(size_t)lr * 2 * W + W + j];
      int8_t* row = in.spins + (int64_t)r * Lx;
      if (vec_io) {
        uint4* dst = reinterpret_cast<uint4*>(row + 64 * j);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const uint2 lo = lut[((E >> (8 * v)) & 0xfu) | (((O >> (8 * v)) & 0xfu) << 4)];
          const uint2 hi = lut[((E >> (8 * v + 4)) & 0xfu) | (((O >> (8 * v + 4)) & 0xfu) << 4)];
          dst[v] = make_uint4(lo.x, lo.y, hi.x, hi.y);
        }
      } else {
        const int vb = vbits(j);
        for (int i = 0; i < vb; ++i) {
          row[64 * j + 2 * i] = ((E >> i) & 1u) ? (int8_t)-1 : (int8_t)1;
          row[64 * j + 2 * i + 1] = ((O >> i) & 1u) ? (int8_t)-1 : (int8_t)1;
        }
      }
    }
    sync_all();  // the bits are reused by the next instance
    if (in.tns && rank == 0 && tid == 0) in.tns[1] = globaltimer_ns();
  }
}

}  // namespace

bool resident_supported(int nd, int Lx, int Ly, int Lz, int cs) {
  if (Lx < 2 || (Lx & 1)) return false;
  const int nrow = Ly * (nd == 3 ? Lz : 1);
  if (cs < 1 || cs > kMaxResidentCluster || nrow < cs) return false;
  return resident_smem(nd, Lx, Ly, Lz, cs) <= 200 * 1024;
}

size_t resident_smem(int nd, int Lx, int Ly, int Lz, int cs) {
  const int W = (Lx + 63) / 64;
  const int nrow = Ly * (nd == 3 ? Lz : 1);
  return (size_t)((nrow + cs - 1) / cs) * 2 * W * 4 + 256 * 8;
}

int resident_cluster_size(int nd, int Lx, int Ly, int Lz, int max_cs) {
  for (int cs = 1; cs <= max_cs; cs *= 2)
    if (resident_supported(nd, Lx, Ly, Lz, cs)) return cs;
  return 0;
}

namespace {

using ResKernel = void (*)(ResArgs);
ResKernel resident_kernel(int nd, int cs, bool al) {
  if (nd == 3)
    return cs > 1 ? (al ? k_resident<3, true, true> : k_resident<3, true, false>)
                  : (al ? k_resident<3, false, true> : k_resident<3, false, false>);
  return cs > 1 ? (al ? k_resident<2, true, true> : k_resident<2, true, false>)
                : (al ? k_resident<2, false, true> : k_resident<2, false, false>);
}

}  // namespace

cudaError_t launch_resident(const ResArgs& a, int nd, int cs, int threads, int ctas, size_t smem, cudaStream_t st) {
  const ResKernel fn = resident_kernel(nd, cs, !a.no_always);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && cs > 8) e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(ctas / cs * cs), 1, 1);
  cfg.blockDim = dim3((unsigned)threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  if (cs > 1) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  e = cudaLaunchKernelEx(&cfg, fn, a);
  count_launches(1);
  return e;
}

namespace {

int max_ctas_of(ResKernel fn, int cs, int threads, size_t smem) {
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (cs > 1) {
    // clusters are placed within one GPC: fewer fit than CTAs per SM x SMs suggests
    if (cs > 8) cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cs, 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, fn, &cfg) != cudaSuccess || nc <= 0) {
      cudaGetLastError();
      nc = 1;
    }
    return nc * cs;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
  if (per_sm <= 0) per_sm = 1;
  return per_sm * device_sm_count();
}

}  // namespace

// the fewer of the two kernels (with and without the always-accepted test)
int resident_max_ctas(int nd, int cs, int threads, size_t smem) {
  return std::min(max_ctas_of(resident_kernel(nd, cs, true), cs, threads, smem),
                  max_ctas_of(resident_kernel(nd, cs, false), cs, threads, smem));
}

}  // namespace spn
