// Wavefront streaming sweep of a large 3D Ising lattice (J = 1): one launch is
// one full sweep in the canonical two-colour order of Sec. 3 (all of colour 0,
// then all of colour 1), each int8 spin read from HBM once and written once.
//
// A CTA owns a band of TY rows (y) of a segment of planes [zs, ze) and walks
// down z.  Its compute warps own 32 / W consecutive rows of the band each (W
// 64-site words per row, one word per lane); a halo warp owns the rows just
// outside the band.  Every warp streams its own rows on its own:
//
//   * its int8 rows of each plane (2 KB; the halo warp: the two rows on each
//     side of the band) arrive by bulk asynchronous copies (TMA engine) into a
//     private ring of shared-memory slots, completed on the slot's mbarrier;
//   * each lane turns its 64 sites into colour-separated bit words (E: even x,
//     O: odd x, 32 sites per word) in a ring of four bit planes shared by the CTA;
//   * step k converts plane k+3, updates colour 0 of plane k+2 and colour 1 of
//     plane k+1, so that colour 1 of a plane sees the final colour-0 spins of
//     its plane and the planes above and below (the tile plus halo of Sec. 3);
//     the halo warp updates colour 0 of the rows next to the band, which the
//     band's edge rows need, from the spins before the sweep;
//   * a site's move is decided from its 6 neighbours by bit-sliced adders and
//     the uint32 compare u < floor(exp(-beta dE) 2^32) of Eq. 2, with u drawn
//     from Philox4x32-10 bit planes (top 12 planes for every site, further
//     planes for a warp with a tie);
//   * each row goes back to HBM as int8 (through a 256-entry table) once both
//     of its colours are final.
//
// The only coupling between warps is the y-neighbour of a warp's first and last
// rows, which lives in the neighbouring warp's rows: a warp starts step k once
// both neighbouring warps have finished step k - 1 (each warp arrives on a step
// mbarrier after a step; its neighbours wait on it, suspended in hardware), so
// warps run as a wavefront at most one step apart and no CTA-wide barrier is
// needed.  Planes next to a segment boundary and rows next to a band boundary
// are loaded (and their colour 0 updated) by both neighbouring CTAs; the
// counter-based random numbers make the copies identical.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "philox.cuh"
#include "spn_internal.h"
#include "sweep_common.cuh"

namespace spn {
namespace {

constexpr int kW3Compute = 8;                  // compute warps at most (TY = 32 / W rows each)
constexpr int kW3Warps = kW3Compute + 1;       // plus the halo warp
constexpr int kW3Ring = 3;                     // raw slots per warp
constexpr int kW3Planes = 4;                   // bit planes k .. k+3 live at step k
constexpr int kW3PkPlanes = 8;                 // bit-packed lattices: four more planes on their way
constexpr int kW3PkAhead = 4;                  // bit-packed: plane k + 3 + kW3PkAhead is requested at step k
constexpr int kW3Slot = 2048;                  // bytes of one raw slot
constexpr int kW3First = 3;                    // Philox calls of the first decision stage (12 planes)
// A CTA holds several units (band, segment) side by side, as many as one SM
// keeps resident, so that an SM runs one CTA: its schedulers favour the warps
// of the first of several CTAs, and the last CTA then ran alone at the end of
// the sweep.
constexpr int kW3MaxThreads = 3 * 32 * kW3Warps;  // three units of the largest band

struct Wave3Args {
  const int8_t* in;
  int8_t* out;
  int Lx, Ly, Lz, W;  // W: 64-site words per row (1, 2, 4 or 8)
  int TY, nwc, nseg;  // band rows, compute warps (TY = nwc * 32 / W), segments along z
  int units;          // units per CTA
  unsigned unit_smem;  // shared-memory bytes of one unit
  uint32_t sweep, stream_id;
  uint32_t always;     // bit q + 1: class q (dE = 4 (q + 1)) is always accepted
  PhiloxKeys K;
  uint32_t tm[3][32];  // 0 / ~0: bit 31 - p of the threshold of class q, plane p
  unsigned long long* acc;
  int* err;
  uint32_t wait_limit;  // polls of a bounded wait before it gives up
  uint32_t skip_first;  // test support: plane 0's copies are never issued
  const uint32_t* in_pk;  // bit-packed lattices: rows of RS words (W words of even-x sites, W of odd-x)
  uint32_t* out_pk;
  int RS;
};

size_t wave3_smem_packed(int TY, int W, int nwc) {
  return (size_t)kW3PkPlanes * (TY + 4) * 2 * W * 4 + (size_t)(nwc + 1) * 2 * 8;  // bit planes, step mbarriers
}

size_t wave3_smem(int TY, int W, int nwc) {
  const int nw = nwc + 1;
  return (size_t)nw * kW3Ring * kW3Slot                // raw slots
         + (size_t)kW3Planes * (TY + 4) * 2 * W * 4    // bit planes
         + 256 * 8                                     // int8 output table
         + (size_t)nw * kW3Ring * 8                    // copy mbarriers
         + (size_t)nw * 2 * 8;                         // step mbarriers (even / odd steps)
}

__device__ __forceinline__ void mbar_arrive3(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void cp_async4_w3(uint32_t* dst, const uint32_t* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// AL: some class with dE > 0 may be always accepted (beta = 0 or tiny), else that test is left out.
// PK: the lattice is bit-packed; a lane copies its E and O word of each of its
// rows straight into the plane ring (cp.async, a commit group per plane) and
// writes them back as they are, so no raw slots, no conversion, no int8 table.
template <bool AL, bool PK>
__global__ void __launch_bounds__(kW3MaxThreads, 1) k_sweep_wave3(const __grid_constant__ Wave3Args a) {
  constexpr int NC = 3;  // classes with dE > 0: dE = 4, 8, 12
  extern __shared__ __align__(128) uint8_t smem_all[];
  const int W = a.W, Lx = a.Lx, Ly = a.Ly, Lz = a.Lz, TY = a.TY, nwc = a.nwc;
  const int nw = nwc + 1, RPW = 32 / W, W2 = 2 * W, rows = TY + 4;
  const int lane = threadIdx.x & 31;
  const int sub = (int)(threadIdx.x >> 5) / nw;        // unit of this warp within the CTA
  const int warp = (int)(threadIdx.x >> 5) - sub * nw;  // warp within its unit
  const int tid = (int)threadIdx.x - 32 * nw * sub;     // thread within its unit
  uint8_t* smem = smem_all + (size_t)sub * a.unit_smem;
  const bool halo = warp == nwc;
  constexpr int NPL = PK ? kW3PkPlanes : kW3Planes;  // planes of the ring
  uint8_t* raw = smem + (size_t)warp * kW3Ring * kW3Slot;  // this warp's slots (int8)
  uint32_t* bits = PK ? reinterpret_cast<uint32_t*>(smem)
                      : reinterpret_cast<uint32_t*>(smem + (size_t)nw * kW3Ring * kW3Slot);
  uint2* lut = reinterpret_cast<uint2*>(bits + (size_t)kW3Planes * rows * W2);  // int8 only
  uint64_t* bars = reinterpret_cast<uint64_t*>(lut + 256) + warp * kW3Ring;   // int8 only
  uint64_t* steps = PK ? reinterpret_cast<uint64_t*>(bits + (size_t)kW3PkPlanes * rows * W2)
                       : reinterpret_cast<uint64_t*>(lut + 256) + nw * kW3Ring;  // [warp][2]
  const uint4* raw16 = reinterpret_cast<const uint4*>(raw);

  const int bands = Ly / TY;
  const int unit = (int)blockIdx.x * a.units + sub;  // (band, segment), band fastest
  const int useg = unit / bands;
  const int y0 = (unit - useg * bands) * TY;
  const int zs = (int)(((int64_t)useg * Lz) / a.nseg);
  const int ze = (int)(((int64_t)(useg + 1) * Lz) / a.nseg);
  const int H = ze - zs;
  const int nload = H + 4;  // local planes li = 0 .. H + 3 <-> global zs - 2 + li
  // warps to the left (smaller y) and right of this one: the halo warp sits
  // beyond both ends of the chain of compute warps
  const int wl = halo ? 0 : (warp == 0 ? nwc : warp - 1);
  const int wr = halo ? nwc - 1 : (warp == nwc - 1 ? nwc : warp + 1);

  // int8 pattern of 8 sites [e0 o0 e1 o1 e2 o2 e3 o3] for index e | o << 4
  for (int i = tid; !PK && i < 256; i += 32 * nw) {
    uint32_t lo = 0, hi = 0;
    for (int k = 0; k < 4; ++k) {
      const uint32_t pair = (((i >> k) & 1) ? 0xffu : 0x01u) | ((((i >> (4 + k)) & 1) ? 0xffu : 0x01u) << 8);
      if (k < 2) lo |= pair << (16 * k); else hi |= pair << (16 * (k - 2));
    }
    lut[i] = make_uint2(lo, hi);
  }
  if (lane == 0) {
    for (int b = 0; !PK && b < kW3Ring; ++b) mbar_init(&bars[b], 1);
    mbar_init(&steps[2 * warp], 1);
    mbar_init(&steps[2 * warp + 1], 1);
    fence_mbar_init();
  }
  __syncthreads();  // the table and the barriers; from here on warps only wait for their neighbours
  if (unit >= bands * a.nseg) return;  // an empty place of the last CTA

  auto gz = [&](int li) {  // global plane of local plane li
    int z = zs - 2 + li;
    z = z < 0 ? z + Lz : z;
    return z >= Lz ? z - Lz : z;
  };
  auto gy = [&](int rr) {  // global row of band row rr (-2 .. TY + 1)
    int y = y0 + rr;
    y = y < 0 ? y + Ly : y;
    return y >= Ly ? y - Ly : y;
  };
  // this warp's rows: a compute warp RPW rows from band row RPW * warp; the halo
  // warp the rows -2, -1, TY, TY + 1 (copied in two runs of two rows)
  const int r0 = halo ? -2 : RPW * warp;
  const int slotBytes = halo ? 4 * Lx : RPW * Lx;
  auto issue = [&](int li) {
    if (!PK && lane == 0 && li < nload) {
      uint64_t* bar = &bars[li % kW3Ring];
      uint8_t* dst = raw + (size_t)(li % kW3Ring) * kW3Slot;
      const int8_t* plane = a.in + (int64_t)gz(li) * Ly * Lx;
      fence_proxy_async();  // earlier generic reads of the slot before the async writes
      mbar_arrive_expect_tx(bar, (uint32_t)slotBytes);
      if (!(a.skip_first && li == 0)) {
        if (halo) {
          bulk_g2s(dst, plane + (int64_t)gy(-2) * Lx, (uint32_t)(2 * Lx), bar);
          bulk_g2s(dst + 2 * Lx, plane + (int64_t)gy(TY) * Lx, (uint32_t)(2 * Lx), bar);
        } else {
          bulk_g2s(dst, plane + (int64_t)(y0 + r0) * Lx, (uint32_t)slotBytes, bar);
        }
      }
    }
  };
  int issued = 0;
  if constexpr (!PK)
    for (; issued < kW3Ring && issued < nload; ++issued) issue(issued);

  const int rot = (lane >> 1) & 3;
  const uint32_t rot_sel = (uint32_t)(((0 - rot) & 3) | (((1 - rot) & 3) << 4) | (((2 - rot) & 3) << 8) |
                                      (((3 - rot) & 3) << 12));
  auto plane_bits = [&](int li) { return bits + (size_t)(li & (NPL - 1)) * rows * W2; };
  // conversion: lane -> (row of the slot, word); the halo warp's slot holds rows -2, -1, TY, TY + 1
  const int cslot_row = lane / W, cj = lane - (lane / W) * W;
  const bool cvalid = halo ? lane < 4 * W : true;
  const int crr = halo ? (cslot_row < 2 ? cslot_row - 2 : TY + cslot_row - 2) : r0 + cslot_row;
  // bit-packed: request plane li, this lane's E and O word of its row; one commit
  // group per call (an empty one past the last plane keeps the count)
  auto issue_pk = [&](int li) {
    if (cvalid && li < nload) {
      const uint32_t* src = a.in_pk + ((int64_t)gz(li) * Ly + gy(crr)) * a.RS;
      uint32_t* dst = plane_bits(li) + (size_t)(crr + 2) * W2;
      cp_async4_w3(dst + cj, src + cj);
      cp_async4_w3(dst + W + cj, src + W + cj);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };

  auto convert = [&](int li) -> bool {
    unsigned n = 0;
    while (!mbar_try_wait(&bars[li % kW3Ring], (uint32_t)((li / kW3Ring) & 1))) {
      if (++n > a.wait_limit) return false;
    }
    if (cvalid) {
      const uint32_t span = (uint32_t)(li % kW3Ring) * (kW3Slot >> 4) + (uint32_t)(cslot_row * (Lx >> 4) + 4 * cj);
      uint32_t pe[4], po[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const uint4 c = raw16[span + (uint32_t)((v + rot) & 3)];
        pe[v] = gather_e(c.x, c.y, c.z, c.w);
        po[v] = gather_o(c.x, c.y, c.z, c.w);
      }
      uint32_t* row = plane_bits(li) + (size_t)(crr + 2) * W2;
      row[cj] = __byte_perm(top_bytes(pe[0], pe[1], pe[2], pe[3]), 0u, rot_sel);
      row[W + cj] = __byte_perm(top_bytes(po[0], po[1], po[2], po[3]), 0u, rot_sel);
    }
    return true;
  };

  // update lanes: a compute warp's lane -> (band row, word); the halo warp's
  // first 2 W lanes -> rows -1 and TY (the rest repeat them and store nothing)
  const int ul = halo ? lane % W2 : lane;
  const int urr = halo ? (ul < W ? -1 : TY) : r0 + lane / W;
  const int uj = ul - (ul / W) * W;
  const bool ustore = halo ? lane < W2 : true;
  const int ubase = lane - uj;  // first lane of this lane's row group
  const int src_m = ubase + (uj == 0 ? W - 1 : uj - 1), src_p = ubase + (uj + 1 == W ? 0 : uj + 1);
  int de = 0, dm = 0;

  // colour c of local plane li: the lane's colour-c word is rewritten from the
  // other colour's words of its row (x), the rows above and below (y) and the
  // same row of the planes above and below (z); colour 1 also sends the
  // finished row out as int8
  auto update = [&](int li, int c) {
    const int z = gz(li), y = gy(urr);
    const int par = (y + z + c) & 1;  // 0: the E word holds colour c, 1: the O word
    const uint32_t* pm = plane_bits(li - 1) + (size_t)(urr + 2) * W2;
    uint32_t* p0 = plane_bits(li) + (size_t)(urr + 2) * W2;
    const uint32_t* pp = plane_bits(li + 1) + (size_t)(urr + 2) * W2;
    const int ws = par ? W + uj : uj, wo = par ? uj : W + uj;
    const uint32_t b = p0[ws], oj = p0[wo];
    // x - 1 of an even site 0 is the last odd site of the previous word; x + 1
    // of the odd site 31 is the first even site of the next word (periodic in x)
    const uint32_t onm = __shfl_sync(0xffffffffu, oj, src_m), onp = __shfl_sync(0xffffffffu, oj, src_p);
    const uint32_t left = par ? oj : (oj << 1) | (onm >> 31);
    const uint32_t right = par ? (oj >> 1) | (onp << 31) : oj;
    uint32_t s0, s1, s2, cls[NC];
    count6(b ^ left, b ^ right, b ^ p0[ws - W2], b ^ p0[ws + W2], b ^ pm[ws], b ^ pp[ws], s0, s1, s2);
    uint32_t acc = classes<3>(s0, s1, s2, 0xffffffffu, cls);
    uint32_t eq[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      const bool always = AL && ((a.always >> (k + 1)) & 1u);  // AL false: no class is (compile time)
      acc |= always ? cls[k] : 0u;
      eq[k] = always ? 0u : cls[k];
    }
    const uint32_t c0 = 8u * ((uint32_t)uj + (uint32_t)W * ((uint32_t)y + (uint32_t)Ly * (uint32_t)z));
    const uint32_t c2 = (uint32_t)c | (kMetropolis << 1);
    uint32_t pl[4 * kW3First];
#pragma unroll
    for (int call = 0; call < kW3First; ++call) {
      const U4 P = philox10(c0 + (uint32_t)call, a.sweep, c2, a.stream_id, a.K);
      pl[4 * call + 0] = P.x;
      pl[4 * call + 1] = P.y;
      pl[4 * call + 2] = P.z;
      pl[4 * call + 3] = P.w;
    }
    compare_top<NC, 4 * kW3First>(acc, eq, pl, a.tm);
    acc |= tail_planes<NC, kW3First>(eq, a.tm, a.K, c0, a.sweep, c2, a.stream_id);
    const uint32_t nb = b ^ acc;
    if (ustore) p0[ws] = nb;
    if (!halo && li >= 2 && li < H + 2) tally<3>(acc, b, s0, s1, s2, de, dm);
    if (c == 1 && PK) {
      uint32_t* o = a.out_pk + ((int64_t)z * Ly + y) * a.RS;
      o[uj] = par ? oj : nb;
      o[W + uj] = par ? nb : oj;
    } else if (c == 1) {
      const uint32_t E = par ? oj : nb, O = par ? nb : oj;
      const uint32_t X = (E & 0x0f0f0f0fu) | ((O << 4) & 0xf0f0f0f0u);  // byte v: sites 16v .. 16v + 7
      const uint32_t Y = ((E >> 4) & 0x0f0f0f0fu) | (O & 0xf0f0f0f0u);  // byte v: sites 16v + 8 .. 16v + 15
      uint4* dst = reinterpret_cast<uint4*>(a.out + ((int64_t)z * Ly + y) * Lx + 64 * uj);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const uint2 lo = lut[(X >> (8 * v)) & 0xffu];
        const uint2 hi = lut[(Y >> (8 * v)) & 0xffu];
        dst[v] = make_uint4(lo.x, lo.y, hi.x, hi.y);
      }
    }
  };

  // Completed steps of a warp: the c-th completion (c = 1, 2, ...) arrives on
  // the warp's step mbarrier c & 1, completing its phase (c - 1) >> 1.  A
  // neighbour is never more than one step ahead, so the phase waited for is
  // unambiguous; the wait suspends the warp in hardware.
  auto publish = [&](int c) {
    __syncwarp();
    if (lane == 0) mbar_arrive3(&steps[2 * warp + (c & 1)]);
  };
  auto wait_neighbours = [&](int c) -> bool {  // both neighbours have completed c steps
    const uint32_t par = (uint32_t)(((c - 1) >> 1) & 1);
    bool ok = true;
    unsigned n = 0;
    while (!mbar_try_wait(&steps[2 * wl + (c & 1)], par)) {
      if (++n > a.wait_limit) {
        ok = false;
        break;
      }
    }
    n = 0;
    while (ok && !mbar_try_wait(&steps[2 * wr + (c & 1)], par)) {
      if (++n > a.wait_limit) {
        ok = false;
        break;
      }
    }
    return __all_sync(0xffffffffu, ok);
  };

  // prologue (counts as step 1): planes 0, 1, 2 converted (bit-packed: landed); then colour 0 of plane 1
  bool ok = true;
  if constexpr (PK) {
    for (int li = 0; li < 3 + kW3PkAhead; ++li) issue_pk(li);
    asm volatile("cp.async.wait_group %0;" ::"n"(kW3PkAhead) : "memory");
    __syncwarp();
  } else {
    for (int li = 0; li < 3 && ok; ++li) {
      ok = __all_sync(0xffffffffu, convert(li));
      __syncwarp();
      if (ok) issue(issued++);
    }
  }
  if (ok) {
    publish(1);
    ok = wait_neighbours(1);
  }
  if (ok) {
    update(1, 0);
    publish(2);
  }
  // step k (counter k + 3): convert plane k + 3, colour 0 of plane k + 2,
  // colour 1 of plane k + 1 (owned planes 2 .. H + 1 only; compute warps only)
  for (int k = 0; ok && k <= H; ++k) {
    ok = wait_neighbours(k + 2);
    if (!ok) break;
    if constexpr (PK) {
      // the neighbours have finished step k - 1, the last to read plane k - 1:
      // its ring plane takes plane k + 3 + kW3PkAhead; plane k + 3 has landed
      __syncwarp();
      issue_pk(k + 3 + kW3PkAhead);
      asm volatile("cp.async.wait_group %0;" ::"n"(kW3PkAhead) : "memory");
      __syncwarp();
    } else {
      ok = __all_sync(0xffffffffu, convert(k + 3));
      if (!ok) break;
      __syncwarp();
      issue(issued++);
    }
    update(k + 2, 0);
    if (k >= 1 && !halo) update(k + 1, 1);
    publish(k + 3);
  }
  if (!ok && PK) {  // this warp gives up; its copies land before it exits
    if (lane == 0) atomicExch(a.err, 1);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncwarp();
    return;
  }
  if (!ok) {  // this warp gives up; its neighbours' waits then run out as well
    if (lane == 0) {
      atomicExch(a.err, 1);
      // let the copies still in flight land before the warp exits: every issued
      // plane gets the full poll bound, and a plane whose copy was never issued is skipped
      const int last = issued < nload ? issued : nload;
      for (int li = last > kW3Ring ? last - kW3Ring : 0; li < last; ++li) {
        if (a.skip_first && li == 0) continue;
        unsigned n = 0;
        while (!mbar_try_wait(&bars[li % kW3Ring], (uint32_t)((li / kW3Ring) & 1)) && ++n < kWaitLimit) {
        }
      }
    }
    __syncwarp();
    return;
  }
  if constexpr (PK) asm volatile("cp.async.wait_group 0;" ::: "memory");
  block_accumulate(de, dm, a.acc);
}

}  // namespace

bool wave3_supported(const Lattice& g, int TY) {
  if (g.nd != 3 || g.bonds) return false;
  if (g.pitch && g.pitch != g.Lx) return false;
  if (g.Lx % 64) return false;
  const int W = g.Lx / 64;
  if (W != 1 && W != 2 && W != 4 && W != 8) return false;
  const int RPW = 32 / W;
  if (TY < RPW || TY % RPW || TY / RPW > kW3Compute || g.Ly % TY) return false;
  return g.Lz >= 2;
}


namespace {

void set_wave3_attributes() {
  using W3Kernel = void (*)(Wave3Args);
  const W3Kernel ks[4] = {k_sweep_wave3<false, false>, k_sweep_wave3<true, false>, k_sweep_wave3<false, true>,
                          k_sweep_wave3<true, true>};
  for (W3Kernel k : ks) {
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  }
}

size_t unit_smem_of(int TY, int W, int nwc, bool pk) {
  return ((pk ? wave3_smem_packed(TY, W, nwc) : wave3_smem(TY, W, nwc)) + 127) & ~(size_t)127;
}

// Units one SM holds at once (from the occupancy of a one-unit CTA, within the
// thread and shared-memory limits of one CTA): the units of a CTA.
int units_per_cta(int TY, int W, int nwc, bool pk) {
  static std::mutex mu;
  static int per_sm[2][kW3Compute + 1][4] = {};  // [packed][compute warps][log2 W]
  const int lw = W == 1 ? 0 : W == 2 ? 1 : W == 4 ? 2 : 3;
  std::lock_guard<std::mutex> lock(mu);
  int& cached = per_sm[pk ? 1 : 0][nwc][lw];
  if (!cached) {
    const size_t sm = unit_smem_of(TY, W, nwc, pk);
    set_wave3_attributes();
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, pk ? k_sweep_wave3<false, true> : k_sweep_wave3<false, false>,
                                                      32 * (nwc + 1), sm) != cudaSuccess)
      blocks = 1;
    int u = std::max(1, blocks);
    u = std::min(u, kW3MaxThreads / (32 * (nwc + 1)));
    u = std::min<int>(u, (int)((227 * 1024) / sm));
    cached = std::max(1, u);
  }
  return cached;
}

}  // namespace

size_t wave3_smem_bytes(const Lattice& g, int TY, bool packed) {
  const int W = g.Lx / 64, nwc = TY / (32 / W);
  return (size_t)units_per_cta(TY, W, nwc, packed) * unit_smem_of(TY, W, nwc, packed);
}

int wave3_cta_threads(const Lattice& g, int TY, bool packed) {
  const int W = g.Lx / 64, nwc = TY / (32 / W);
  return 32 * (nwc + 1) * units_per_cta(TY, W, nwc, packed);
}

int wave3_default_segments(const Lattice& g, int TY, bool packed) {
  const int W = g.Lx / 64, nwc = TY / (32 / W);
  // one wave: a CTA per SM holding as many units as the SM keeps resident
  const int bands = g.Ly / TY;
  const int want = device_sm_count() * units_per_cta(TY, W, nwc, packed);
  return std::max(1, std::min(g.Lz, want / bands));
}

namespace {

// shared by the int8 and the bit-packed launch: in / out are int8 lattices or
// bit-packed rows (pk), the rest of the arguments as for launch_sweep_wave3
cudaError_t launch_w3(const Lattice& g, const void* in, void* out, bool pk, int TY, int nseg, const DevThr& T,
                      const PhiloxKeys& K, uint32_t stream_id, uint32_t sweep, unsigned long long* acc, int* err,
                      cudaStream_t st, uint32_t expire_polls) {
  if (!wave3_supported(g, TY) || nseg < 1 || nseg > g.Lz) return cudaErrorInvalidConfiguration;
  if (pk ? (((uintptr_t)in & 3) || ((uintptr_t)out & 3)) : (((uintptr_t)in & 15) || ((uintptr_t)out & 15)))
    return cudaErrorMisalignedAddress;  // int8: bulk copies and 16-byte stores; bit-packed: 4-byte copies
  Wave3Args a;
  a.in = pk ? nullptr : static_cast<const int8_t*>(in);
  a.out = pk ? nullptr : static_cast<int8_t*>(out);
  a.in_pk = pk ? static_cast<const uint32_t*>(in) : nullptr;
  a.out_pk = pk ? static_cast<uint32_t*>(out) : nullptr;
  a.RS = packed_row_words(g.Lx);
  a.Lx = g.Lx;
  a.Ly = g.Ly;
  a.Lz = g.Lz;
  a.W = g.Lx / 64;
  a.TY = TY;
  a.nwc = TY / (32 / a.W);
  a.nseg = nseg;
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
  if (expire_polls) {  // plane 0 of every warp is never copied; waits give up after `expire_polls` polls
    a.skip_first = 1;
    a.wait_limit = expire_polls;
  }
  a.units = units_per_cta(TY, a.W, a.nwc, pk);
  a.unit_smem = (unsigned)unit_smem_of(TY, a.W, a.nwc, pk);
  const size_t sm = (size_t)a.units * a.unit_smem;
  {
    static std::mutex mu;
    static bool set[128] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    if (!set[dev & 127]) {
      set_wave3_attributes();
      set[dev & 127] = true;
    }
  }
  const int64_t units = (int64_t)(g.Ly / TY) * nseg;
  const unsigned grid = (unsigned)((units + a.units - 1) / a.units), block = 32 * (a.nwc + 1) * a.units;
  const bool al = (T.always & 14u) != 0;
  if (pk)
    (al ? k_sweep_wave3<true, true> : k_sweep_wave3<false, true>)<<<grid, block, sm, st>>>(a);
  else
    (al ? k_sweep_wave3<true, false> : k_sweep_wave3<false, false>)<<<grid, block, sm, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sweep_wave3(const Lattice& g, const int8_t* in, int8_t* out, int TY, int nseg, const DevThr& T,
                               const PhiloxKeys& K, uint32_t stream_id, uint32_t sweep, unsigned long long* acc,
                               int* err, cudaStream_t st, uint32_t expire_polls) {
  return launch_w3(g, in, out, false, TY, nseg, T, K, stream_id, sweep, acc, err, st, expire_polls);
}

cudaError_t launch_sweep_wave3_packed(const Lattice& g, const uint32_t* in, uint32_t* out, int TY, int nseg,
                                      const DevThr& T, const PhiloxKeys& K, uint32_t stream_id, uint32_t sweep,
                                      unsigned long long* acc, int* err, cudaStream_t st) {
  return launch_w3(g, in, out, true, TY, nseg, T, K, stream_id, sweep, acc, err, st, 0);
}

}  // namespace spn
