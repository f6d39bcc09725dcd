// Classical Heisenberg (O(3)) spins with the checkerboard Metropolis sweep:
// the continuous-spin generalisation Sec. 4 names for single-precision GPU
// arithmetic.  H = -sum_<ij> S_i . S_j (J = 1, |S| = 1), spins as binary32
// (x, y, z, 0) per site.  A site of colour c proposes a direction uniform on the
// sphere (Marsaglia's method) and takes it iff dE = -(S' - S) . h <= 0 or
// u < exp(-beta dE), h the sum of its 2 nd neighbours.
//
// Every floating-point step is one correctly rounded binary32 operation in a
// fixed order (the _rn intrinsics keep the compiler from fusing or reordering),
// and exp is computed by Cody-Waite reduction and a Taylor polynomial from
// those operations alone, so the lattice is bit-identical to any other
// implementation of the same steps.  Random words:
//   proposal call k (tries 2k, 2k+1 from words (0,1), (2,3)):
//     R(m, sweep, c | 5 << 1 | k << 4, stream), m = n >> 1, at most 8 calls;
//   hot start: the same with purpose 7 and sweep 0;
//   Metropolis u: word m & 3 of R(m >> 2, sweep, c | 6 << 1, stream).
//
// One launch updates one colour; a warp takes groups of 128 consecutive
// within-colour indices from a counter in global memory until none is left (the
// schedulers of an SM favour the warps of its first CTA, so a fixed share per
// warp left the last CTAs running alone at the end), a site per lane at a time: a lane's seven 16-byte loads are issued
// together, and each Metropolis Philox call (four sites' words) is drawn once
// per warp and passed to the lanes by shuffles.  A site whose first proposal
// call misses both tries (about 4.6% of sites) is not retried at once, which
// would run the warp through a second call for one or two lanes in most
// steps: it waits in a per-warp queue until 32 such sites have gathered, and
// the warp then finishes them together (same-colour sites are independent, so
// the order of their updates does not change the result).  The
// energy and magnetisation changes of accepted moves are added as 64-bit
// fixed-point integers in units of 2^-40 (each binary32 dE, dS rounded once to
// that grid), so the per-sweep sums are exact and independent of the order of
// the atomics.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "fastdiv.cuh"
#include "philox.cuh"
#include "spn.h"
#include "spn_internal.h"

namespace spn {
namespace {

enum : uint32_t { kHeisPropose = 5u, kHeisMetropolis = 6u, kHeisInit = 7u };

struct HeisArgs {
  float4* s;
  int nd, Lx, Ly, Lz;
  uint32_t half;  // sites per colour
  FastDiv div_h, div_ly;
  float beta;
  uint32_t sweep, stream_id, colour;
  PhiloxKeys K;
  unsigned long long* acc;  // [4]: dE, dMx, dMy, dMz of this sweep, two's complement in units of 2^-40
  unsigned long long* work;  // group counter: a warp takes group (counter - work_base) until none is left
  unsigned long long work_base;
  uint32_t ngroups;  // groups of 128 within-colour indices
};

__device__ __forceinline__ float heis_exp_dev(float x) {
  const float log2e = (float)(1.0 / 0.6931471805599453);
  const float ln2_hi = 45426.0f / 65536.0f;
  const float ln2_lo = (float)(0.6931471805599453 - 45426.0 / 65536.0);
  const float c7 = (float)(1.0 / 5040.0), c6 = (float)(1.0 / 720.0), c5 = (float)(1.0 / 120.0),
              c4 = (float)(1.0 / 24.0), c3 = (float)(1.0 / 6.0);
  if (x < -87.0f) return 0.0f;
  if (x > 0.0f) return 1.0f;
  const float kf = rintf(__fmul_rn(x, log2e));
  const float r = __fsub_rn(__fsub_rn(x, __fmul_rn(kf, ln2_hi)), __fmul_rn(kf, ln2_lo));
  float p = c7;
  p = __fadd_rn(__fmul_rn(p, r), c6);
  p = __fadd_rn(__fmul_rn(p, r), c5);
  p = __fadd_rn(__fmul_rn(p, r), c4);
  p = __fadd_rn(__fmul_rn(p, r), c3);
  p = __fadd_rn(__fmul_rn(p, r), 0.5f);
  p = __fadd_rn(__fmul_rn(p, r), 1.0f);
  p = __fadd_rn(__fmul_rn(p, r), 1.0f);
  return __fmul_rn(p, __int_as_float((127 + (int)kf) << 23));
}

// Proposal call k of site m: tries 2k and 2k+1, the first inside the unit disc
// taken.  Both pairs are formed and the accepted one selected without a
// branch, so the square root and the point are computed once (the same
// operations on the same values as taking the tries one after the other).
__device__ __forceinline__ bool proposal_call(const PhiloxKeys& K, uint32_t m, uint32_t t, uint32_t c, uint32_t purpose,
                                              uint32_t k, uint32_t stream, float3& out) {
  const U4 P = philox10(m, t, c | (purpose << 1) | (k << 4), stream, K);
  const float a1 = __fsub_rn(__fmul_rn(__uint2float_rn(P.x >> 8), 1.0f / 8388608.0f), 1.0f);
  const float a2 = __fsub_rn(__fmul_rn(__uint2float_rn(P.y >> 8), 1.0f / 8388608.0f), 1.0f);
  const float b1 = __fsub_rn(__fmul_rn(__uint2float_rn(P.z >> 8), 1.0f / 8388608.0f), 1.0f);
  const float b2 = __fsub_rn(__fmul_rn(__uint2float_rn(P.w >> 8), 1.0f / 8388608.0f), 1.0f);
  const float sa = __fadd_rn(__fmul_rn(a1, a1), __fmul_rn(a2, a2));
  const float sb = __fadd_rn(__fmul_rn(b1, b1), __fmul_rn(b2, b2));
  const bool first = sa < 1.0f;
  if (!first && !(sb < 1.0f)) return false;
  const float v1 = first ? a1 : b1, v2 = first ? a2 : b2, ss = first ? sa : sb;
  const float f = __fmul_rn(2.0f, __fsqrt_rn(__fsub_rn(1.0f, ss)));
  out = make_float3(__fmul_rn(v1, f), __fmul_rn(v2, f), __fsub_rn(1.0f, __fmul_rn(2.0f, ss)));
  return true;
}

// Site of within-colour index m of colour c.
template <int ND>
__device__ __forceinline__ uint32_t site_of(const HeisArgs& a, uint32_t m, uint32_t c, int& x, int& y, int& z) {
  const uint32_t row = fdiv(m, a.div_h);
  const int i = (int)(m - row * (uint32_t)(a.Lx >> 1));
  z = ND == 3 ? (int)fdiv(row, a.div_ly) : 0;
  y = (int)row - z * a.Ly;
  x = 2 * i + (int)((c ^ (uint32_t)(y + z)) & 1u);
  return (uint32_t)x + (uint32_t)a.Lx * row;
}

__device__ __forceinline__ void add3(float3& h, const float4 v) {
  h.x = __fadd_rn(h.x, v.x);
  h.y = __fadd_rn(h.y, v.y);
  h.z = __fadd_rn(h.z, v.z);
}

__device__ __forceinline__ void block_add4_fixed(long long v[4], unsigned long long* acc) {
  __shared__ long long red[32][4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int o = 16; o; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < 4; ++i) red[warp][i] = v[i];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      long long x = lane < nw ? red[lane][i] : 0;
#pragma unroll
      for (int o = 16; o; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (lane == 0 && x != 0) atomicAdd(&acc[i], (unsigned long long)x);
    }
  }
}

// binary32 value on the 2^-40 grid (exact scaling by a power of two, one rounding)
__device__ __forceinline__ long long fixed40(float v) { return __float2ll_rn(__fmul_rn(v, 1099511627776.0f)); }

__device__ __forceinline__ void block_add4(double v[4], double* acc) {
  __shared__ double red[32][4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int o = 16; o; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < 4; ++i) red[warp][i] = v[i];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      double x = lane < nw ? red[lane][i] : 0.0;
#pragma unroll
      for (int o = 16; o; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (lane == 0 && x != 0.0) atomicAdd(&acc[i], x);
    }
  }
}

// Neighbour sum h and own spin s of the site n of within-colour index m of
// colour c: the seven 16-byte loads are issued together (32-bit site indices:
// N < 2^31).
template <int ND>
__device__ __forceinline__ uint32_t heis_gather(const HeisArgs& a, uint32_t m, uint32_t c, float4& s, float3& h) {
  int x, y, z;
  const uint32_t n = site_of<ND>(a, m, c, x, y, z);
  const uint32_t sx = (uint32_t)a.Lx - 1u, sy = (uint32_t)a.Lx, wy = (uint32_t)(a.Ly - 1) * sy;
  const float4 bx = a.s[x == 0 ? n + sx : n - 1u];
  const float4 fx = a.s[x + 1 == a.Lx ? n - sx : n + 1u];
  const float4 by = a.s[y == 0 ? n + wy : n - sy];
  const float4 fy = a.s[y + 1 == a.Ly ? n - wy : n + sy];
  float4 bz = make_float4(0.0f, 0.0f, 0.0f, 0.0f), fz = bz;
  if constexpr (ND == 3) {
    const uint32_t sz = sy * (uint32_t)a.Ly, wz = (uint32_t)(a.Lz - 1) * sz;
    bz = a.s[z == 0 ? n + wz : n - sz];
    fz = a.s[z + 1 == a.Lz ? n - wz : n + sz];
  }
  s = a.s[n];
  h = make_float3(0.0f, 0.0f, 0.0f);
  add3(h, bx);
  add3(h, fx);
  add3(h, by);
  add3(h, fy);
  if constexpr (ND == 3) {
    add3(h, bz);
    add3(h, fz);
  }
  return n;
}

// Metropolis decision of Eq. 2 for the proposal prop of site n (own spin s,
// neighbour sum h, Metropolis word uw) and, if taken, the store and the
// fixed-point sums of dE and dS.
__device__ __forceinline__ void heis_decide(const HeisArgs& a, uint32_t n, const float4& s, const float3& h,
                                            const float3& prop, uint32_t uw, long long (&sum)[4]) {
  const float dx = __fsub_rn(prop.x, s.x), dy = __fsub_rn(prop.y, s.y), dz = __fsub_rn(prop.z, s.z);
  float dot = __fmul_rn(dx, h.x);
  dot = __fadd_rn(dot, __fmul_rn(dy, h.y));
  dot = __fadd_rn(dot, __fmul_rn(dz, h.z));
  const float de = -dot;
  bool accept = de <= 0.0f;
  if (!accept) {
    const float u = __fmul_rn(__uint2float_rn(uw >> 8), 1.0f / 16777216.0f);
    accept = u < heis_exp_dev(-__fmul_rn(a.beta, de));
  }
  if (accept) {
    a.s[n] = make_float4(prop.x, prop.y, prop.z, 0.0f);
    sum[0] += fixed40(de);
    sum[1] += fixed40(dx);
    sum[2] += fixed40(dy);
    sum[3] += fixed40(dz);
  }
}

constexpr int kHeisThreads = 256;
constexpr int kHeisQueue = 64;  // deferred sites per warp: fewer than 32 left after a drain, plus one pass

template <int ND>
__global__ void __launch_bounds__(kHeisThreads, 5) k_heis_half(const HeisArgs a) {
  // sites whose first proposal call missed twice, waiting for a full warp of
  // them: (m, Metropolis word) per entry
  __shared__ uint2 queue[kHeisThreads / 32][kHeisQueue];
  const uint32_t c = a.colour, lane = threadIdx.x & 31u;
  uint2* q = queue[threadIdx.x >> 5];
  const uint32_t below = (1u << lane) - 1u;
  long long sum[4] = {0, 0, 0, 0};
  uint32_t qn = 0;  // warp-uniform
  // a deferred site, on the lanes below `count`: its proposal calls 1 .. 7 (16
  // misses in all: no move), then the decision.  Same-colour sites are
  // independent, so the order of their updates changes nothing.
  auto drain = [&](uint32_t first, uint32_t count) {
    __syncwarp();
    if (lane < count) {
      const uint2 e = q[first + lane];
      float4 s;
      float3 h;
      const uint32_t n = heis_gather<ND>(a, e.x, c, s, h);
      float3 prop = make_float3(0.0f, 0.0f, 1.0f);
      bool got = false;
      for (uint32_t k = 1; k < 8u && !got; ++k) got = proposal_call(a.K, e.x, a.sweep, c, kHeisPropose, k, a.stream_id, prop);
      if (got) heis_decide(a, n, s, h, prop, e.y, sum);
    }
    __syncwarp();
  };
  // a warp takes 128 consecutive within-colour indices, 32 at a time; lane l
  // draws the Metropolis call of indices base + 4l .. base + 4l + 3 once.
  // Every warp ends after one add that finds no group left, so a launch adds
  // exactly ngroups + (warps of the grid) to the counter.
  for (;;) {
    uint32_t grp = 0;
    if (lane == 0) grp = (uint32_t)(atomicAdd(a.work, 1ull) - a.work_base);
    grp = __shfl_sync(0xffffffffu, grp, 0);
    if (grp >= a.ngroups) break;
    const uint32_t base = 128u * grp;
    const U4 U = philox10((base >> 2) + lane, a.sweep, c | (kHeisMetropolis << 1), a.stream_id, a.K);
#pragma unroll 1
    for (uint32_t i = 0; i < 4; ++i) {
      const uint32_t m = base + 32u * i + lane;
      const int src = (int)(8u * i + (lane >> 2));  // the lane holding call m >> 2
      const uint32_t w0 = __shfl_sync(0xffffffffu, U.x, src), w1 = __shfl_sync(0xffffffffu, U.y, src);
      const uint32_t w2 = __shfl_sync(0xffffffffu, U.z, src), w3 = __shfl_sync(0xffffffffu, U.w, src);
      const uint32_t uw = (m & 2u) ? ((m & 1u) ? w3 : w2) : ((m & 1u) ? w1 : w0);
      const bool live = m < a.half;
      uint32_t n = 0;
      float4 s = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      float3 h = make_float3(0.0f, 0.0f, 0.0f);
      if (live) n = heis_gather<ND>(a, m, c, s, h);
      // the first call's two tries; a site that misses both waits in the queue
      float3 prop = make_float3(0.0f, 0.0f, 1.0f);
      const bool got = live && proposal_call(a.K, m, a.sweep, c, kHeisPropose, 0u, a.stream_id, prop);
      const uint32_t miss = __ballot_sync(0xffffffffu, live && !got);
      if (live && !got) q[qn + __popc(miss & below)] = make_uint2(m, uw);
      qn += (uint32_t)__popc(miss);
      if (got) heis_decide(a, n, s, h, prop, uw, sum);
      if (qn >= 32u) {
        qn -= 32u;
        drain(qn, 32u);
      }
    }
  }
  if (qn) drain(0u, qn);
  block_add4_fixed(sum, a.acc);
}

__global__ void k_heis_init(float4* s, int nd, int Lx, int Ly, int64_t N, PhiloxKeys K, uint32_t stream, int cold) {
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
    if (cold) {
      s[n] = make_float4(0.0f, 0.0f, 1.0f, 0.0f);
      continue;
    }
    const int x = (int)(n % Lx);
    const int64_t r = n / Lx;
    const int y = (int)(r % Ly), z = nd == 3 ? (int)(r / Ly) : 0;
    const uint32_t c = (uint32_t)(x + y + z) & 1u;
    float3 p = make_float3(0.0f, 0.0f, 1.0f);
    for (uint32_t k = 0; k < 8; ++k)
      if (proposal_call(K, (uint32_t)(n >> 1), 0u, c, kHeisInit, k, stream, p)) break;
    s[n] = make_float4(p.x, p.y, p.z, 0.0f);
  }
}

// E = -sum_n sum_d S_n . S_{n+e_d}, M = sum S (binary64; products of binary32 values are exact)
__global__ void k_heis_observables(const float4* s, int nd, int Lx, int Ly, int Lz, int64_t N, double* out) {
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(n % Lx);
    const int64_t r = n / Lx;
    const int y = (int)(r % Ly), z = (int)(r / Ly);
    const float4 a = s[n];
    const int64_t f[3] = {n - x + (x + 1 == Lx ? 0 : x + 1), n + (int64_t)((y + 1 == Ly ? 0 : y + 1) - y) * Lx,
                          n + (int64_t)((z + 1 == Lz ? 0 : z + 1) - z) * Lx * Ly};
    for (int d = 0; d < nd; ++d) {
      const float4 b = s[f[d]];
      v[0] -= (double)a.x * b.x + (double)a.y * b.y + (double)a.z * b.z;
    }
    v[1] += a.x;
    v[2] += a.y;
    v[3] += a.z;
  }
  block_add4(v, out);
}

__global__ void k_heis_exp(const float* x, float* y, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = heis_exp_dev(x[i]);
}

int grid_for(int64_t threads_needed, int per_sm) {
  const int64_t want = (threads_needed + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)device_sm_count() * per_sm));
}

}  // namespace

bool heis_dims_ok(int nd, const int32_t* dims) {
  int64_t N = 1;
  for (int d = 0; d < nd; ++d) {
    if (dims[d] < 2 || (dims[d] & 1)) return false;
    N *= dims[d];
  }
  return N < ((int64_t)1 << 31);
}

cudaError_t launch_heis_init(float4* s, int nd, const int* L, int64_t N, uint64_t seed, uint32_t stream, bool cold,
                             cudaStream_t st) {
  k_heis_init<<<grid_for(N, 8), 256, 0, st>>>(s, nd, L[0], L[1], N, philox_keys(seed), stream, cold ? 1 : 0);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_heis_sweep(float4* s, int nd, const int* L, int64_t N, float beta, uint64_t seed,
                              uint32_t stream, uint32_t sweep, unsigned long long* acc, unsigned long long* work,
                              unsigned long long* work_base, cudaStream_t st) {
  HeisArgs a;
  a.s = s;
  a.nd = nd;
  a.Lx = L[0];
  a.Ly = L[1];
  a.Lz = nd == 3 ? L[2] : 1;
  a.half = (uint32_t)(N / 2);
  a.div_h = fastdiv((uint32_t)(L[0] / 2));
  a.div_ly = fastdiv((uint32_t)L[1]);
  a.beta = beta;
  a.sweep = sweep;
  a.stream_id = stream;
  a.K = philox_keys(seed);
  a.acc = acc;
  const int grid = grid_for(((int64_t)a.half + 3) / 4, 5);  // a thread per four sites (a warp per 128)
  a.work = work;
  a.ngroups = (a.half + 127u) / 128u;
  for (uint32_t c = 0; c < 2; ++c) {
    a.colour = c;
    a.work_base = *work_base;
    *work_base += a.ngroups + (unsigned long long)grid * 8u;
    if (nd == 3)
      k_heis_half<3><<<grid, 256, 0, st>>>(a);
    else
      k_heis_half<2><<<grid, 256, 0, st>>>(a);
  }
  count_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_heis_observables(const float4* s, int nd, const int* L, int64_t N, double* out4,
                                    cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out4, 0, 4 * sizeof(double), st);
  if (e != cudaSuccess) return e;
  k_heis_observables<<<grid_for(N, 4), 256, 0, st>>>(s, nd, L[0], L[1], nd == 3 ? L[2] : 1, N, out4);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_heis_exp(const float* x, float* y, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_heis_exp<<<(n + 255) / 256, 256, 0, st>>>(x, y, n);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace spn

// ---------------------------------------------------------------- handles

struct HeisState {
  int nd = 2;
  int L[3] = {0, 0, 1};
  int64_t N = 0;
  float4* d_s = nullptr;
  unsigned long long* d_acc = nullptr;  // [cap][4] per-sweep (dE, dM) since `folded`, units of 2^-40
  int64_t acc_cap = 0;
  uint64_t folded = 0;
  double* d_obs = nullptr;
  unsigned long long* d_work = nullptr;  // group counter of the sweep kernel
  double E = 0.0, M[3] = {0.0, 0.0, 0.0};
  std::vector<double> traceE, traceM;
};

namespace {

int heis_fail(int code, const char* msg) {
  spn::set_last_error(msg);
  return code;
}

int heis_recompute(spn_ctx* h, double* E, double* M) {
  HeisState* s = h->heis;
  if (spn::launch_heis_observables(s->d_s, s->nd, s->L, s->N, s->d_obs, h->st) != cudaSuccess)
    return heis_fail(SPN_E_CUDA, "Heisenberg observables launch");
  double r[4];
  if (cudaMemcpyAsync(r, s->d_obs, sizeof r, cudaMemcpyDeviceToHost, h->st) != cudaSuccess ||
      cudaStreamSynchronize(h->st) != cudaSuccess)
    return heis_fail(SPN_E_CUDA, "reading the Heisenberg observables");
  *E = r[0];
  for (int i = 0; i < 3; ++i) M[i] = r[1 + i];
  return SPN_OK;
}

int heis_fold(spn_ctx* h) {
  HeisState* s = h->heis;
  if (cudaStreamSynchronize(h->st) != cudaSuccess) return heis_fail(SPN_E_CUDA, "cudaStreamSynchronize");
  const int64_t live = (int64_t)(h->sweeps - s->folded);
  if (live <= 0) return SPN_OK;
  std::vector<unsigned long long> d((size_t)live * 4);
  if (cudaMemcpy(d.data(), s->d_acc, d.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost) != cudaSuccess)
    return heis_fail(SPN_E_CUDA, "reading the Heisenberg trace");
  const double unit = 1.0 / 1099511627776.0;  // 2^-40
  for (int64_t i = 0; i < live; ++i) {
    s->E += (double)(long long)d[4 * i] * unit;
    for (int k = 0; k < 3; ++k) s->M[k] += (double)(long long)d[4 * i + 1 + k] * unit;
    s->traceE.push_back(s->E);
    for (int k = 0; k < 3; ++k) s->traceM.push_back(s->M[k]);
  }
  s->folded = h->sweeps;
  if (cudaMemsetAsync(s->d_acc, 0, (size_t)s->acc_cap * 4 * sizeof(unsigned long long), h->st) != cudaSuccess)
    return heis_fail(SPN_E_CUDA, "clearing the Heisenberg trace");
  return SPN_OK;
}

int heis_ensure_acc(spn_ctx* h, int64_t n) {
  HeisState* s = h->heis;
  const int64_t need = (int64_t)(h->sweeps - s->folded) + n;
  if (need <= s->acc_cap) return SPN_OK;
  int rc = heis_fold(h);  // empties the device deltas, so the buffer can be replaced
  if (rc) return rc;
  int64_t cap = std::max<int64_t>(1024, s->acc_cap);
  while (cap < n) cap *= 2;
  cudaFree(s->d_acc);
  s->d_acc = nullptr;
  if (cudaMalloc(&s->d_acc, (size_t)cap * 4 * sizeof(unsigned long long)) != cudaSuccess)
    return heis_fail(SPN_E_NOMEM, "cudaMalloc(Heisenberg trace)");
  if (cudaMemsetAsync(s->d_acc, 0, (size_t)cap * 4 * sizeof(unsigned long long), h->st) != cudaSuccess)
    return heis_fail(SPN_E_CUDA, "clearing the Heisenberg trace");
  s->acc_cap = cap;
  return SPN_OK;
}

int heis_reset(spn_ctx* h, int init) {
  HeisState* s = h->heis;
  if (spn::launch_heis_init(s->d_s, s->nd, s->L, s->N, h->seed, h->stream_id, init == SPN_INIT_COLD, h->st) !=
      cudaSuccess)
    return heis_fail(SPN_E_CUDA, "Heisenberg init launch");
  return heis_recompute(h, &s->E, s->M);
}

}  // namespace

namespace spn {

bool is_heis_model(int model) { return model == SPN_HEIS2D || model == SPN_HEIS3D; }

void heis_free(HeisState* s) {
  if (!s) return;
  cudaFree(s->d_s);
  cudaFree(s->d_acc);
  cudaFree(s->d_obs);
  cudaFree(s->d_work);
  delete s;
}

int heis_create(spn_ctx* h, const int32_t* dims, int init) {
  HeisState* s = new (std::nothrow) HeisState;
  if (!s) return heis_fail(SPN_E_NOMEM, "host allocation failed");
  h->heis = s;
  s->nd = h->model == SPN_HEIS3D ? 3 : 2;
  if (!heis_dims_ok(s->nd, dims)) return heis_fail(SPN_E_ARG, "extents must be even, >= 2, and N < 2^31");
  s->N = 1;
  for (int d = 0; d < s->nd; ++d) {
    s->L[d] = dims[d];
    s->N *= dims[d];
  }
  if (cudaMalloc(&s->d_s, (size_t)s->N * sizeof(float4)) != cudaSuccess ||
      cudaMalloc(&s->d_obs, 4 * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&s->d_work, sizeof(unsigned long long)) != cudaSuccess)
    return heis_fail(SPN_E_NOMEM, "cudaMalloc(Heisenberg lattice)");
  int rc = heis_ensure_acc(h, 1024);
  if (rc) return rc;
  return heis_reset(h, init);
}

int heis_sweep(spn_ctx* h, double beta, int64_t nsweeps) {
  HeisState* s = h->heis;
  int rc = heis_ensure_acc(h, nsweeps);
  if (rc) return rc;
  const float bf = (float)beta;
  unsigned long long work_base = 0;
  if (nsweeps > 0 && cudaMemsetAsync(s->d_work, 0, sizeof(unsigned long long), h->st) != cudaSuccess)
    return heis_fail(SPN_E_CUDA, "clearing the Heisenberg group counter");
  for (int64_t t = 0; t < nsweeps; ++t) {
    const uint32_t sweep = (uint32_t)(h->sweeps + t);
    unsigned long long* acc = s->d_acc + 4 * (int64_t)(sweep - s->folded);
    const cudaError_t e =
        launch_heis_sweep(s->d_s, s->nd, s->L, s->N, bf, h->seed, h->stream_id, sweep, acc, s->d_work, &work_base, h->st);
    if (e != cudaSuccess) {
      h->sweeps += (uint64_t)t;
      return heis_fail(SPN_E_CUDA, cudaGetErrorString(e));
    }
  }
  h->sweeps += (uint64_t)nsweeps;
  return SPN_OK;
}

int heis_reinit(spn_ctx* h, int init) {
  HeisState* s = h->heis;
  int rc = heis_fold(h);
  if (rc) return rc;
  s->traceE.clear();
  s->traceM.clear();
  s->folded = 0;
  return heis_reset(h, init);
}

}  // namespace spn

extern "C" {

static int heis_handle(spn_handle h) {
  if (!h) return heis_fail(SPN_E_ARG, "handle is NULL");
  if (!h->heis) return heis_fail(SPN_E_STATE, "not a Heisenberg handle");
  return SPN_OK;
}

int spn_heis_get_spins(spn_handle h, float* xyz, size_t count) {
  int rc = heis_handle(h);
  if (rc) return rc;
  HeisState* s = h->heis;
  if (!xyz || count != (size_t)s->N * 3) return heis_fail(SPN_E_ARG, "xyz must hold 3 N floats");
  std::vector<float4> v((size_t)s->N);
  if (cudaMemcpyAsync(v.data(), s->d_s, v.size() * sizeof(float4), cudaMemcpyDeviceToHost, h->st) != cudaSuccess ||
      cudaStreamSynchronize(h->st) != cudaSuccess)
    return heis_fail(SPN_E_CUDA, "reading the spins");
  for (size_t n = 0; n < v.size(); ++n) {
    xyz[3 * n] = v[n].x;
    xyz[3 * n + 1] = v[n].y;
    xyz[3 * n + 2] = v[n].z;
  }
  return SPN_OK;
}

int spn_heis_set_spins(spn_handle h, const float* xyz, size_t count) {
  int rc = heis_handle(h);
  if (rc) return rc;
  HeisState* s = h->heis;
  if (!xyz || count != (size_t)s->N * 3) return heis_fail(SPN_E_ARG, "xyz must hold 3 N floats");
  if ((rc = heis_fold(h))) return rc;
  std::vector<float4> v((size_t)s->N);
  for (size_t n = 0; n < v.size(); ++n) v[n] = make_float4(xyz[3 * n], xyz[3 * n + 1], xyz[3 * n + 2], 0.0f);
  if (cudaMemcpy(s->d_s, v.data(), v.size() * sizeof(float4), cudaMemcpyHostToDevice) != cudaSuccess)
    return heis_fail(SPN_E_CUDA, "writing the spins");
  return heis_recompute(h, &s->E, s->M);
}

int spn_heis_observables(spn_handle h, double* E, double* M) {
  int rc = heis_handle(h);
  if (rc) return rc;
  if (!E || !M) return heis_fail(SPN_E_ARG, "NULL argument");
  if ((rc = heis_fold(h))) return rc;
  *E = h->heis->E;
  for (int i = 0; i < 3; ++i) M[i] = h->heis->M[i];
  return SPN_OK;
}

int spn_heis_recompute(spn_handle h, double* E, double* M) {
  int rc = heis_handle(h);
  if (rc) return rc;
  if (!E || !M) return heis_fail(SPN_E_ARG, "NULL argument");
  return heis_recompute(h, E, M);
}

int spn_heis_trace(spn_handle h, double* E, double* M, int64_t cap, int64_t* n) {
  int rc = heis_handle(h);
  if (rc) return rc;
  if (!n || cap < 0 || (cap > 0 && (!E || !M))) return heis_fail(SPN_E_ARG, "bad trace arguments");
  if ((rc = heis_fold(h))) return rc;
  HeisState* s = h->heis;
  const int64_t total = (int64_t)s->traceE.size();
  const int64_t k = std::min(cap, total);
  if (k > 0) {
    std::memcpy(E, s->traceE.data(), (size_t)k * sizeof(double));
    std::memcpy(M, s->traceM.data(), (size_t)k * 3 * sizeof(double));
  }
  *n = total;
  return SPN_OK;
}

int spn_test_heis_exp(const float* x, float* y, size_t n) {
  if (!x || !y) return heis_fail(SPN_E_ARG, "NULL argument");
  if (n == 0) return SPN_OK;
  if (n > (size_t)1 << 28) return heis_fail(SPN_E_ARG, "n too large");
  float *dx = nullptr, *dy = nullptr;
  cudaError_t e = cudaMalloc(&dx, n * 4);
  if (e == cudaSuccess) e = cudaMalloc(&dy, n * 4);
  if (e == cudaSuccess) e = cudaMemcpy(dx, x, n * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = spn::launch_heis_exp(dx, dy, (int)n, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(y, dy, n * 4, cudaMemcpyDeviceToHost);
  cudaFree(dx);
  cudaFree(dy);
  return e == cudaSuccess ? SPN_OK : heis_fail(SPN_E_CUDA, cudaGetErrorString(e));
}

}  // extern "C"
