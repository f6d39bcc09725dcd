// spn_sweep_noalloc: sweeps of a caller-owned device lattice without any
// device allocation.
//
// Some callers cannot let a library call cudaMalloc: a host framework whose
// caching allocator has reserved the device memory (a raw allocation would
// fail or fragment its pool), plugin hosts that only hand out buffers, and
// latency-critical loops in which cudaMalloc / cudaFree would synchronise the
// device.  For them this entry point keeps its only scratch -- the second
// ping-pong lattice of the streaming sweep and an error word -- in fixed
// file-scope device arrays that every GPU loading the library holds until the
// process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "spn.h"
#include "spn_internal.h"

namespace {

constexpr size_t kScratchBytes = (size_t)16 << 20;  // ping-pong lattice: up to 16,777,216 sites

static __device__ __align__(256) int8_t g_scratch[kScratchBytes];
static __device__ __align__(256) int g_scratch_err[64];

struct DeviceScratch {
  int8_t* lattice = nullptr;
  int* err = nullptr;
};

std::mutex g_mu;
DeviceScratch g_dev[128];

// The device addresses of the scratch arrays, looked up once per device with
// that device current (the array names are host-side stand-ins in host code).
int scratch_for_device(int dev, DeviceScratch* out, const char** why) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (dev < 0 || dev >= 128) {
    *why = "device ordinal out of range";
    return SPN_E_ARG;
  }
  if (!g_dev[dev].lattice) {
    void* p = nullptr;
    void* e = nullptr;
    cudaError_t rc = cudaGetSymbolAddress(&p, g_scratch);
    if (rc != cudaSuccess) {
      *why = cudaGetErrorString(rc);
      return SPN_E_CUDA;
    }
    rc = cudaGetSymbolAddress(&e, g_scratch_err);
    if (rc != cudaSuccess) {
      *why = cudaGetErrorString(rc);
      return SPN_E_CUDA;
    }
    g_dev[dev].lattice = static_cast<int8_t*>(p);
    g_dev[dev].err = static_cast<int*>(e);
  }
  *out = g_dev[dev];
  return SPN_OK;
}

}  // namespace

extern "C" int spn_sweep_noalloc(int model, const int32_t* dims, int8_t* d_spins, double beta, uint64_t seed,
                                 uint32_t stream_id, uint32_t sweep0, int64_t nsweeps, int64_t* d_trace,
                                 void* cuda_stream) {
  auto fail = [](int code, const char* what) {
    char msg[256];
    std::snprintf(msg, sizeof msg, "spn_sweep_noalloc: %s", what);
    spn::set_last_error(msg);
    return code;
  };
  if (model != SPN_ISING2D && model != SPN_ISING3D) return fail(SPN_E_ARG, "model must be SPN_ISING2D or SPN_ISING3D");
  if (!dims || !d_spins || !d_trace) return fail(SPN_E_ARG, "NULL argument");
  if (!(beta >= 0.0)) return fail(SPN_E_ARG, "beta must be >= 0");
  if (nsweeps < 0) return fail(SPN_E_ARG, "nsweeps must be >= 0");
  spn::Lattice g;
  g.nd = model == SPN_ISING2D ? 2 : 3;
  g.Lx = dims[0];
  g.Ly = dims[1];
  g.Lz = g.nd == 3 ? dims[2] : 1;
  const int ext[3] = {g.Lx, g.Ly, g.Lz};
  for (int d = 0; d < g.nd; ++d)
    if (ext[d] < 2 || (ext[d] & 1)) return fail(SPN_E_ARG, "every extent must be even and >= 2");
  g.N = (int64_t)g.Lx * g.Ly * g.Lz;
  if ((size_t)g.N > kScratchBytes)
    return fail(SPN_E_ARG, "lattice larger than the 16,777,216-site static scratch of this entry point");
  if ((uint64_t)sweep0 + (uint64_t)nsweeps > 0xffffffffull) return fail(SPN_E_ARG, "sweep counter would exceed 2^32");
  if (nsweeps == 0) return SPN_OK;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(SPN_E_CUDA, "cudaGetDevice failed");
  DeviceScratch sc;
  const char* why = "";
  int rc = scratch_for_device(dev, &sc, &why);
  if (rc) return fail(rc, why);

  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // the arrays keep the previous call's contents: clear what must start at zero
  if (cudaMemsetAsync(sc.err, 0, sizeof(int), st) != cudaSuccess) return fail(SPN_E_CUDA, "clearing the error word");
  if (cudaMemsetAsync(d_trace, 0, (size_t)nsweeps * 2 * sizeof(int64_t), st) != cudaSuccess)
    return fail(SPN_E_CUDA, "clearing the trace");

  const spn::DevThr T = spn::make_thresholds(beta);
  const spn::PhiloxKeys K = spn::philox_keys(seed);
  // the streaming sweep with the tallest band (3D: even, at most 32 rows, dividing
  // Ly) whose geometry fits one CTA; otherwise the generic sweep.  The streaming
  // sweep moves whole rows with bulk copies and 16-byte stores, so it needs a
  // 16-byte aligned lattice; a caller's pointer into the middle of a buffer that
  // is not takes the generic sweep (byte accesses), with the same results.
  bool stream = false;
  spn::StreamGeom geo{};
  const bool aligned16 = ((uintptr_t)d_spins & 15u) == 0;
  for (int ty = g.nd == 3 ? 32 : 1; aligned16 && ty >= 1 && !stream; ty -= (g.nd == 3 ? 2 : 1)) {
    if (g.nd == 3 && (ty < 2 || g.Ly % ty)) continue;
    if (!spn::stream_path_supported(g, ty)) continue;
    geo = spn::stream_geometry(g, ty, 0, 0);
    stream = spn::stream_geometry_ok(g, geo);
  }
  int8_t* bufs[2] = {d_spins, sc.lattice};
  int cur = 0;
  for (int64_t t = 0; t < nsweeps; ++t) {
    unsigned long long* acc = reinterpret_cast<unsigned long long*>(d_trace + 2 * t);
    cudaError_t e;
    if (stream) {
      e = spn::launch_sweep_stream(g, bufs[cur], bufs[cur ^ 1], geo, T, K, stream_id, sweep0 + (uint32_t)t, acc,
                                   sc.err, st);
      cur ^= 1;
    } else {
      e = spn::launch_sweep_generic(g, d_spins, T, K, stream_id, sweep0 + (uint32_t)t, acc, st);
    }
    if (e != cudaSuccess) return fail(SPN_E_CUDA, cudaGetErrorString(e));
  }
  if (cur == 1 && cudaMemcpyAsync(d_spins, sc.lattice, (size_t)g.N, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return fail(SPN_E_CUDA, "copying the result back");
  int err = 0;
  if (cudaMemcpyAsync(&err, sc.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(SPN_E_CUDA, "synchronising the stream");
  if (err) return fail(SPN_E_TIMEOUT, "a bounded device wait ran out");
  return SPN_OK;
}
