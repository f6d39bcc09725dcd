// C ABI of libspn (declared in include/spn.h): single-lattice handles.
//
// A handle owns its device buffers: two int8 spin buffers (ping-pong for the
// streaming kernel), optional per-site bond bytes, a per-sweep (dE, dM) delta
// array and an error word.  Sweeps are queued on the handle's stream; the host
// folds the per-sweep deltas into E, M and the trace when it is asked for them.
#include <cuda_runtime.h>

#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <utility>
#include <tuple>
#include <vector>

#include "spn.h"
#include "spn_testing.h"
#include "spn_internal.h"

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(SPN_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define SPN_CUDA(call, what)                         \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

int check_dims(int model, const int32_t* dims, spn::Lattice& g) {
  if (!dims) return fail(SPN_E_ARG, "dims is NULL");
  if (model != SPN_ISING2D && model != SPN_ISING3D && model != SPN_EA3D_PMJ)
    return fail(SPN_E_ARG, "unknown model %d", model);
  g.nd = model == SPN_ISING2D ? 2 : 3;
  g.Lx = dims[0];
  g.Ly = dims[1];
  g.Lz = g.nd == 3 ? dims[2] : 1;
  const int ext[3] = {g.Lx, g.Ly, g.Lz};
  for (int d = 0; d < g.nd; ++d)
    if (ext[d] < 2 || (ext[d] & 1)) return fail(SPN_E_ARG, "extent %d along axis %d must be even and >= 2", ext[d], d);
  g.N = (int64_t)g.Lx * g.Ly * g.Lz;
  if (g.N >= ((int64_t)1 << 35)) return fail(SPN_E_ARG, "lattice too large (%lld sites)", (long long)g.N);
  if (!spn::counter_range_ok(g.Lx, g.Ly, g.Lz))
    return fail(SPN_E_ARG, "lattice too large for the random-number counter (more than 2^29 row words)");
  return SPN_OK;
}

// Bit-packed [dir][ceil(N/64)] words -> per-site byte, bit d set iff J(n, d) = -1.
std::vector<uint8_t> unpack_site_bonds(const uint64_t* words, int nd, int64_t N) {
  const int64_t nw = (N + 63) / 64;
  std::vector<uint8_t> out((size_t)N, 0);
  for (int d = 0; d < nd; ++d)
    for (int64_t n = 0; n < N; ++n)
      if ((words[d * nw + (n >> 6)] >> (n & 63)) & 1) out[(size_t)n] |= (uint8_t)(1u << d);
  return out;
}

// The lattice as the streaming sweep sees it: rows padded to 64 bytes unless
// Lx is a multiple of 64.
spn::Lattice stream_lattice(const spn_ctx* h) {
  spn::Lattice g = h->g;
  g.pitch = (g.Lx % 64) ? (g.Lx + 63) / 64 * 64 : 0;
  return g;
}

// Device buffers the streaming path needs: the ping-pong partner, or the two
// padded staging lattices.
int ensure_stream_buffers(spn_ctx* h) {
  const spn::Lattice g = stream_lattice(h);
  if (g.pitch) {
    const size_t bytes = (size_t)g.pitch * (size_t)(g.N / g.Lx);
    for (int i = 0; i < 2; ++i)
      if (!h->staged[i]) {
        SPN_CUDA(cudaMalloc(&h->staged[i], bytes), "cudaMalloc(staged)");
        SPN_CUDA(cudaMemset(h->staged[i], 1, bytes), "cudaMemset(staged)");
      }
  } else if (!h->spins[1]) {
    SPN_CUDA(cudaMalloc(&h->spins[1], (size_t)g.N), "cudaMalloc(spins)");
  }
  return SPN_OK;
}

// Bit-packed path: both packed buffers, padding words zeroed once (the sweep
// writes data words only).
// Resident path (the batched kernel on one instance): the lattice lives in the
// shared memory of one CTA, or of a cluster of up to 8, for all sweeps of a call.
int resident_shape(const spn_ctx* h, int& cs, int& threads, size_t& smem) {
  const spn::Lattice& g = h->g;
  if (g.bonds || h->model == SPN_EA3D_PMJ) return 0;
  cs = spn::resident_cluster_size(g.nd, g.Lx, g.Ly, g.Lz);
  if (cs == 0) return 0;
  const int W = (g.Lx + 63) / 64;
  const int items = (int)((g.N / g.Lx + cs - 1) / cs) * W;
  threads = std::min(512, std::max(64, (items + 31) / 32 * 32));
  smem = spn::resident_smem(g.nd, g.Lx, g.Ly, g.Lz, cs);
  return 1;
}

int ensure_resident_buffers(spn_ctx* h) {
  if (h->d_res) return SPN_OK;
  SPN_CUDA(cudaMalloc(&h->d_res, sizeof(spn::ResInst)), "cudaMalloc(resident)");
  SPN_CUDA(cudaMalloc(&h->d_resq, 2 * sizeof(int)), "cudaMalloc(resident)");
  SPN_CUDA(cudaMemsetAsync(h->d_resq, 0, 2 * sizeof(int), h->st), "cudaMemsetAsync");
  return SPN_OK;
}

int ensure_packed_buffers(spn_ctx* h) {
  const size_t bytes = (size_t)spn::packed_row_words(h->g.Lx) * 4 * (size_t)(h->g.N / h->g.Lx);
  for (int i = 0; i < 2; ++i)
    if (!h->packed[i]) {
      SPN_CUDA(cudaMalloc(&h->packed[i], bytes), "cudaMalloc(packed)");
      SPN_CUDA(cudaMemsetAsync(h->packed[i], 0, bytes, h->st), "cudaMemsetAsync(packed)");
    }
  return SPN_OK;
}

// Make the int8 buffer current again after packed sweeps.
int unpack_if_live(spn_ctx* h) {
  if (!h->packed_live) return SPN_OK;
  SPN_CUDA(spn::launch_unpack(h->g, h->packed[h->pcur], h->spins[h->cur], h->st), "unpack");
  h->packed_live = false;
  return SPN_OK;
}

void pick_default_path(spn_ctx* h) {
  const spn::Lattice g = stream_lattice(h);
  h->step_slices = 0;
  h->seg = 0;
  bool fits = false;
  if (g.nd == 2) {
    h->tile_y = 1;
    fits = spn::stream_path_supported(g, 1) && spn::stream_geometry_ok(g, spn::stream_geometry(g, 1, 0, 0));
  } else {
    // the tallest even band of at most 32 rows that divides Ly and fits one CTA
    // (else the tallest dividing one, for explicit tilings)
    h->tile_y = 0;
    for (int ty = 32; ty >= 2 && !fits; ty -= 2) {
      if (g.Ly % ty) continue;
      if (!h->tile_y) h->tile_y = ty;
      if (spn::stream_path_supported(g, ty) && spn::stream_geometry_ok(g, spn::stream_geometry(g, ty, 0, 0))) {
        h->tile_y = ty;
        fits = true;
      }
    }
  }
  // Small lattices run all sweeps of a call in one resident launch when their
  // bits fit one CTA (1.8-7.6 us per sweep up to 2D L = 256 and 3D L = 32 on
  // GB300, against 8-16 us for one streaming launch); larger ones stream.
  int cs = 0, threads = 0;
  size_t smem = 0;
  if (g.N <= (1 << 16) && resident_shape(h, cs, threads, smem) && cs == 1)
    h->path = spn::kPathResident;
  else
    h->path = fits && g.N >= (1 << 16) ? spn::kPathStream : spn::kPathGeneric;
}

int ensure_acc(spn_ctx* h, int64_t n) {
  // deltas for sweeps [folded, sweeps + n)
  const int64_t need = (int64_t)(h->sweeps - h->folded) + n;
  if (need <= h->acc_cap) return SPN_OK;
  int64_t cap = h->acc_cap ? h->acc_cap : 1024;
  while (cap < need) cap *= 2;
  unsigned long long* p = nullptr;
  SPN_CUDA(cudaMalloc(&p, (size_t)cap * 2 * sizeof(unsigned long long)), "cudaMalloc(trace)");
  SPN_CUDA(cudaMemsetAsync(p, 0, (size_t)cap * 2 * sizeof(unsigned long long), h->st), "cudaMemsetAsync");
  const int64_t live = (int64_t)(h->sweeps - h->folded);
  if (live > 0 && h->d_acc)
    SPN_CUDA(cudaMemcpyAsync(p, h->d_acc, (size_t)live * 2 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice,
                             h->st),
             "cudaMemcpyAsync(trace)");
  if (h->d_acc) {
    cudaStreamSynchronize(h->st);
    cudaFree(h->d_acc);
  }
  h->d_acc = p;
  h->acc_cap = cap;
  return SPN_OK;
}

// Fold the device deltas of all sweeps so far into E, M and the host trace.
int fold(spn_ctx* h) {
  SPN_CUDA(cudaStreamSynchronize(h->st), "cudaStreamSynchronize");
  int err = 0;
  SPN_CUDA(cudaMemcpy(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost), "cudaMemcpy(err)");
  if (err) return fail(SPN_E_TIMEOUT, "a bounded device wait ran out in a sweep kernel (code %d)", err);
  const int64_t live = (int64_t)(h->sweeps - h->folded);
  if (live <= 0) return SPN_OK;
  std::vector<unsigned long long> d((size_t)live * 2);
  SPN_CUDA(cudaMemcpy(d.data(), h->d_acc, d.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost),
           "cudaMemcpy(trace)");
  for (int64_t i = 0; i < live; ++i) {
    h->E += (int64_t)d[2 * i];
    h->M += (int64_t)d[2 * i + 1];
    h->traceE.push_back(h->E);
    h->traceM.push_back(h->M);
  }
  h->folded = h->sweeps;
  SPN_CUDA(cudaMemsetAsync(h->d_acc, 0, (size_t)h->acc_cap * 2 * sizeof(unsigned long long), h->st),
           "cudaMemsetAsync(trace)");
  return SPN_OK;
}

int recompute(spn_ctx* h, int64_t* E, int64_t* M) {
  if (int rc = unpack_if_live(h)) return rc;
  SPN_CUDA(cudaMemsetAsync(h->d_bad, 0, sizeof(int), h->st), "cudaMemsetAsync");
  SPN_CUDA(spn::launch_observables(h->g, h->spins[h->cur], h->d_obs, h->d_bad, h->st), "observables");
  unsigned long long r[3];
  SPN_CUDA(cudaMemcpyAsync(r, h->d_obs, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->st),
           "cudaMemcpyAsync(obs)");
  int bad = 0;
  SPN_CUDA(cudaMemcpyAsync(&bad, h->d_bad, sizeof(int), cudaMemcpyDeviceToHost, h->st), "cudaMemcpyAsync(bad)");
  SPN_CUDA(cudaStreamSynchronize(h->st), "cudaStreamSynchronize");
  if (bad) return fail(SPN_E_ARG, "spin values other than +-1 in the lattice");
  *E = (int64_t)r[0];
  *M = (int64_t)r[1];
  return SPN_OK;
}

void destroy(spn_ctx* h) {
  if (!h) return;
  if (h->st) cudaStreamSynchronize(h->st);
  spn_ea_free(h->ea);
  spn::heis_free(h->heis);
  // only what was allocated: a batch handle owns none of these, and its frees
  // must not wait for the device
  for (void* p : {(void*)h->spins[0], (void*)h->spins[1], (void*)h->staged[0], (void*)h->staged[1],
                  (void*)h->packed[0], (void*)h->packed[1], (void*)h->d_bonds, (void*)h->d_acc, (void*)h->d_err,
                  (void*)h->d_bad, (void*)h->d_obs, (void*)h->d_res, (void*)h->d_resq})
    if (p) cudaFree(p);
  delete h;
}

}  // namespace

void spn::set_last_error(const char* msg) { g_last_error = msg; }

extern "C" {

const char* spn_last_error(void) { return g_last_error.c_str(); }

const char* spn_version(void) { return "libspn 0.1 (sm_103a)"; }

int spn_create_ex(spn_handle* out, int model, const int32_t* dims, const void* couplings, uint64_t seed,
                  uint32_t stream, int init) {
  if (!out) return fail(SPN_E_ARG, "out is NULL");
  *out = nullptr;
  if (spn::is_heis_model(model)) {
    if (!dims) return fail(SPN_E_ARG, "dims is NULL");
    if (couplings) return fail(SPN_E_ARG, "Heisenberg models take no couplings");
    if (init != SPN_INIT_HOT && init != SPN_INIT_COLD) return fail(SPN_E_ARG, "unknown init %d", init);
    spn_ctx* h = new (std::nothrow) spn_ctx;
    if (!h) return fail(SPN_E_NOMEM, "host allocation failed");
    h->model = model;
    h->seed = seed;
    h->stream_id = stream;
    const int rc = spn::heis_create(h, dims, init);
    if (rc) {
      const std::string msg = spn_last_error();
      destroy(h);
      return fail(rc, "%s", msg.c_str());
    }
    *out = h;
    return SPN_OK;
  }
  spn::Lattice g;
  int rc = check_dims(model, dims, g);
  if (rc) return rc;
  if (model == SPN_EA3D_PMJ && !couplings) return fail(SPN_E_ARG, "SPN_EA3D_PMJ needs couplings");
  if (model != SPN_EA3D_PMJ && couplings) return fail(SPN_E_ARG, "Ising models take no couplings");
  if (init != SPN_INIT_HOT && init != SPN_INIT_COLD) return fail(SPN_E_ARG, "unknown init %d", init);
  spn_ctx* h = new (std::nothrow) spn_ctx;
  if (!h) return fail(SPN_E_NOMEM, "host allocation failed");
  h->model = model;
  h->g = g;
  h->seed = seed;
  h->stream_id = stream;
  auto bail = [&](int code) {
    destroy(h);
    return code;
  };
  cudaError_t e;
  if ((e = cudaMalloc(&h->spins[0], (size_t)g.N)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc(spins)"));
  if ((e = cudaMalloc(&h->d_err, sizeof(int))) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc(err)"));
  if ((e = cudaMalloc(&h->d_bad, sizeof(int))) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc(bad)"));
  if ((e = cudaMalloc(&h->d_obs, 2 * sizeof(unsigned long long))) != cudaSuccess)
    return bail(cuda_fail(e, "cudaMalloc(obs)"));
  if ((e = cudaMemsetAsync(h->d_err, 0, sizeof(int), h->st)) != cudaSuccess) return bail(cuda_fail(e, "memset"));
  if (couplings) {
    std::vector<uint8_t> sb = unpack_site_bonds(static_cast<const uint64_t*>(couplings), g.nd, g.N);
    if ((e = cudaMalloc(&h->d_bonds, (size_t)g.N)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc(bonds)"));
    if ((e = cudaMemcpy(h->d_bonds, sb.data(), (size_t)g.N, cudaMemcpyHostToDevice)) != cudaSuccess)
      return bail(cuda_fail(e, "cudaMemcpy(bonds)"));
    h->g.bonds = h->d_bonds;
  }
  pick_default_path(h);
  if (h->path == spn::kPathStream)
    if ((rc = ensure_stream_buffers(h))) return bail(rc);
  if (h->path == spn::kPathResident)
    if ((rc = ensure_resident_buffers(h))) return bail(rc);
  if (init == SPN_INIT_HOT) {
    if ((e = spn::launch_init_hot(h->g, h->spins[0], seed, stream, h->st)) != cudaSuccess)
      return bail(cuda_fail(e, "init"));
  } else {
    if ((e = cudaMemsetAsync(h->spins[0], 1, (size_t)g.N, h->st)) != cudaSuccess) return bail(cuda_fail(e, "init"));
  }
  if ((rc = ensure_acc(h, 1024))) return bail(rc);
  int64_t E, M;
  if ((rc = recompute(h, &E, &M))) return bail(rc);
  h->E = E;
  h->M = M;
  *out = h;
  return SPN_OK;
}

int spn_create(spn_handle* out, int model, const int32_t* dims, const void* couplings, uint64_t seed) {
  return spn_create_ex(out, model, dims, couplings, seed, 0, SPN_INIT_HOT);
}

int spn_sweep(spn_handle h, double beta, int64_t nsweeps) {
  if (!h) return fail(SPN_E_ARG, "handle is NULL");
  if (h->ea) return fail(SPN_E_STATE, "a batch handle takes the spn_batch_* calls");
  if (!(beta >= 0.0)) return fail(SPN_E_ARG, "beta must be >= 0 (got %g)", beta);
  if (nsweeps < 0) return fail(SPN_E_ARG, "nsweeps must be >= 0");
  if (nsweeps == 0) return SPN_OK;
  if (h->sweeps + (uint64_t)nsweeps > 0xffffffffull) return fail(SPN_E_ARG, "sweep counter would exceed 2^32");
  if (h->heis) {
    if (!(beta < 3.4e38)) return fail(SPN_E_ARG, "Heisenberg beta must be finite in binary32");
    return spn::heis_sweep(h, beta, nsweeps);
  }
  int rc = ensure_acc(h, nsweeps);
  if (rc) return rc;
  const spn::DevThr T = spn::make_thresholds(beta);
  const spn::PhiloxKeys K = spn::philox_keys(h->seed);
  spn::StreamGeom geo{};
  const spn::Lattice gs = stream_lattice(h);
  const bool staged = h->path == spn::kPathStream && gs.pitch != 0;
  const size_t nrow = (size_t)(h->g.N / h->g.Lx);
  int sc = 0;  // current staged lattice
  if (h->path == spn::kPathPacked) {
    geo = spn::stream_geometry(h->g, h->tile_y, h->step_slices, h->seg, true);
    if (!spn::stream_geometry_ok(h->g, geo)) return fail(SPN_E_STATE, "packed geometry does not fit one CTA");
    if ((rc = ensure_packed_buffers(h))) return rc;
    if (!h->packed_live) {
      SPN_CUDA(spn::launch_pack(h->g, h->spins[h->cur], h->packed[h->pcur], h->st), "pack");
      h->packed_live = true;
    }
  } else if ((rc = unpack_if_live(h))) {
    return rc;
  }
  if (h->path == spn::kPathResident) {
    int cs = 0, threads = 0;
    size_t smem = 0;
    if (!resident_shape(h, cs, threads, smem)) return fail(SPN_E_STATE, "the lattice does not fit the resident kernel");
    if ((rc = ensure_resident_buffers(h))) return rc;
    // every sweep of the call in one launch (chunks keep the count an int)
    for (int64_t t0 = 0; t0 < nsweeps; t0 += (int64_t)1 << 30) {
      const int n = (int)std::min<int64_t>(nsweeps - t0, (int64_t)1 << 30);
      spn::ResInst r{};
      r.spins = h->spins[h->cur];
      r.trace = h->d_acc + 2 * (int64_t)(h->sweeps + (uint64_t)t0 - h->folded);
      r.em0 = nullptr;
      r.seed = h->seed;
      r.stream = h->stream_id;
      r.sweep0 = (uint32_t)(h->sweeps + (uint64_t)t0);
      r.nsweeps = n;
      r.init_hot = 0;
      r.Lx = h->g.Lx;
      r.Ly = h->g.Ly;
      r.Lz = h->g.Lz;
      r.T = T;
      spn::ResArgs a{};
      a.inst = h->d_res;
      a.ninst = 1;
      a.order = h->d_resq;
      a.counter = h->d_resq + 1;
      a.err = h->d_err;
      a.no_always = spn::no_always_class(T);
      // r is pageable: the copy is staged before the call returns
      cudaError_t e = cudaMemcpyAsync(h->d_res, &r, sizeof r, cudaMemcpyHostToDevice, h->st);
      if (e == cudaSuccess) e = cudaMemsetAsync(h->d_resq + 1, 0, sizeof(int), h->st);
      if (e == cudaSuccess) e = spn::launch_resident(a, h->g.nd, cs, threads, cs, smem, h->st);
      if (e != cudaSuccess) {
        h->sweeps += (uint64_t)t0;
        return cuda_fail(e, "resident launch");
      }
    }
    h->sweeps += (uint64_t)nsweeps;
    return SPN_OK;
  }
  if (h->path == spn::kPathStream) {
    geo = spn::stream_geometry(gs, h->tile_y, h->step_slices, h->seg);
    if (!spn::stream_geometry_ok(gs, geo)) return fail(SPN_E_STATE, "streaming geometry does not fit one CTA");
    if ((rc = ensure_stream_buffers(h))) return rc;
    if (staged)
      SPN_CUDA(cudaMemcpy2DAsync(h->staged[0], (size_t)gs.pitch, h->spins[h->cur], (size_t)gs.Lx, (size_t)gs.Lx, nrow,
                                 cudaMemcpyDeviceToDevice, h->st),
               "staging the lattice");
  }
  for (int64_t t = 0; t < nsweeps; ++t) {
    const uint32_t sweep = (uint32_t)(h->sweeps + t);
    unsigned long long* acc = h->d_acc + 2 * (int64_t)(sweep - h->folded);
    cudaError_t e;
    if (h->path == spn::kPathPacked) {
      e = spn::launch_sweep_stream(h->g, h->packed[h->pcur], h->packed[h->pcur ^ 1], geo, T, K, h->stream_id, sweep,
                                   acc, h->d_err, h->st, std::exchange(h->expire_polls, 0u));
      if (e == cudaSuccess) h->pcur ^= 1;
    } else if (staged) {
      e = spn::launch_sweep_stream(gs, h->staged[sc], h->staged[sc ^ 1], geo, T, K, h->stream_id, sweep, acc,
                                   h->d_err, h->st, std::exchange(h->expire_polls, 0u));
      if (e == cudaSuccess) sc ^= 1;
    } else if (h->path == spn::kPathStream) {
      e = spn::launch_sweep_stream(h->g, h->spins[h->cur], h->spins[h->cur ^ 1], geo, T, K, h->stream_id, sweep,
                                   acc, h->d_err, h->st, std::exchange(h->expire_polls, 0u));
      if (e == cudaSuccess) h->cur ^= 1;
    } else {
      e = spn::launch_sweep_generic(h->g, h->spins[h->cur], T, K, h->stream_id, sweep, acc, h->st);
    }
    if (e != cudaSuccess) {
      h->sweeps += (uint64_t)t;
      if (staged && t > 0)
        cudaMemcpy2DAsync(h->spins[h->cur], (size_t)gs.Lx, h->staged[sc], (size_t)gs.pitch, (size_t)gs.Lx, nrow,
                          cudaMemcpyDeviceToDevice, h->st);
      return cuda_fail(e, "sweep launch");
    }
  }
  if (staged)
    SPN_CUDA(cudaMemcpy2DAsync(h->spins[h->cur], (size_t)gs.Lx, h->staged[sc], (size_t)gs.pitch, (size_t)gs.Lx, nrow,
                               cudaMemcpyDeviceToDevice, h->st),
             "unstaging the lattice");
  h->sweeps += (uint64_t)nsweeps;
  return SPN_OK;
}

int spn_sweep_dc(spn_handle h, double beta, int64_t nsweeps, const int32_t* tile, int32_t hits) {
  if (!h || !tile) return fail(SPN_E_ARG, "NULL argument");
  if (h->ea || h->heis || h->model == SPN_EA3D_PMJ)
    return fail(SPN_E_STATE, "the double-checkerboard sweep is for Ising lattices");
  if (!(beta >= 0.0)) return fail(SPN_E_ARG, "beta must be >= 0 (got %g)", beta);
  if (nsweeps < 0 || hits < 1) return fail(SPN_E_ARG, "nsweeps must be >= 0 and hits >= 1");
  if (nsweeps == 0) return SPN_OK;
  const int tz = h->g.nd == 3 ? tile[2] : 1;
  if (!spn::dc_supported(h->g, tile[0], tile[1], tz))
    return fail(SPN_E_ARG, "tiles must have Tx a multiple of 64 and an even number of tiles along every axis");
  if ((h->sweeps + (uint64_t)nsweeps) * (uint64_t)hits > 0xffffffffull)
    return fail(SPN_E_ARG, "sweep counter times hits would exceed 2^32");
  int rc = ensure_acc(h, nsweeps);
  if (rc) return rc;
  if ((rc = unpack_if_live(h))) return rc;
  const spn::DevThr T = spn::make_thresholds(beta);
  const spn::PhiloxKeys K = spn::philox_keys(h->seed);
  // one hit on rows of at least 2048 sites in whole words: the band-parallel
  // wavefront form (one read and one write of every spin a sweep, ping-pong
  // buffers); otherwise a CTA per tile, in place, one launch per tile parity
  if (spn::dcwave_supported(h->g, tile[0], tile[1], hits)) {
    if ((rc = ensure_stream_buffers(h))) return rc;
    const int nseg = spn::dcwave_default_segments(h->g, hits);
    for (int64_t t = 0; t < nsweeps; ++t) {
      const uint32_t sweep = (uint32_t)(h->sweeps + t);
      unsigned long long* acc = h->d_acc + 2 * (int64_t)(sweep - h->folded);
      const cudaError_t e = spn::launch_sweep_dcwave(h->g, h->spins[h->cur], h->spins[h->cur ^ 1], tile[0], tile[1],
                                                     hits, nseg, T, K, h->stream_id, sweep, acc, h->d_err, h->st,
                                                     std::exchange(h->expire_polls, 0u));
      if (e != cudaSuccess) {
        h->sweeps += (uint64_t)t;
        return cuda_fail(e, "double-checkerboard launch");
      }
      h->cur ^= 1;
    }
    h->sweeps += (uint64_t)nsweeps;
    return SPN_OK;
  }
  for (int64_t t = 0; t < nsweeps; ++t) {
    const uint32_t sweep = (uint32_t)(h->sweeps + t);
    unsigned long long* acc = h->d_acc + 2 * (int64_t)(sweep - h->folded);
    const cudaError_t e = spn::launch_sweep_dc(h->g, h->spins[h->cur], tile[0], tile[1], tz, hits, T, K,
                                               h->stream_id, sweep, acc, h->st);
    if (e != cudaSuccess) {
      h->sweeps += (uint64_t)t;
      return cuda_fail(e, "double-checkerboard launch");
    }
  }
  h->sweeps += (uint64_t)nsweeps;
  return SPN_OK;
}

int spn_test_expire_next_waits(spn_handle h, uint32_t polls) {
  if (!h || h->ea || h->heis) return fail(SPN_E_STATE, "an Ising lattice handle is required");
  h->expire_polls = polls ? polls : 1;
  return SPN_OK;
}

int spn_observables(spn_handle h, int64_t* E, int64_t* M) {
  if (!h || !E || !M) return fail(SPN_E_ARG, "NULL argument");
  if (h->ea) return fail(SPN_E_STATE, "a batch handle takes the spn_batch_* calls");
  if (h->heis) return fail(SPN_E_STATE, "a Heisenberg handle takes spn_heis_observables");
  int rc = fold(h);
  if (rc) return rc;
  *E = h->E;
  *M = h->M;
  return SPN_OK;
}

int spn_recompute(spn_handle h, int64_t* E, int64_t* M) {
  if (!h || !E || !M) return fail(SPN_E_ARG, "NULL argument");
  if (h->ea) return fail(SPN_E_STATE, "a batch handle takes the spn_batch_* calls");
  if (h->heis) return fail(SPN_E_STATE, "a Heisenberg handle takes spn_heis_recompute");
  return recompute(h, E, M);
}

int spn_trace(spn_handle h, int64_t* E, int64_t* M, int64_t cap, int64_t* n) {
  if (!h || !n || cap < 0 || (cap > 0 && (!E || !M))) return fail(SPN_E_ARG, "bad trace arguments");
  if (h->ea) return fail(SPN_E_STATE, "a batch handle takes the spn_batch_* calls");
  if (h->heis) return fail(SPN_E_STATE, "a Heisenberg handle takes spn_heis_trace");
  int rc = fold(h);
  if (rc) return rc;
  const int64_t total = (int64_t)h->traceE.size();
  const int64_t k = cap < total ? cap : total;
  if (k > 0) {
    std::memcpy(E, h->traceE.data(), (size_t)k * sizeof(int64_t));
    std::memcpy(M, h->traceM.data(), (size_t)k * sizeof(int64_t));
  }
  *n = total;
  return SPN_OK;
}

int spn_get_spins(spn_handle h, int8_t* host_out, size_t bytes) {
  if (!h || !host_out) return fail(SPN_E_ARG, "NULL argument");
  if (h->ea) return fail(SPN_E_STATE, "a batch handle takes the spn_batch_* calls");
  if (h->heis) return fail(SPN_E_STATE, "a Heisenberg handle takes spn_heis_get_spins");
  if (bytes != (size_t)h->g.N) return fail(SPN_E_ARG, "bytes must be N = %lld", (long long)h->g.N);
  if (int rc = unpack_if_live(h)) return rc;
  SPN_CUDA(cudaMemcpyAsync(host_out, h->spins[h->cur], bytes, cudaMemcpyDeviceToHost, h->st), "cudaMemcpyAsync");
  SPN_CUDA(cudaStreamSynchronize(h->st), "cudaStreamSynchronize");
  return SPN_OK;
}

int spn_set_spins(spn_handle h, const int8_t* host_in, size_t bytes) {
  if (!h || !host_in) return fail(SPN_E_ARG, "NULL argument");
  if (h->ea) return fail(SPN_E_STATE, "a batch handle takes the spn_batch_* calls");
  if (h->heis) return fail(SPN_E_STATE, "a Heisenberg handle takes spn_heis_set_spins");
  if (bytes != (size_t)h->g.N) return fail(SPN_E_ARG, "bytes must be N = %lld", (long long)h->g.N);
  int rc = fold(h);
  if (rc) return rc;
  h->packed_live = false;  // the new spins replace the packed lattice
  SPN_CUDA(cudaMemcpyAsync(h->spins[h->cur], host_in, bytes, cudaMemcpyHostToDevice, h->st), "cudaMemcpyAsync");
  int64_t E, M;
  if ((rc = recompute(h, &E, &M))) return rc;
  h->E = E;
  h->M = M;
  return SPN_OK;
}

int spn_reinit(spn_handle h, uint64_t seed, uint32_t stream, int init) {
  if (!h) return fail(SPN_E_ARG, "handle is NULL");
  if (h->ea) return fail(SPN_E_STATE, "a batch handle takes the spn_batch_* calls");
  if (init != SPN_INIT_HOT && init != SPN_INIT_COLD) return fail(SPN_E_ARG, "unknown init %d", init);
  if (h->heis) {
    h->seed = seed;
    h->stream_id = stream;
    const int rc = spn::heis_reinit(h, init);
    h->sweeps = 0;
    return rc;
  }
  int rc = fold(h);
  if (rc) return rc;
  h->seed = seed;
  h->stream_id = stream;
  h->sweeps = 0;
  h->folded = 0;
  h->traceE.clear();
  h->traceM.clear();
  h->packed_live = false;
  if (init == SPN_INIT_HOT)
    SPN_CUDA(spn::launch_init_hot(h->g, h->spins[h->cur], seed, stream, h->st), "init");
  else
    SPN_CUDA(cudaMemsetAsync(h->spins[h->cur], 1, (size_t)h->g.N, h->st), "init");
  int64_t E, M;
  if ((rc = recompute(h, &E, &M))) return rc;
  h->E = E;
  h->M = M;
  return SPN_OK;
}

int spn_launch_count(uint64_t* count) {
  if (!count) return fail(SPN_E_ARG, "NULL argument");
  *count = spn::launch_count();
  return SPN_OK;
}

int spn_sweep_count(spn_handle h, uint64_t* count) {
  if (!h || !count) return fail(SPN_E_ARG, "NULL argument");
  *count = h->sweeps;
  return SPN_OK;
}

int spn_set_stream(spn_handle h, void* cuda_stream) {
  if (!h) return fail(SPN_E_ARG, "handle is NULL");
  SPN_CUDA(cudaStreamSynchronize(h->st), "cudaStreamSynchronize");
  h->st = static_cast<cudaStream_t>(cuda_stream);
  return SPN_OK;
}

int spn_sync(spn_handle h) {
  if (!h) return fail(SPN_E_ARG, "handle is NULL");
  SPN_CUDA(cudaStreamSynchronize(h->st), "cudaStreamSynchronize");
  return SPN_OK;
}

int spn_destroy(spn_handle h) {
  if (!h) return fail(SPN_E_ARG, "handle is NULL");
  destroy(h);
  return SPN_OK;
}

int spn_set_tiling(spn_handle h, int32_t tile_y, int32_t step_slices, int32_t seg) {
  if (!h) return fail(SPN_E_ARG, "handle is NULL");
  if (h->ea || h->heis) return fail(SPN_E_STATE, "tiling applies to Ising lattices");
  const int ty = h->g.nd == 3 ? tile_y : 1;
  if (step_slices < 0 || seg < 0) return fail(SPN_E_ARG, "negative tiling parameter");
  const bool packed = h->path == spn::kPathPacked;
  const spn::Lattice gs = packed ? h->g : stream_lattice(h);
  if (!spn::stream_path_supported(gs, ty, packed))
    return fail(SPN_E_ARG, "band of %d rows does not divide the lattice (or the lattice has bonds)", tile_y);
  const spn::StreamGeom geo = spn::stream_geometry(gs, ty, step_slices, seg, packed);
  if (!spn::stream_geometry_ok(gs, geo)) return fail(SPN_E_ARG, "tiling too large for one CTA");
  h->tile_y = ty;
  h->step_slices = step_slices;
  h->seg = seg;
  return SPN_OK;
}

int spn_autotune(spn_handle h, double beta, int32_t trial_sweeps, int32_t* chosen) {
  if (!h) return fail(SPN_E_ARG, "handle is NULL");
  if (h->ea || h->heis) return fail(SPN_E_STATE, "the autotuner tunes the streaming sweep of Ising lattices");
  if (h->path != spn::kPathStream && h->path != spn::kPathPacked)
    return fail(SPN_E_STATE, "the handle's path is not a streaming one");
  if (!(beta >= 0.0) || trial_sweeps < 1) return fail(SPN_E_ARG, "bad arguments");
  const bool packed = h->path == spn::kPathPacked;
  const spn::Lattice g = packed ? h->g : stream_lattice(h);
  static std::mutex mu;
  static std::map<std::tuple<int, int, int, int, int, int>, std::array<int, 3>> cache;
  const auto key = std::make_tuple(g.nd, g.Lx, g.Ly, g.Lz, (int)packed, spn::device_sm_count());
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      h->tile_y = it->second[0];
      h->step_slices = it->second[1];
      h->seg = it->second[2];
      if (chosen) std::memcpy(chosen, it->second.data(), 3 * sizeof(int32_t));
      return SPN_OK;
    }
  }
  SPN_CUDA(cudaStreamSynchronize(h->st), "cudaStreamSynchronize");
  // scratch ping-pong lattices from a hot start: the handle's own state is untouched
  const size_t rows = (size_t)(g.N / g.Lx);
  const size_t bytes = packed ? (size_t)spn::packed_row_words(g.Lx) * 4 * rows : (size_t)(g.pitch ? g.pitch : g.Lx) * rows;
  void* buf[2] = {nullptr, nullptr};
  int8_t* dense = nullptr;
  unsigned long long* acc = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = SPN_OK;
  auto cleanup = [&] {
    cudaFree(buf[0]);
    cudaFree(buf[1]);
    cudaFree(dense);
    cudaFree(acc);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  if (cudaMalloc(&buf[0], bytes) != cudaSuccess || cudaMalloc(&buf[1], bytes) != cudaSuccess ||
      cudaMalloc(&dense, (size_t)g.N) != cudaSuccess || cudaMalloc(&acc, 16) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cleanup();
    return fail(SPN_E_NOMEM, "autotune scratch");
  }
  cudaError_t e = spn::launch_init_hot(h->g, dense, h->seed, h->stream_id, h->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(buf[0], packed ? 0 : 1, bytes, h->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(buf[1], packed ? 0 : 1, bytes, h->st);
  if (e == cudaSuccess)
    e = packed ? spn::launch_pack(h->g, dense, static_cast<uint32_t*>(buf[0]), h->st)
               : cudaMemcpy2DAsync(buf[0], g.pitch ? g.pitch : g.Lx, dense, g.Lx, g.Lx, rows, cudaMemcpyDeviceToDevice,
                                   h->st);
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "autotune set-up");
  }
  const spn::DevThr T = spn::make_thresholds(beta);
  const spn::PhiloxKeys K = spn::philox_keys(h->seed);
  // candidates: bands (3D), slices per step, segments per band
  std::vector<int> tys;
  if (g.nd == 3) {
    for (int ty = 32; ty >= 2; ty -= 2)
      if (g.Ly % ty == 0 && spn::stream_path_supported(g, ty, packed)) tys.push_back(ty);
  } else {
    tys.push_back(1);
  }
  const int sms = spn::device_sm_count();
  double best = -1.0;
  std::array<int, 3> pick = {h->tile_y, h->step_slices, h->seg};
  for (int ty : tys) {
    const int S = g.nd == 3 ? g.Lz : g.Ly, tiles = g.nd == 3 ? g.Ly / ty : 1;
    for (int R : {0, 1, 2, 4}) {
      for (int per_sm : {0, 2, 4, 6, 8}) {  // 0: the default segment count
        const int seg = per_sm ? std::max(1, std::min(S, (per_sm * sms + tiles - 1) / tiles)) : 0;
        const spn::StreamGeom geo = spn::stream_geometry(g, ty, R, seg, packed);
        if (!spn::stream_geometry_ok(g, geo)) continue;
        float ms = 0.0f;
        int cur = 0;
        for (int rep = 0; rep < 2 && rc == SPN_OK; ++rep) {  // the first pass warms up
          if (cudaEventRecord(e0, h->st) != cudaSuccess) rc = SPN_E_CUDA;
          for (int t = 0; t < trial_sweeps && rc == SPN_OK; ++t, cur ^= 1)
            if (spn::launch_sweep_stream(g, buf[cur], buf[cur ^ 1], geo, T, K, h->stream_id, (uint32_t)t, acc, h->d_err,
                                         h->st) != cudaSuccess)
              rc = SPN_E_CUDA;
          if (rc == SPN_OK && (cudaEventRecord(e1, h->st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                               cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            rc = SPN_E_CUDA;
        }
        if (rc != SPN_OK) break;
        const double rate = (double)g.N * trial_sweeps / ((double)ms * 1e6);
        // the first candidate (tallest band, default slices and segments) is the
        // default tiling; another must beat the best by more than 1% (trial
        // noise) to be taken
        if (best < 0.0 || rate > 1.01 * best) {
          best = rate;
          pick = {ty, R, seg};
        }
      }
    }
  }
  cleanup();
  if (rc != SPN_OK) return fail(SPN_E_CUDA, "autotune trial");
  h->tile_y = pick[0];
  h->step_slices = pick[1];
  h->seg = pick[2];
  {
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = pick;
  }
  if (chosen) std::memcpy(chosen, pick.data(), 3 * sizeof(int32_t));
  return SPN_OK;
}

int spn_get_path(spn_handle h, int32_t* path) {
  if (!h || !path) return fail(SPN_E_ARG, "NULL argument");
  *path = h->path;
  return SPN_OK;
}

int spn_set_path(spn_handle h, int32_t path) {
  if (!h) return fail(SPN_E_ARG, "handle is NULL");
  if (h->ea || h->heis) return fail(SPN_E_STATE, "kernel paths apply to Ising lattices");
  if (path == spn::kPathStream) {
    if (!spn::stream_path_supported(stream_lattice(h), h->tile_y))
      return fail(SPN_E_ARG, "streaming path needs a dividing band and no bonds");
    const int rc = ensure_stream_buffers(h);
    if (rc) return rc;
  } else if (path == spn::kPathPacked) {
    if (!spn::stream_path_supported(h->g, h->tile_y, true))
      return fail(SPN_E_ARG, "bit-packed path needs a dividing band and no bonds");
    const spn::StreamGeom geo = spn::stream_geometry(h->g, h->tile_y, h->step_slices, h->seg, true);
    if (!spn::stream_geometry_ok(h->g, geo)) return fail(SPN_E_ARG, "bit-packed tiling too large for one CTA");
    const int rc = ensure_packed_buffers(h);
    if (rc) return rc;
  } else if (path == spn::kPathResident) {
    int cs = 0, threads = 0;
    size_t smem = 0;
    if (!resident_shape(h, cs, threads, smem))
      return fail(SPN_E_ARG, "resident path needs an Ising lattice whose bits fit a cluster of 8 x 200 KB");
    const int rc = ensure_resident_buffers(h);
    if (rc) return rc;
  } else if (path != spn::kPathGeneric) {
    return fail(SPN_E_ARG, "unknown path %d", path);
  }
  h->path = path;
  return SPN_OK;
}

}  // extern "C"
