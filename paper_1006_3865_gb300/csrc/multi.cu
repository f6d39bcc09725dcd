// Batched runs of many independent lattices (the spn_multi_* ABI).
//
// A run starts every job from its Philox hot start and does its sweeps.
// SPN_RUN_BATCHED groups the jobs by model and extents; each group is one
// persistent, shared-memory-resident launch (batched.cu) on its own stream, the
// groups run concurrently, and the whole run -- zeroing, launches, fork and
// join -- is captured once into a CUDA graph that later runs replay.
// SPN_RUN_LOOP is the plain per-instance launch loop: for each job in turn,
// hot start, E/M and one launch per sweep (streaming or generic kernel).  Both
// produce bit-identical lattices and traces.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <tuple>
#include <vector>

#include "spn.h"
#include "spn_internal.h"

namespace {

int mfail(int code, const char* msg) {
  spn::set_last_error(msg);
  return code;
}

// Launch shapes chosen by the autotuner, per lattice shape and device (SM
// count), for the process.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, std::pair<int, int>> g_tuned;  // -> (cluster size, threads)

struct Group {
  int nd, Lx, Ly, Lz, cs, threads, ctas;
  size_t smem = 0;
  double tuned_rate = 0.0;  // attempts/ns of the autotuner's trial (0: not tuned)
  bool no_always = true;    // no instance has an always-accepted class with dE > 0
  std::vector<int> jobs;  // job indices, longest first
  spn::ResInst* d_inst = nullptr;
  int* d_order = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
};

}  // namespace

struct spn_multi_ctx {
  std::vector<spn_job> jobs;
  std::vector<int64_t> N;
  std::vector<size_t> spin_off, trace_off;  // offsets into the pools
  int8_t* d_spins = nullptr;                // all lattices, 256-byte aligned each
  unsigned long long* d_trace = nullptr;    // per job [nsweeps][2]
  unsigned long long* d_em0 = nullptr;      // per job [2]
  int* d_counters = nullptr;                // one queue head per group
  int8_t* d_scratch = nullptr;              // ping-pong buffer of the loop mode
  int* d_err = nullptr;
  unsigned long long* d_obs = nullptr;
  size_t spin_bytes = 0, trace_words = 0;
  int64_t maxN = 0;
  std::vector<Group> groups;
  cudaStream_t st = nullptr;
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t graph = nullptr;
  int last_mode = -1;
};

namespace {

void multi_free(spn_multi_ctx* m) {
  if (!m) return;
  if (m->graph) cudaGraphExecDestroy(m->graph);
  for (Group& g : m->groups) {
    cudaFree(g.d_inst);
    cudaFree(g.d_order);
    if (g.st) cudaStreamDestroy(g.st);
    if (g.done) cudaEventDestroy(g.done);
  }
  if (m->fork) cudaEventDestroy(m->fork);
  cudaFree(m->d_spins);
  cudaFree(m->d_trace);
  cudaFree(m->d_em0);
  cudaFree(m->d_counters);
  cudaFree(m->d_scratch);
  cudaFree(m->d_err);
  cudaFree(m->d_obs);
  delete m;
}

// Launch shape of a group: cs CTAs (a cluster) per lattice, `threads` per CTA,
// as many CTAs as fit the GPU (at most one cluster per job).
void set_launch(Group& g, int cs, int threads) {
  g.cs = cs;
  g.threads = threads;
  g.smem = spn::resident_smem(g.nd, g.Lx, g.Ly, g.Lz, cs);
  const int maxc = spn::resident_max_ctas(g.nd, cs, threads, g.smem);
  g.ctas = std::max(cs, std::min<int>(maxc, (int)g.jobs.size() * cs));
}

// zeroing + the group launches, on m->st (forks to the group streams)
cudaError_t enqueue_batched(spn_multi_ctx* m) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(m->d_trace, 0, m->trace_words * 8, m->st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(m->d_em0, 0, m->jobs.size() * 16, m->st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(m->d_counters, 0, m->groups.size() * sizeof(int), m->st)) != cudaSuccess) return e;
  if ((e = cudaEventRecord(m->fork, m->st)) != cudaSuccess) return e;
  for (size_t gi = 0; gi < m->groups.size(); ++gi) {
    Group& g = m->groups[gi];
    if ((e = cudaStreamWaitEvent(g.st, m->fork, 0)) != cudaSuccess) return e;
    spn::ResArgs a{};
    a.inst = g.d_inst;
    a.ninst = (int)g.jobs.size();
    a.order = g.d_order;
    a.counter = m->d_counters + gi;
    a.err = m->d_err;
    a.no_always = g.no_always;
    if ((e = spn::launch_resident(a, g.nd, g.cs, g.threads, g.ctas, g.smem, g.st)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(g.done, g.st)) != cudaSuccess) return e;
  }
  for (Group& g : m->groups)
    if ((e = cudaStreamWaitEvent(m->st, g.done, 0)) != cudaSuccess) return e;
  return cudaSuccess;
}

cudaError_t run_loop(spn_multi_ctx* m) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(m->d_trace, 0, m->trace_words * 8, m->st)) != cudaSuccess) return e;
  for (size_t i = 0; i < m->jobs.size(); ++i) {
    const spn_job& j = m->jobs[i];
    spn::Lattice g;
    g.nd = j.model == SPN_ISING2D ? 2 : 3;
    g.Lx = j.dims[0];
    g.Ly = j.dims[1];
    g.Lz = g.nd == 3 ? j.dims[2] : 1;
    g.N = m->N[i];
    int8_t* s = m->d_spins + m->spin_off[i];
    if ((e = spn::launch_init_hot(g, s, j.seed, j.stream, m->st)) != cudaSuccess) return e;
    if ((e = spn::launch_observables(g, s, m->d_em0 + 2 * i, nullptr, m->st)) != cudaSuccess) return e;
    const spn::DevThr T = spn::make_thresholds(j.beta);
    const spn::PhiloxKeys K = spn::philox_keys(j.seed);
    const int ty = g.nd == 3 ? (g.Ly % 32 == 0 ? 32 : (g.Ly % 16 == 0 ? 16 : (g.Ly % 8 == 0 ? 8 : 2))) : 1;
    bool stream = spn::stream_path_supported(g, ty) && g.N >= (1 << 16);
    spn::StreamGeom geo{};
    if (stream) {
      geo = spn::stream_geometry(g, ty, 0, 0);
      stream = spn::stream_geometry_ok(g, geo);
    }
    int8_t* bufs[2] = {s, m->d_scratch};
    int cur = 0;
    for (int64_t t = 0; t < j.nsweeps; ++t) {
      unsigned long long* acc = m->d_trace + m->trace_off[i] + 2 * t;
      if (stream) {
        e = spn::launch_sweep_stream(g, bufs[cur], bufs[cur ^ 1], geo, T, K, j.stream, (uint32_t)t, acc, m->d_err,
                                     m->st);
        cur ^= 1;
      } else {
        e = spn::launch_sweep_generic(g, s, T, K, j.stream, (uint32_t)t, acc, m->st);
      }
      if (e != cudaSuccess) return e;
    }
    if (cur == 1 && (e = cudaMemcpyAsync(s, m->d_scratch, (size_t)g.N, cudaMemcpyDeviceToDevice, m->st)) !=
                        cudaSuccess)
      return e;
  }
  return cudaSuccess;
}

}  // namespace

extern "C" {

int spn_multi_create(spn_multi* out, const spn_job* jobs, int njobs) {
  if (!out || !jobs || njobs < 1) return mfail(SPN_E_ARG, "bad arguments");
  *out = nullptr;
  spn_multi_ctx* m = new (std::nothrow) spn_multi_ctx;
  if (!m) return mfail(SPN_E_NOMEM, "host allocation failed");
  auto bail = [&](int code, const char* msg) {
    multi_free(m);
    return mfail(code, msg);
  };
  m->jobs.assign(jobs, jobs + njobs);
  std::map<std::tuple<int, int, int, int>, std::vector<int>> by_shape;
  for (int i = 0; i < njobs; ++i) {
    const spn_job& j = jobs[i];
    if (j.model != SPN_ISING2D && j.model != SPN_ISING3D) return bail(SPN_E_ARG, "jobs must be Ising 2D or 3D");
    const int nd = j.model == SPN_ISING2D ? 2 : 3;
    const int ext[3] = {j.dims[0], j.dims[1], nd == 3 ? j.dims[2] : 1};
    for (int d = 0; d < nd; ++d)
      if (ext[d] < 2 || (ext[d] & 1)) return bail(SPN_E_ARG, "every extent must be even and >= 2");
    if (!spn::counter_range_ok(ext[0], ext[1], ext[2]))
      return bail(SPN_E_ARG, "lattice too large for the random-number counter (more than 2^29 row words)");
    if (!(j.beta >= 0.0)) return bail(SPN_E_ARG, "beta must be >= 0");
    if (j.nsweeps < 0 || j.nsweeps > 0xffffffffLL) return bail(SPN_E_ARG, "bad nsweeps");
    const int64_t N = (int64_t)ext[0] * ext[1] * ext[2];
    m->N.push_back(N);
    m->maxN = std::max(m->maxN, N);
    m->spin_off.push_back(m->spin_bytes);
    m->spin_bytes += ((size_t)N + 255) & ~(size_t)255;
    m->trace_off.push_back(m->trace_words);
    m->trace_words += 2 * (size_t)j.nsweeps;
    by_shape[{nd, ext[0], ext[1], ext[2]}].push_back(i);
  }
  if (m->trace_words == 0) m->trace_words = 2;
  cudaError_t e;
  if ((e = cudaMalloc(&m->d_spins, m->spin_bytes)) != cudaSuccess) return bail(SPN_E_NOMEM, "cudaMalloc(spins)");
  if ((e = cudaMalloc(&m->d_trace, m->trace_words * 8)) != cudaSuccess) return bail(SPN_E_NOMEM, "cudaMalloc");
  if ((e = cudaMalloc(&m->d_em0, (size_t)njobs * 16)) != cudaSuccess) return bail(SPN_E_NOMEM, "cudaMalloc");
  if ((e = cudaMalloc(&m->d_err, 4)) != cudaSuccess) return bail(SPN_E_NOMEM, "cudaMalloc");
  if ((e = cudaMalloc(&m->d_obs, 16)) != cudaSuccess) return bail(SPN_E_NOMEM, "cudaMalloc");
  if (cudaMemset(m->d_err, 0, 4) != cudaSuccess) return bail(SPN_E_CUDA, "cudaMemset");
  if (cudaEventCreateWithFlags(&m->fork, cudaEventDisableTiming) != cudaSuccess) return bail(SPN_E_CUDA, "event");
  for (auto& kv : by_shape) {
    Group g;
    std::tie(g.nd, g.Lx, g.Ly, g.Lz) = kv.first;
    g.cs = spn::resident_cluster_size(g.nd, g.Lx, g.Ly, g.Lz);
    if (g.cs == 0) return bail(SPN_E_ARG, "a job lattice does not fit the resident batched kernel (at most "
                                          "8 x 200 KB of bits, rows divisible among the cluster)");
    g.jobs = kv.second;
    std::stable_sort(g.jobs.begin(), g.jobs.end(),
                     [&](int a, int b) { return m->jobs[a].nsweeps > m->jobs[b].nsweeps; });
    {
      const int W = (g.Lx + 63) / 64;
      const int items = (g.Ly * (g.nd == 3 ? g.Lz : 1) + g.cs - 1) / g.cs * W;
      int cs = g.cs, threads = std::min(512, std::max(64, (items + 31) / 32 * 32));
      std::lock_guard<std::mutex> lock(g_tune_mu);
      auto it = g_tuned.find({g.nd, g.Lx, g.Ly, g.Lz, spn::device_sm_count()});
      if (it != g_tuned.end()) std::tie(cs, threads) = it->second;  // an earlier autotune of this shape
      set_launch(g, cs, threads);
    }
    std::vector<spn::ResInst> inst(g.jobs.size());
    std::vector<int> order(g.jobs.size());
    for (size_t k = 0; k < g.jobs.size(); ++k) {
      const int i = g.jobs[k];
      const spn_job& j = m->jobs[i];
      spn::ResInst& r = inst[k];
      r.spins = m->d_spins + m->spin_off[i];
      r.trace = m->d_trace + m->trace_off[i];
      r.em0 = m->d_em0 + 2 * i;
      r.seed = j.seed;
      r.stream = j.stream;
      r.sweep0 = 0;
      r.nsweeps = (int)j.nsweeps;
      r.init_hot = 1;
      r.Lx = g.Lx;
      r.Ly = g.Ly;
      r.Lz = g.Lz;
      r.T = spn::make_thresholds(j.beta);
      g.no_always = g.no_always && spn::no_always_class(r.T);
      order[k] = (int)k;
    }
    if (cudaMalloc(&g.d_inst, inst.size() * sizeof(spn::ResInst)) != cudaSuccess ||
        cudaMalloc(&g.d_order, order.size() * sizeof(int)) != cudaSuccess) {
      m->groups.push_back(g);
      return bail(SPN_E_NOMEM, "cudaMalloc(instances)");
    }
    cudaMemcpy(g.d_inst, inst.data(), inst.size() * sizeof(spn::ResInst), cudaMemcpyHostToDevice);
    cudaMemcpy(g.d_order, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice);
    cudaStreamCreateWithFlags(&g.st, cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming);
    m->groups.push_back(g);
  }
  if (cudaMalloc(&m->d_counters, m->groups.size() * sizeof(int)) != cudaSuccess)
    return bail(SPN_E_NOMEM, "cudaMalloc(counters)");
  *out = m;
  return SPN_OK;
}

int spn_multi_set_stream(spn_multi m, void* cuda_stream) {
  if (!m) return mfail(SPN_E_ARG, "NULL handle");
  cudaStreamSynchronize(m->st);
  m->st = static_cast<cudaStream_t>(cuda_stream);
  if (m->graph) {
    cudaGraphExecDestroy(m->graph);
    m->graph = nullptr;
  }
  return SPN_OK;
}

int spn_multi_run(spn_multi m, int mode) {
  if (!m) return mfail(SPN_E_ARG, "NULL handle");
  cudaError_t e;
  if (mode == SPN_RUN_LOOP) {
    if (!m->d_scratch && cudaMalloc(&m->d_scratch, (size_t)m->maxN) != cudaSuccess)
      return mfail(SPN_E_NOMEM, "cudaMalloc(scratch)");
    if ((e = run_loop(m)) != cudaSuccess) return mfail(SPN_E_CUDA, cudaGetErrorString(e));
    m->last_mode = mode;
    return SPN_OK;
  }
  if (mode != SPN_RUN_BATCHED) return mfail(SPN_E_ARG, "unknown mode");
  if (!m->graph) {
    // capture the zeroing and the concurrent group launches once
    cudaStream_t cap = nullptr;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return mfail(SPN_E_CUDA, "stream");
    cudaStream_t user = m->st;
    m->st = cap;
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e2 = enqueue_batched(m);
      e = cudaStreamEndCapture(cap, &graph);
      if (e2 != cudaSuccess) e = e2;
    }
    m->st = user;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&m->graph, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) return mfail(SPN_E_CUDA, cudaGetErrorString(e));
  }
  if ((e = cudaGraphLaunch(m->graph, m->st)) != cudaSuccess) return mfail(SPN_E_CUDA, cudaGetErrorString(e));
  m->last_mode = mode;
  return SPN_OK;
}

int spn_multi_sync(spn_multi m) {
  if (!m) return mfail(SPN_E_ARG, "NULL handle");
  cudaError_t e = cudaStreamSynchronize(m->st);
  if (e != cudaSuccess) return mfail(SPN_E_CUDA, cudaGetErrorString(e));
  int err = 0;
  cudaMemcpy(&err, m->d_err, 4, cudaMemcpyDeviceToHost);
  if (err) return mfail(SPN_E_TIMEOUT, "a bounded device wait ran out");
  return SPN_OK;
}

int spn_multi_result(spn_multi m, int job, int8_t* spins, size_t bytes, int64_t* E, int64_t* M, int64_t cap) {
  if (!m || job < 0 || job >= (int)m->jobs.size()) return mfail(SPN_E_ARG, "bad job index");
  int rc = spn_multi_sync(m);
  if (rc) return rc;
  if (spins) {
    if (bytes != (size_t)m->N[job]) return mfail(SPN_E_ARG, "bytes must be N of the job");
    if (cudaMemcpy(spins, m->d_spins + m->spin_off[job], bytes, cudaMemcpyDeviceToHost) != cudaSuccess)
      return mfail(SPN_E_CUDA, "reading the lattice");
  }
  if (cap > 0 && E && M) {
    const int64_t n = std::min<int64_t>(cap, m->jobs[job].nsweeps);
    std::vector<unsigned long long> d((size_t)2 * m->jobs[job].nsweeps + 2);
    unsigned long long em[2];
    if (cudaMemcpy(em, m->d_em0 + 2 * job, 16, cudaMemcpyDeviceToHost) != cudaSuccess ||
        (m->jobs[job].nsweeps > 0 && cudaMemcpy(d.data(), m->d_trace + m->trace_off[job],
                                                (size_t)m->jobs[job].nsweeps * 16, cudaMemcpyDeviceToHost) !=
                                         cudaSuccess))
      return mfail(SPN_E_CUDA, "reading the trace");
    int64_t e = (int64_t)em[0], mm = (int64_t)em[1];
    for (int64_t t = 0; t < n; ++t) {
      e += (int64_t)d[2 * t];
      mm += (int64_t)d[2 * t + 1];
      E[t] = e;
      M[t] = mm;
    }
  }
  return SPN_OK;
}

int spn_multi_destroy(spn_multi m) {
  if (!m) return mfail(SPN_E_ARG, "NULL handle");
  cudaStreamSynchronize(m->st);
  multi_free(m);
  return SPN_OK;
}

// The autotuner of the batched run (the best tile depends on the lattice size,
// Sec. 4).  A trial is the whole batch at reduced length -- every job from its
// hot start with its sweeps scaled so the longest has trial_sweeps, no traces
// -- with all lattice shapes launched together as in a real run, so launch
// shapes are judged by how they share the GPU.  Starting from the current
// shapes, each lattice shape in turn tries every cluster size and thread count
// and keeps the fastest trial (coordinate descent).
int spn_multi_autotune(spn_multi m, int32_t trial_sweeps, double* rates, size_t count) {
  if (!m || trial_sweeps < 1) return mfail(SPN_E_ARG, "bad arguments");
  if (rates && count != m->groups.size()) return mfail(SPN_E_ARG, "count must be the number of lattice shapes");
  if (cudaStreamSynchronize(m->st) != cudaSuccess) return mfail(SPN_E_CUDA, "synchronising");
  int64_t longest = 1;
  for (const spn_job& j : m->jobs) longest = std::max<int64_t>(longest, j.nsweeps);
  const double scale = std::min(1.0, (double)trial_sweeps / (double)longest);
  std::vector<spn::ResInst*> trial(m->groups.size(), nullptr);
  double att = 0.0;
  int rc = SPN_OK;
  for (size_t gi = 0; gi < m->groups.size() && rc == SPN_OK; ++gi) {
    Group& g = m->groups[gi];
    std::vector<spn::ResInst> inst(g.jobs.size());
    if (cudaMemcpy(inst.data(), g.d_inst, inst.size() * sizeof(spn::ResInst), cudaMemcpyDeviceToHost) != cudaSuccess) {
      rc = mfail(SPN_E_CUDA, "reading the instances");
      break;
    }
    for (size_t k = 0; k < inst.size(); ++k) {
      inst[k].nsweeps = inst[k].nsweeps > 0 ? std::max(1, (int)std::lround(inst[k].nsweeps * scale)) : 0;
      inst[k].trace = nullptr;
      inst[k].em0 = nullptr;
      att += (double)m->N[g.jobs[k]] * inst[k].nsweeps;
    }
    if (cudaMalloc(&trial[gi], inst.size() * sizeof(spn::ResInst)) != cudaSuccess ||
        cudaMemcpy(trial[gi], inst.data(), inst.size() * sizeof(spn::ResInst), cudaMemcpyHostToDevice) != cudaSuccess)
      rc = mfail(SPN_E_NOMEM, "trial instances");
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (rc == SPN_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    rc = mfail(SPN_E_CUDA, "events");
  // one trial of the current launch shapes: attempts/ns (the better of two runs)
  auto run_trial = [&](double* rate) -> int {
    double best = 0.0;
    for (int rep = 0; rep < 2; ++rep) {
      if (cudaMemsetAsync(m->d_counters, 0, m->groups.size() * sizeof(int), m->st) != cudaSuccess ||
          cudaEventRecord(e0, m->st) != cudaSuccess || cudaEventRecord(m->fork, m->st) != cudaSuccess)
        return SPN_E_CUDA;
      for (size_t gi = 0; gi < m->groups.size(); ++gi) {
        Group& g = m->groups[gi];
        spn::ResArgs a{};
        a.inst = trial[gi];
        a.ninst = (int)g.jobs.size();
        a.order = g.d_order;
        a.counter = m->d_counters + gi;
        a.err = m->d_err;
        a.no_always = g.no_always;
        if (cudaStreamWaitEvent(g.st, m->fork, 0) != cudaSuccess ||
            spn::launch_resident(a, g.nd, g.cs, g.threads, g.ctas, g.smem, g.st) != cudaSuccess ||
            cudaEventRecord(g.done, g.st) != cudaSuccess || cudaStreamWaitEvent(m->st, g.done, 0) != cudaSuccess)
          return SPN_E_CUDA;
      }
      float ms = 0.0f;
      if (cudaEventRecord(e1, m->st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        return SPN_E_CUDA;
      best = std::max(best, att / ((double)ms * 1e6));
    }
    *rate = best;
    return SPN_OK;
  };
  double best_rate = 0.0;
  if (rc == SPN_OK && run_trial(&best_rate) != SPN_OK) rc = mfail(SPN_E_CUDA, "autotune trial");
  for (size_t gi = 0; gi < m->groups.size() && rc == SPN_OK; ++gi) {
    Group& g = m->groups[gi];
    int best_cs = g.cs, best_t = g.threads;
    const int cs_min = spn::resident_cluster_size(g.nd, g.Lx, g.Ly, g.Lz);
    for (int cs = cs_min; cs <= 8 && rc == SPN_OK; cs *= 2) {
      if (!spn::resident_supported(g.nd, g.Lx, g.Ly, g.Lz, cs)) continue;
      const int W = (g.Lx + 63) / 64;
      const int items = (g.Ly * (g.nd == 3 ? g.Lz : 1) + cs - 1) / cs * W;
      for (int threads = 64; threads <= 512 && rc == SPN_OK; threads *= 2) {
        if (threads > 64 && threads / 2 >= items) break;  // no more useful threads
        if (cs == best_cs && threads == best_t) continue;  // the incumbent
        set_launch(g, cs, threads);
        double r = 0.0;
        if (run_trial(&r) != SPN_OK) {
          rc = mfail(SPN_E_CUDA, "autotune trial");
        } else if (r > best_rate * 1.01) {  // a clear win only
          best_rate = r;
          best_cs = cs;
          best_t = threads;
        }
      }
    }
    set_launch(g, best_cs, best_t);
    if (rates) rates[gi] = best_rate;
    if (rc == SPN_OK) {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      g_tuned[{g.nd, g.Lx, g.Ly, g.Lz, spn::device_sm_count()}] = {best_cs, best_t};
    }
  }
  for (spn::ResInst* p : trial) cudaFree(p);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (m->graph) {  // the next batched run captures the new launch shapes
    cudaGraphExecDestroy(m->graph);
    m->graph = nullptr;
  }
  return rc;
}

int spn_multi_groups(spn_multi m, int32_t* out, size_t count) {
  if (!m || !out || count != m->groups.size() * 7) return mfail(SPN_E_ARG, "count must be 7 per lattice shape");
  for (size_t gi = 0; gi < m->groups.size(); ++gi) {
    const Group& g = m->groups[gi];
    const int32_t v[7] = {g.nd, g.Lx, g.Ly, g.Lz, g.cs, g.threads, g.ctas};
    std::memcpy(out + 7 * gi, v, sizeof v);
  }
  return SPN_OK;
}

int spn_multi_set_launch(spn_multi m, int32_t group, int32_t cs, int32_t threads) {
  if (!m || group < 0 || group >= (int)m->groups.size()) return mfail(SPN_E_ARG, "bad group index");
  Group& g = m->groups[group];
  if (threads < 32 || threads > 512 || threads % 32 || cs > 8 || !spn::resident_supported(g.nd, g.Lx, g.Ly, g.Lz, cs) ||
      (cs & (cs - 1)))
    return mfail(SPN_E_ARG, "cluster size must be 1, 2, 4 or 8 and fit; threads a multiple of 32 up to 512");
  if (cudaStreamSynchronize(m->st) != cudaSuccess) return mfail(SPN_E_CUDA, "synchronising");
  set_launch(g, cs, threads);
  if (m->graph) {
    cudaGraphExecDestroy(m->graph);
    m->graph = nullptr;
  }
  return SPN_OK;
}

}  // extern "C"
