// Request server with continuous batching (spn_server_* ABI).
//
// Clients submit jobs at any time; spn_submit copies the request and returns a
// ticket without touching the GPU.  A scheduler thread works in rounds: it
// admits queued jobs while their device memory fits the HBM budget (stream-
// ordered allocations), then advances every admitted job by one window of
// sweeps.  Ising jobs whose lattice fits the resident kernel share one
// persistent launch per lattice shape; other Ising shapes and the
// multi-spin coded EA jobs get their own launches on a pool of streams, so the
// whole round overlaps on the device.  Jobs that arrive during a round join the
// next one.  A finished job's lattice and energy are copied to host memory, its
// device memory returns to the budget, and spn_poll reports it with its
// submit / admit / done times.  A window only splits the sweep sequence, and
// the random numbers are counters of (seed, stream, sweep, site), so a job's
// result does not depend on what else runs with it.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <numeric>
#include <thread>
#include <tuple>
#include <vector>

#include "spn.h"
#include "spn_internal.h"

namespace {

// A round runs up to a few dozen launches at once on the stream pool; the
// default 8 hardware work queues would serialise the ninth launch behind the
// first.  Set when the library is loaded, before any CUDA context exists (a
// value the process already has is kept; once a context exists it has no effect).
__attribute__((constructor)) void more_hardware_queues() { setenv("CUDA_DEVICE_MAX_CONNECTIONS", "32", 0); }

double now_s() {
  using clk = std::chrono::steady_clock;
  static const clk::time_point t0 = clk::now();
  return std::chrono::duration<double>(clk::now() - t0).count();
}

int sfail(int code, const char* msg) {
  spn::set_last_error(msg);
  return code;
}

enum JobState { kPending = 0, kAdmitted = 1, kDone = 2, kFailed = 3 };

constexpr int kPoolStreams = 32;  // concurrent launches of one round

struct Job {
  uint64_t ticket = 0;
  spn_request req{};
  std::vector<double> betas;
  std::vector<uint64_t> bonds;
  int state = kPending;
  int status = SPN_OK;
  double t_submit = 0, t_admit = 0, t_done = 0;
  int64_t done = 0;  // sweeps done
  int64_t window = 0;  // sweeps of the current round
  size_t bytes = 0;  // device bytes charged to the budget
  int nd = 2;
  int64_t N = 0;
  int cs = 0;        // resident cluster size (0: not resident)
  bool streaming = false;  // bit-packed ping-pong lattices for the streaming sweep
  spn::StreamGeom geo{};
  int8_t* d_spins = nullptr;
  int8_t* d_scratch = nullptr;
  uint32_t* d_p0 = nullptr;  // bit-packed lattice (current)
  uint32_t* d_p1 = nullptr;  // bit-packed ping-pong partner
  unsigned long long* d_acc = nullptr;  // window deltas / start E, M
  spn_handle ea = nullptr;
  std::unique_ptr<spn::EaPrep> prep;  // EA: host part built on a worker thread before admission
  int prep_rc = SPN_OK;
  int stream_slot = 0;
  // round planning: the SM equivalents the job's launch shape takes while it
  // runs, its attempts per ns while running (estimated at first, then
  // measured per window on the resident path) and the last round that gave it
  // a window
  double fsm = 0;
  double rsm = 0;  // attempts per ns and SM equivalent (0: not yet known)
  uint64_t last_run = 0;
  // resident: this round's cluster size (cs or wider) and its launch shape:
  // threads (a power of two, 64 .. 512), shared memory, CTAs resident at once
  int rcs = 0;
  int threads = 64;
  size_t smem = 0;
  int occ = 1;
  // results
  int64_t E = 0, M = 0;
  std::vector<int8_t> spins;
  std::vector<uint32_t> words;
  std::vector<uint8_t> slots;
};

}  // namespace

struct spn_server_ctx {
  size_t budget = 0;
  size_t used = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::shared_ptr<Job>> pending;
  std::vector<std::shared_ptr<Job>> active;
  std::map<uint64_t, std::shared_ptr<Job>> all;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  int device = 0;
  cudaStream_t main = nullptr;
  // admissions and finished-job read-back run here while a round executes; a
  // round starts after the admissions enqueued before it (aux_ev)
  cudaStream_t aux = nullptr;
  cudaEvent_t aux_ev = nullptr;
  std::vector<cudaStream_t> pool;
  std::vector<cudaEvent_t> pool_done;
  cudaEvent_t fork = nullptr;
  spn::ResInst* d_inst = nullptr;  // per-round resident instances
  spn::EaArgs* d_ea = nullptr;     // per-round EA job blocks
  size_t ea_cap = 0;
  int* d_order = nullptr;
  int* d_counters = nullptr;
  int* d_err = nullptr;
  size_t inst_cap = 0;
  double round_ns = 3.0e7;  // a window is about this much of its job's own run time
  // share of the SMs a round plans for: clusters sit within one GPC, so the
  // GPU holds less than its SM count in mixed launches; lowered when an
  // instance of a round started late (a second wave), raised otherwise
  double fill = 0.9;
  uint64_t round_no = 0;
  std::map<std::tuple<int, int, int, size_t>, int> max_ctas;  // resident launch shape -> CTAs resident at once
  unsigned long long* d_tns = nullptr;  // per-round instance clocks [instance][start, end]
  unsigned long long* h_tns = nullptr;  // pinned copy, read after the round
  std::vector<Job*> res_jobs;           // per-round instance -> its job
  int64_t stream_sites = (int64_t)1 << 20;     // Ising jobs from this many sites up stream (if not resident)
  std::atomic<unsigned long long> attempts{0};
  std::atomic<unsigned long long> rounds{0};
  double busy = 0;
  std::FILE* trace = nullptr;  // per-round log when SPN_SERVER_TRACE names a file
  // with a trace: a timing event after each launch group of a round (resident
  // launch, EA launch, streaming job), its path and attempts, and the round's start
  std::vector<cudaEvent_t> tev;
  std::vector<std::pair<int, long long>> tmark;
  cudaEvent_t tstart = nullptr;
  int* h_err = nullptr;        // pinned: the round's device error word, read back with the round
  // Finished jobs are read back on a thread and a high-priority stream of
  // their own: the next round starts at once, the read-back's small kernels
  // slip in beside it, and its copies to the host overlap the round.
  std::thread reader;
  std::deque<std::shared_ptr<Job>> rb_queue;  // guarded by mu
  std::condition_variable rb_cv;
  bool rb_stop = false;
  cudaStream_t rb = nullptr;
};

namespace {

size_t job_bytes(const Job& j) {
  if (j.req.model == SPN_EA3D_PMJ) return (size_t)j.N * 9 + 64 * 1024;  // words + bond bytes + tables
  size_t b = (size_t)j.N + 4096;
  if (j.streaming) b += 2 * (size_t)spn::packed_row_words(j.req.dims[0]) * 4 * (size_t)(j.N / j.req.dims[0]);
  return b;
}

// A job's device memory goes back in stream order on st: its last kernels ran
// in a round that has completed, or on st itself (read-back, admission).
void release(Job& j, cudaStream_t st) {
  if (j.d_spins) cudaFreeAsync(j.d_spins, st);
  if (j.d_scratch) cudaFreeAsync(j.d_scratch, st);
  if (j.d_p0) cudaFreeAsync(j.d_p0, st);
  if (j.d_p1) cudaFreeAsync(j.d_p1, st);
  if (j.d_acc) cudaFreeAsync(j.d_acc, st);
  j.d_spins = j.d_scratch = nullptr;
  j.d_p0 = j.d_p1 = nullptr;
  j.d_acc = nullptr;
  if (j.ea) {
    spn_destroy(j.ea);
    j.ea = nullptr;
  }
}

// Allocate and initialise an admitted job (scheduler thread), stream-ordered on
// aux: nothing here waits for the device.
int admit(spn_server_ctx* s, Job& j) {
  const spn_request& r = j.req;
  if (r.model == SPN_EA3D_PMJ) {
    if (j.prep_rc) return j.prep_rc;
    const int rc = spn::ea_upload_async(&j.ea, *j.prep, s->aux);
    j.prep.reset();
    return rc;
  }
  spn::Lattice g;
  g.nd = j.nd;
  g.Lx = r.dims[0];
  g.Ly = r.dims[1];
  g.Lz = j.nd == 3 ? r.dims[2] : 1;
  g.N = j.N;
  if (cudaMallocAsync(&j.d_spins, (size_t)j.N, s->aux) != cudaSuccess) return SPN_E_NOMEM;
  if (cudaMallocAsync(&j.d_acc, 4096, s->aux) != cudaSuccess) return SPN_E_NOMEM;
  if (spn::launch_init_hot(g, j.d_spins, r.seed, r.stream, s->aux) != cudaSuccess) return SPN_E_CUDA;
  if (j.streaming) {  // the hot start packed to 1 bit per spin; padding words of both buffers zero
    const size_t pb = (size_t)spn::packed_row_words(g.Lx) * 4 * (size_t)(j.N / g.Lx);
    if (cudaMallocAsync(&j.d_p0, pb, s->aux) != cudaSuccess || cudaMallocAsync(&j.d_p1, pb, s->aux) != cudaSuccess)
      return SPN_E_NOMEM;
    if (cudaMemsetAsync(j.d_p0, 0, pb, s->aux) != cudaSuccess || cudaMemsetAsync(j.d_p1, 0, pb, s->aux) != cudaSuccess ||
        spn::launch_pack(g, j.d_spins, j.d_p0, s->aux) != cudaSuccess)
      return SPN_E_CUDA;
  }
  return SPN_OK;
}

// Final E, M and the host copies of a finished job (its rounds have completed),
// ordered on st.
int finish(Job& j, cudaStream_t st) {
  if (j.ea) {
    const size_t n = (size_t)j.N;
    j.words.resize(n);
    j.slots.resize(32);
    std::vector<int64_t> E(32), M(32);
    int rc = spn_batch_get_words(j.ea, j.words.data(), n);
    if (!rc) rc = spn_batch_get_slots(j.ea, j.slots.data(), 32);
    if (!rc) rc = spn_batch_energies(j.ea, E.data(), M.data(), 32);
    if (rc) return rc;
    int s0 = 0;  // slot of the lowest temperature
    for (int k = 0; k < 32; ++k)
      if (j.slots[k] == 0) s0 = k;
    j.E = E[s0];
    j.M = M[s0];
    return SPN_OK;
  }
  spn::Lattice g;
  g.nd = j.nd;
  g.Lx = j.req.dims[0];
  g.Ly = j.req.dims[1];
  g.Lz = j.nd == 3 ? j.req.dims[2] : 1;
  g.N = j.N;
  if (j.streaming && spn::launch_unpack(g, j.d_p0, j.d_spins, st) != cudaSuccess) return SPN_E_CUDA;
  if (spn::launch_observables(g, j.d_spins, j.d_acc, nullptr, st) != cudaSuccess) return SPN_E_CUDA;
  unsigned long long em[2];
  j.spins.resize((size_t)j.N);
  if (cudaMemcpyAsync(em, j.d_acc, 16, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(j.spins.data(), j.d_spins, (size_t)j.N, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SPN_E_CUDA;
  j.E = (int64_t)em[0];
  j.M = (int64_t)em[1];
  return SPN_OK;
}

// Trace only: a timing event on st after a launch group of path kind (0
// resident, 1 EA, 2 streaming / generic) that carries att attempts.
void trace_mark(spn_server_ctx* s, cudaStream_t st, int kind, long long att) {
  if (!s->trace) return;
  const size_t k = s->tmark.size();
  if (k == s->tev.size()) {
    cudaEvent_t ev;
    if (cudaEventCreate(&ev) != cudaSuccess) return;
    s->tev.push_back(ev);
  }
  cudaEventRecord(s->tev[k], st);
  s->tmark.emplace_back(kind, att);
}

// Attempts per ns and SM while a job runs, by path: starting estimates, on the
// low side of what a job reaches with the GPU full (a first window that
// overruns stretches the whole round; one that falls short only leaves its
// SMs early); resident jobs then carry the rate measured in their last window.
constexpr double kRateSm2d = 9.0, kRateSm3d = 5.0, kRateSmEa = 16.0;

// Attempts per ns and SM equivalent a job starts with, by path.
double default_rsm(const Job& j) { return j.ea ? kRateSmEa : (j.nd == 2 ? kRateSm2d : kRateSm3d); }

// SM equivalents of a job that is not resident (scheduler thread).
void estimate_other(Job& j) {
  if (j.ea)
    j.fsm = 1.0 / spn::ea_job_per_sm(j.ea);
  else  // one launch per sweep over a share of the GPU
    j.fsm = 0.25 * spn::device_sm_count();
}

// Launch shape of resident job j on clusters of cs CTAs, and its SM equivalents
// (a cluster sits within one GPC, so it may take more SMs than it has CTAs).
void res_shape(spn_server_ctx* s, Job& j, int cs) {
  const int Lx = j.req.dims[0], Ly = j.req.dims[1], Lz = j.nd == 3 ? j.req.dims[2] : 1;
  const int items = (Ly * Lz + cs - 1) / cs * ((Lx + 63) / 64);  // words of one parity per CTA
  int t = 64;
  while (t < 512 && t < items) t *= 2;
  j.rcs = cs;
  j.threads = t;
  j.smem = spn::resident_smem(j.nd, Lx, Ly, Lz, cs);
  // a CTA of more than a quarter of an SM's shared memory gets an SM of its own:
  // CTAs of different launches that would share SMs leave unusable remainders,
  // and one 512-thread CTA already keeps an SM nearly as busy as three
  if (cs == 1 && j.smem > 56 * 1024) j.smem = std::max<size_t>(j.smem, 120 * 1024);
  const auto key = std::make_tuple(j.nd, cs, t, j.smem);
  auto it = s->max_ctas.find(key);
  if (it == s->max_ctas.end())
    it = s->max_ctas.emplace(key, std::max(1, spn::resident_max_ctas(j.nd, cs, t, j.smem))).first;
  j.occ = it->second;
  const double sms = spn::device_sm_count();
  j.fsm = std::min(sms, sms * cs / j.occ);
}

// One round: a window of sweeps for every active job.  round_launch enqueues it
// (after the admissions on aux) and returns; round_wait waits for it.
int round_launch(spn_server_ctx* s, std::vector<std::shared_ptr<Job>>& act) {
  cudaError_t e;
  if (cudaEventRecord(s->aux_ev, s->aux) != cudaSuccess || cudaStreamWaitEvent(s->main, s->aux_ev, 0) != cudaSuccess)
    return SPN_E_CUDA;
  if ((e = cudaEventRecord(s->fork, s->main)) != cudaSuccess) return SPN_E_CUDA;
  for (cudaStream_t p : s->pool) cudaStreamWaitEvent(p, s->fork, 0);
  if (s->trace) {
    s->tmark.clear();
    if (!s->tstart) cudaEventCreate(&s->tstart);
    cudaEventRecord(s->tstart, s->main);
  }
  // Round plan.  The jobs given a window least recently go first, each a
  // window of about round_ns of its own run time at its rate, while the SM
  // equivalents of the windows chosen fit the GPU (a window shorter than
  // round_ns counts in proportion); the others wait for the next round.  Every
  // window then takes about as long as the round, so no launch of the round
  // waits for one long instance, and no cluster waits for a second wave.  When
  // the chosen windows leave SMs idle (few jobs), resident jobs with the most
  // work left run on wider clusters (up to 16 CTAs): the lattice lives in HBM
  // between windows, and the cluster size does not change the result.
  ++s->round_no;
  const double sms = spn::device_sm_count(), cap = s->fill * sms;
  std::vector<int64_t> win(act.size(), 0);
  std::vector<double> cost(act.size(), 0.0);
  auto window = [&](Job& j, int64_t* w, double* c) {
    const int64_t units = j.ea ? 32 * j.N : j.N;  // attempts of one sweep (every replica of an EA job)
    const double rate = (j.rsm > 0 ? j.rsm : default_rsm(j)) * j.fsm;  // attempts per ns
    int64_t n = (int64_t)(s->round_ns * rate / (double)units);
    n = std::max<int64_t>(1, std::min<int64_t>(n, j.req.nsweeps - j.done));
    if (j.ea) n = std::min<int64_t>(n, 2000);  // sweeps of one EA launch
    *w = n;
    *c = j.fsm * std::min(1.0, (double)n * (double)units / (rate * s->round_ns));
  };
  std::vector<size_t> ord(act.size());
  std::iota(ord.begin(), ord.end(), (size_t)0);
  std::stable_sort(ord.begin(), ord.end(), [&](size_t x, size_t y) {
    return act[x]->last_run != act[y]->last_run ? act[x]->last_run < act[y]->last_run : act[x]->ticket < act[y]->ticket;
  });
  double used = 0;
  std::vector<size_t> chosen;
  for (size_t k : ord) {
    Job& j = *act[k];
    j.window = 0;
    if (j.cs > 0)
      res_shape(s, j, j.cs);
    else if (j.fsm <= 0)
      estimate_other(j);
    int64_t w;
    double c;
    window(j, &w, &c);
    if (used > 0 && used + c > cap) continue;
    used += c;
    win[k] = w;
    cost[k] = c;
    chosen.push_back(k);
  }
  if (chosen.size() == act.size() && used < 0.75 * cap) {  // every job has a window: widen clusters, most work left first
    std::vector<size_t> wide;
    for (size_t k : chosen)
      if (act[k]->cs > 0 && win[k] < act[k]->req.nsweeps - act[k]->done) wide.push_back(k);
    std::stable_sort(wide.begin(), wide.end(), [&](size_t x, size_t y) {
      return (act[x]->req.nsweeps - act[x]->done) * act[x]->N > (act[y]->req.nsweeps - act[y]->done) * act[y]->N;
    });
    for (size_t k : wide) {
      Job& j = *act[k];
      const int Lx = j.req.dims[0], Ly = j.req.dims[1], Lz = j.nd == 3 ? j.req.dims[2] : 1;
      // at least one word per thread of a 512-thread CTA after the split
      while (j.rcs * 2 <= spn::kMaxResidentCluster && (Ly * Lz) / (j.rcs * 2) * ((Lx + 63) / 64) >= 512 &&
             spn::resident_supported(j.nd, Lx, Ly, Lz, j.rcs * 2)) {
        const int rcs0 = j.rcs;
        res_shape(s, j, rcs0 * 2);
        int64_t w;
        double c;
        window(j, &w, &c);
        if (used - cost[k] + c > 0.95 * cap) {
          res_shape(s, j, rcs0);  // cached: no occupancy query
          break;
        }
        used += c - cost[k];
        cost[k] = c;
        win[k] = w;
      }
    }
  }
  // resident jobs launch by (dimension, cluster size, threads, CTAs resident
  // at once): a launch takes its group's largest shared memory, and within one
  // such class that does not lower the occupancy its members were costed at
  std::map<std::tuple<int, int, int, int>, std::vector<Job*>> groups;
  for (size_t k : chosen) {
    Job& j = *act[k];
    j.window = win[k];
    j.last_run = s->round_no;
    if (j.cs > 0) groups[std::make_tuple(j.nd, j.rcs, j.threads, j.occ)].push_back(&j);
  }
  std::vector<spn::ResInst> inst;
  std::vector<int> order;
  s->res_jobs.clear();
  struct Launch {
    int nd, cs, threads;
    size_t first, count, smem;
  };
  std::vector<Launch> launches;
  for (auto& kv : groups) {
    std::vector<Job*>& js = kv.second;
    std::stable_sort(js.begin(), js.end(), [](const Job* x, const Job* y) { return x->N * x->window > y->N * y->window; });
    Launch L{std::get<0>(kv.first), std::get<1>(kv.first), 64, inst.size(), js.size(), 0};
    for (size_t k = 0; k < js.size(); ++k) {
      Job* j = js[k];
      spn::ResInst r{};
      r.spins = j->d_spins;
      r.trace = nullptr;  // the server reads E and M at the end
      r.em0 = nullptr;
      r.seed = j->req.seed;
      r.stream = j->req.stream;
      r.sweep0 = (uint32_t)j->done;
      r.nsweeps = (int)j->window;
      r.init_hot = 0;
      r.Lx = j->req.dims[0];
      r.Ly = j->req.dims[1];
      r.Lz = j->nd == 3 ? j->req.dims[2] : 1;
      r.T = spn::make_thresholds(j->req.beta);
      r.tns = nullptr;  // set below, once the clock array holds this round's instances
      inst.push_back(r);
      s->res_jobs.push_back(j);
      order.push_back((int)k);
      L.threads = std::max(L.threads, j->threads);
      L.smem = std::max(L.smem, j->smem);
    }
    launches.push_back(L);
  }
  // EA jobs: one launch per lattice size and random-number mode (a u per slot
  // for jobs with replica exchange), one CTA per job (at most 2000 sweeps a launch)
  struct EaLaunch {
    std::vector<spn::EaArgs> args;
    int threads = 0;  // the same for every job of a group (same N and mode)
    size_t smem = 0;
    long long att = 0;  // attempts of the group's windows
  };
  std::map<int64_t, EaLaunch> ea_groups;  // key 2 N + (a u per slot)
  for (size_t k = 0; k < act.size(); ++k)
    if (act[k]->ea && win[k] > 0) {
      spn::EaArgs a;
      size_t smem = 0;
      int threads = 0;
      if (spn::ea_window_args(act[k]->ea, win[k], &a, &smem, &threads) != SPN_OK) return SPN_E_STATE;
      EaLaunch& g = ea_groups[2 * act[k]->N + (a.u_per_slot ? 1 : 0)];
      g.args.push_back(a);
      g.threads = threads;
      g.smem = smem;
      g.att += 32LL * act[k]->N * win[k];
    }
  std::vector<spn::EaArgs> args;
  std::vector<std::tuple<size_t, size_t, int, size_t, bool>> el;  // first, count, threads, smem, per-slot
  std::vector<long long> el_att;
  for (auto& kv : ea_groups) {
    el.emplace_back(args.size(), kv.second.args.size(), kv.second.threads, kv.second.smem, (kv.first & 1) != 0);
    el_att.push_back(kv.second.att);
    args.insert(args.end(), kv.second.args.begin(), kv.second.args.end());
  }
  if (!inst.empty()) {
    if (inst.size() > s->inst_cap) {
      cudaFree(s->d_inst);
      cudaFree(s->d_order);
      cudaFree(s->d_counters);
      cudaFree(s->d_tns);
      cudaFreeHost(s->h_tns);
      s->h_tns = nullptr;
      s->inst_cap = inst.size() * 2;
      if (cudaMalloc(&s->d_inst, s->inst_cap * sizeof(spn::ResInst)) != cudaSuccess ||
          cudaMalloc(&s->d_order, s->inst_cap * sizeof(int)) != cudaSuccess ||
          cudaMalloc(&s->d_counters, s->inst_cap * sizeof(int)) != cudaSuccess ||
          cudaMalloc(&s->d_tns, s->inst_cap * 2 * sizeof(unsigned long long)) != cudaSuccess ||
          cudaMallocHost(&s->h_tns, s->inst_cap * 2 * sizeof(unsigned long long)) != cudaSuccess)
        return SPN_E_NOMEM;
    }
    for (size_t k = 0; k < inst.size(); ++k) inst[k].tns = s->d_tns + 2 * k;
    if (cudaMemcpyAsync(s->d_inst, inst.data(), inst.size() * sizeof(spn::ResInst), cudaMemcpyHostToDevice,
                        s->main) != cudaSuccess ||
        cudaMemcpyAsync(s->d_order, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice, s->main) !=
            cudaSuccess ||
        cudaMemsetAsync(s->d_counters, 0, launches.size() * sizeof(int), s->main) != cudaSuccess ||
        cudaMemsetAsync(s->d_tns, 0, inst.size() * 2 * sizeof(unsigned long long), s->main) != cudaSuccess)
      return SPN_E_CUDA;
  }
  if (!args.empty()) {
    if (args.size() > s->ea_cap) {
      cudaFree(s->d_ea);
      s->ea_cap = args.size() * 2;
      if (cudaMalloc(&s->d_ea, s->ea_cap * sizeof(spn::EaArgs)) != cudaSuccess) return SPN_E_NOMEM;
    }
    if (cudaMemcpyAsync(s->d_ea, args.data(), args.size() * sizeof(spn::EaArgs), cudaMemcpyHostToDevice, s->main) !=
        cudaSuccess)
      return SPN_E_CUDA;
  }
  if (cudaEventRecord(s->fork, s->main) != cudaSuccess) return SPN_E_CUDA;
  // Launch order: the largest clusters first, then the largest shared memory
  // per CTA, on the pool's high-priority streams first.  A cluster needs free
  // SMs within one GPC and a large CTA a nearly free SM: issued after many
  // small CTAs, which spread over every SM, they would wait for those to finish.
  std::vector<std::tuple<int, size_t, int>> issue;  // (cluster size, shared memory per CTA, launch li >= 0 / EA -1 - gi)
  for (size_t li = 0; li < launches.size(); ++li) issue.emplace_back(launches[li].cs, launches[li].smem, (int)li);
  for (size_t gi = 0; gi < el.size(); ++gi) issue.emplace_back(1, std::get<3>(el[gi]), -1 - (int)gi);
  std::stable_sort(issue.begin(), issue.end(),
                   [](const std::tuple<int, size_t, int>& x, const std::tuple<int, size_t, int>& y) {
                     return std::get<0>(x) != std::get<0>(y) ? std::get<0>(x) > std::get<0>(y)
                                                             : std::get<1>(x) > std::get<1>(y);
                   });
  size_t n_hi = 0, n_lo = 0;
  const size_t half = s->pool.size() / 2;
  for (size_t q = 0; q < issue.size(); ++q) {
    const bool big = std::get<0>(issue[q]) > 1 || std::get<1>(issue[q]) > 100 * 1024;
    cudaStream_t st = big ? s->pool[n_hi++ % half] : s->pool[half + n_lo++ % half];
    cudaStreamWaitEvent(st, s->fork, 0);
    const int which = std::get<2>(issue[q]);
    if (which >= 0) {
      const size_t li = (size_t)which;
      const Launch& L = launches[li];
      spn::ResArgs a{};
      a.inst = s->d_inst + L.first;
      a.ninst = (int)L.count;
      a.order = s->d_order + L.first;  // local indices into the launch's slice
      a.counter = s->d_counters + li;
      a.err = s->d_err;
      a.no_always = true;
      for (size_t k = L.first; k < L.first + L.count; ++k) a.no_always = a.no_always && spn::no_always_class(inst[k].T);
      const auto key = std::make_tuple(L.nd, L.cs, L.threads, L.smem);
      auto it = s->max_ctas.find(key);
      if (it == s->max_ctas.end())
        it = s->max_ctas.emplace(key, std::max(1, spn::resident_max_ctas(L.nd, L.cs, L.threads, L.smem))).first;
      const int ctas = std::max(L.cs, std::min<int>(it->second, (int)L.count * L.cs));
      if ((e = spn::launch_resident(a, L.nd, L.cs, L.threads, ctas, L.smem, st)) != cudaSuccess) return SPN_E_CUDA;
      if (s->trace) {
        long long att = 0;
        for (size_t k = L.first; k < L.first + L.count; ++k)
          att += (long long)inst[k].Lx * inst[k].Ly * inst[k].Lz * inst[k].nsweeps;
        trace_mark(s, st, 0, att);
      }
    } else {
      const size_t gi = (size_t)(-1 - which);
      size_t first, count, smem;
      int threads;
      bool ps;
      std::tie(first, count, threads, smem, ps) = el[gi];
      if ((e = spn::launch_ea_jobs(s->d_ea + first, (int)count, 3, ps, threads, smem, st)) != cudaSuccess)
        return SPN_E_CUDA;
      trace_mark(s, st, 1, el_att[gi]);
    }
  }
  // large Ising lattices: own launches on the stream pool
  for (size_t k = 0; k < act.size(); ++k) {
    Job& j = *act[k];
    if (j.cs > 0 || j.ea || win[k] == 0) continue;
    cudaStream_t st = s->pool[j.stream_slot];
    const int64_t w = win[k];
    spn::Lattice g;
    g.nd = j.nd;
    g.Lx = j.req.dims[0];
    g.Ly = j.req.dims[1];
    g.Lz = j.nd == 3 ? j.req.dims[2] : 1;
    g.N = j.N;
    g.pitch = 0;
    const spn::DevThr T = spn::make_thresholds(j.req.beta);
    const spn::PhiloxKeys K = spn::philox_keys(j.req.seed);
    for (int64_t t = 0; t < w; ++t) {
      const uint32_t sweep = (uint32_t)(j.done + t);
      if (j.streaming) {  // ping-pong: the current lattice is always d_p0
        e = spn::launch_sweep_stream(g, j.d_p0, j.d_p1, j.geo, T, K, j.req.stream, sweep, j.d_acc, s->d_err, st);
        std::swap(j.d_p0, j.d_p1);
      } else {
        e = spn::launch_sweep_generic(g, j.d_spins, T, K, j.req.stream, sweep, j.d_acc, st);
      }
      if (e != cudaSuccess) return SPN_E_CUDA;
    }
    trace_mark(s, st, 2, (long long)j.N * w);
  }
  for (size_t p = 0; p < s->pool.size(); ++p) {
    cudaEventRecord(s->pool_done[p], s->pool[p]);
    cudaStreamWaitEvent(s->main, s->pool_done[p], 0);
  }
  if (cudaMemcpyAsync(s->h_err, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, s->main) != cudaSuccess)
    return SPN_E_CUDA;
  if (!s->res_jobs.empty() &&
      cudaMemcpyAsync(s->h_tns, s->d_tns, s->res_jobs.size() * 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                      s->main) != cudaSuccess)
    return SPN_E_CUDA;
  return SPN_OK;
}

int round_wait(spn_server_ctx* s, std::vector<std::shared_ptr<Job>>& act) {
  if (cudaStreamSynchronize(s->main) != cudaSuccess) return SPN_E_CUDA;
  if (*s->h_err) return SPN_E_TIMEOUT;  // a bounded device wait ran out
  // the rate each resident job ran at in this window sizes its next one
  unsigned long long first = ~0ull, last = 0;
  for (size_t k = 0; k < s->res_jobs.size(); ++k) {
    Job& j = *s->res_jobs[k];
    const unsigned long long t0 = s->h_tns[2 * k], t1 = s->h_tns[2 * k + 1];
    // down at once, up by at most 10% a window: a CTA that ran alone on an SM
    // it will share next time would otherwise stretch the next round
    if (t0 && t1 > t0 + 100000ull) {
      const double measured = (double)j.N * (double)j.window / ((double)(t1 - t0) * j.fsm);
      j.rsm = std::min(measured, 1.1 * (j.rsm > 0 ? j.rsm : default_rsm(j)));
    }
    if (t0) {
      first = std::min(first, t0);
      last = std::max(last, t0);
    }
  }
  if (last > first) {  // an instance that started a quarter window late waited for a second wave
    if ((double)(last - first) > 0.25 * s->round_ns)
      s->fill = std::max(0.5, 0.9 * s->fill);
    else
      s->fill = std::min(1.0, 1.02 * s->fill);
  }
  std::lock_guard<std::mutex> lock(s->mu);
  for (auto& jp : act) {
    Job& j = *jp;
    j.done += j.window;
    s->attempts += (unsigned long long)(j.N * j.window * (j.ea ? 32 : 1));
  }
  return SPN_OK;
}

// Mark a finished (or failed) job done and give its bytes back, ordered on st.
void retire(spn_server_ctx* s, const std::shared_ptr<Job>& j, int rc, cudaStream_t st) {
  int frc = rc ? rc : finish(*j, st);
  release(*j, st);
  std::lock_guard<std::mutex> lock(s->mu);
  j->status = frc;
  j->state = frc ? kFailed : kDone;
  j->t_done = now_s();
  s->used -= j->bytes;
}

// The scheduler thread.  Each iteration reads back the jobs the previous round
// completed, launches a round over the active jobs, admits queued jobs while
// it runs (on aux, so nothing waits for the round), and then waits for the
// round.  Newly admitted jobs join the next round.
void scheduler(spn_server_ctx* s) {
  cudaSetDevice(s->device);
  std::vector<std::shared_ptr<Job>> completed;  // finished in the last round, not yet read back
  while (true) {
    std::vector<std::shared_ptr<Job>> admitted_now, act;
    {
      std::unique_lock<std::mutex> lock(s->mu);
      s->cv.wait(lock, [&] {
        return s->stop || !s->pending.empty() || !s->active.empty() || !completed.empty();
      });
      if (s->stop && s->pending.empty() && s->active.empty() && completed.empty()) return;
      // admission against the budget, first come first served
      while (!s->pending.empty()) {
        std::shared_ptr<Job> j = s->pending.front();
        if (s->used + j->bytes > s->budget) break;
        s->pending.pop_front();
        s->used += j->bytes;
        j->state = kAdmitted;
        j->t_admit = now_s();
        admitted_now.push_back(j);
      }
      act = s->active;
    }
    // the jobs the last round completed go to the read-back thread
    if (!completed.empty()) {
      {
        std::lock_guard<std::mutex> lock(s->mu);
        for (auto& j : completed) s->rb_queue.push_back(j);
      }
      s->rb_cv.notify_one();
      completed.clear();
    }
    const double t0 = now_s();
    int rc = SPN_OK;
    if (!act.empty()) rc = round_launch(s, act);
    const double t_launched = now_s();
    // admissions overlap the round: nothing in them waits for the device
    // the host part of EA admissions (bond bytes, exact exchange tables) on worker threads
    {
      std::vector<Job*> ea;
      for (auto& j : admitted_now)
        if (j->req.model == SPN_EA3D_PMJ) ea.push_back(j.get());
      auto prepare = [&](size_t k) {
        Job& j = *ea[k];
        j.prep.reset(new spn::EaPrep);
        j.prep_rc = spn::ea_prepare_single(*j.prep, SPN_EA3D_PMJ, j.req.dims, j.bonds.data(), j.betas.data(),
                                           j.req.seed, j.req.exchange_every);
      };
      const size_t nt = std::min<size_t>(ea.size(), std::max(1u, std::min(8u, std::thread::hardware_concurrency())));
      if (nt <= 1) {
        for (size_t k = 0; k < ea.size(); ++k) prepare(k);
      } else {
        std::atomic<size_t> next{0};
        std::vector<std::thread> workers;
        for (size_t t = 0; t < nt; ++t)
          workers.emplace_back([&] {
            for (size_t k; (k = next.fetch_add(1)) < ea.size();) prepare(k);
          });
        for (auto& w : workers) w.join();
      }
    }
    std::vector<std::shared_ptr<Job>> joined;
    for (auto& j : admitted_now) {
      j->stream_slot = (int)(j->ticket % s->pool.size());
      const int arc = admit(s, *j);
      if (arc) {
        retire(s, j, arc, s->aux);
      } else {
        joined.push_back(j);
      }
    }
    const double t_host = now_s();
    if (!act.empty() && rc == SPN_OK) rc = round_wait(s, act);
    const double t1 = now_s();
    if (!act.empty()) {
      s->busy += t1 - t0;
      s->rounds += 1;
      if (s->trace) {  // one line per round: start, seconds, jobs, attempts, resident / streaming / EA / other
                       // jobs, then seconds spent launching, on overlapped host work, and waiting
        int nr = 0, ns = 0, ne = 0, no = 0;
        long long att = 0;
        for (auto& j : act) {
          att += (long long)j->N * j->window * (j->ea ? 32 : 1);
          if (j->ea) ++ne; else if (j->cs > 0) ++nr; else if (j->streaming) ++ns; else ++no;
        }
        // then per path (resident, EA, streaming): the latest completion after the
        // round's start (ms) and the path's attempts; then the planned share of the SMs
        float tend[3] = {0, 0, 0};
        long long tatt[3] = {0, 0, 0};
        for (size_t k = 0; k < s->tmark.size(); ++k) {
          float ms = 0;
          if (cudaEventElapsedTime(&ms, s->tstart, s->tev[k]) == cudaSuccess)
            tend[s->tmark[k].first] = std::max(tend[s->tmark[k].first], ms);
          tatt[s->tmark[k].first] += s->tmark[k].second;
        }
        std::fprintf(s->trace, "%.4f %.4f %zu %lld %d %d %d %d %.4f %.4f %.4f %zu %.2f %lld %.2f %lld %.2f %lld %.3f\n", t0,
                     t1 - t0, act.size(), att, nr, ns, ne, no, t_launched - t0, t_host - t_launched, t1 - t_host,
                     admitted_now.size(), tend[0], tatt[0], tend[1], tatt[1], tend[2], tatt[2], s->fill);
        std::fflush(s->trace);
      }
    }
    std::vector<std::shared_ptr<Job>> still;
    for (auto& j : act) {
      if (rc != SPN_OK) {
        retire(s, j, rc, s->aux);
      } else if (j->done < j->req.nsweeps) {
        still.push_back(j);
      } else {
        completed.push_back(j);  // read back before the next round
      }
    }
    for (auto& j : joined) still.push_back(j);
    std::lock_guard<std::mutex> lock(s->mu);
    s->active = still;
  }
}

// The read-back thread: final E, M and host copies of finished jobs, one after
// another on the read-back stream, then their bytes back to the budget.
void reader(spn_server_ctx* s) {
  cudaSetDevice(s->device);
  while (true) {
    std::shared_ptr<Job> j;
    {
      std::unique_lock<std::mutex> lock(s->mu);
      s->rb_cv.wait(lock, [&] { return s->rb_stop || !s->rb_queue.empty(); });
      if (s->rb_queue.empty()) return;  // stopped and drained
      j = s->rb_queue.front();
      s->rb_queue.pop_front();
    }
    retire(s, j, SPN_OK, s->rb);
  }
}

}  // namespace

extern "C" {

int spn_server_create(spn_server* out, size_t hbm_budget_bytes) {
  if (!out || hbm_budget_bytes == 0) return sfail(SPN_E_ARG, "bad arguments");
  *out = nullptr;
  spn_server_ctx* s = new (std::nothrow) spn_server_ctx;
  if (!s) return sfail(SPN_E_NOMEM, "host allocation failed");
  s->budget = hbm_budget_bytes;
  cudaGetDevice(&s->device);
  if (cudaStreamCreateWithFlags(&s->main, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->aux, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->aux_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaMallocHost(&s->h_err, sizeof(int)) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaMalloc(&s->d_err, 4) != cudaSuccess || cudaMemset(s->d_err, 0, 4) != cudaSuccess) {
    delete s;
    return sfail(SPN_E_CUDA, "server set-up failed");
  }
  // the first half of the pool at the greatest priority: a round's cluster and
  // large-CTA launches go there, so the block scheduler places them first
  int prio_least = 0, prio_greatest = 0;
  cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
  if (cudaStreamCreateWithPriority(&s->rb, cudaStreamNonBlocking, prio_greatest) != cudaSuccess) {
    delete s;
    return sfail(SPN_E_CUDA, "server set-up failed");
  }
  for (int i = 0; i < kPoolStreams; ++i) {
    cudaStream_t st;
    cudaEvent_t ev;
    cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, i < kPoolStreams / 2 ? prio_greatest : prio_least);
    cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    s->pool.push_back(st);
    s->pool_done.push_back(ev);
  }
  if (const char* path = std::getenv("SPN_SERVER_TRACE")) s->trace = std::fopen(path, "w");
  s->worker = std::thread(scheduler, s);
  s->reader = std::thread(reader, s);
  *out = s;
  return SPN_OK;
}

int spn_submit(spn_server s, const spn_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket) return sfail(SPN_E_ARG, "NULL argument");
  auto j = std::make_shared<Job>();
  j->req = *req;
  j->req.betas = nullptr;
  j->req.couplings = nullptr;
  const int model = req->model;
  if (model != SPN_ISING2D && model != SPN_ISING3D && model != SPN_EA3D_PMJ)
    return sfail(SPN_E_ARG, "unknown model");
  j->nd = model == SPN_ISING2D ? 2 : 3;
  const int ext[3] = {req->dims[0], req->dims[1], j->nd == 3 ? req->dims[2] : 1};
  for (int d = 0; d < j->nd; ++d)
    if (ext[d] < 2 || (ext[d] & 1)) return sfail(SPN_E_ARG, "every extent must be even and >= 2");
  if (!spn::counter_range_ok(ext[0], ext[1], ext[2]))
    return sfail(SPN_E_ARG, "lattice too large for the random-number counter (more than 2^29 row words)");
  if (req->nsweeps < 1 || req->nsweeps > 0xffffffffLL) return sfail(SPN_E_ARG, "nsweeps must be >= 1");
  j->N = (int64_t)ext[0] * ext[1] * ext[2];
  if (model == SPN_EA3D_PMJ) {
    if (!req->betas || !req->couplings) return sfail(SPN_E_ARG, "EA requests need 32 betas and couplings");
    j->betas.assign(req->betas, req->betas + 32);
    const size_t nw = (size_t)((j->N + 63) / 64);
    j->bonds.assign(static_cast<const uint64_t*>(req->couplings), static_cast<const uint64_t*>(req->couplings) + 3 * nw);
  } else {
    if (!(req->beta >= 0.0)) return sfail(SPN_E_ARG, "beta must be >= 0");
    // lattices resident in the shared memory of one CTA or cluster share
    // persistent launches; larger ones stream from bit-packed lattices
    spn::Lattice g;
    g.nd = j->nd;
    g.Lx = ext[0];
    g.Ly = ext[1];
    g.Lz = ext[2];
    g.N = j->N;
    // the tallest dividing band (3D) whose bit-packed streaming geometry fits one CTA
    j->cs = spn::resident_cluster_size(j->nd, ext[0], ext[1], ext[2], spn::kMaxResidentCluster);
    for (int ty = j->nd == 3 ? 32 : 1; j->cs == 0 && j->N >= s->stream_sites && ty >= 1 && !j->streaming;
         ty -= (j->nd == 3 ? 2 : 1)) {
      if (j->nd == 3 && (ty < 2 || ext[1] % ty)) continue;
      if (!spn::stream_path_supported(g, ty, true)) continue;
      const int S = j->nd == 3 ? ext[2] : ext[1];
      const int tiles = j->nd == 3 ? ext[1] / ty : 1;
      // >= 32 slices a CTA: concurrent jobs fill the GPU, and few halo slices are re-read
      const int nseg = std::max(1, std::min(S / 32, 4 * spn::device_sm_count() / tiles));
      j->geo = spn::stream_geometry(g, ty, 0, nseg, true);
      j->streaming = spn::stream_geometry_ok(g, j->geo);
    }

  }
  j->bytes = job_bytes(*j);
  std::lock_guard<std::mutex> lock(s->mu);
  if (j->bytes > s->budget) return sfail(SPN_E_BUDGET, "the job alone exceeds the server's HBM budget");
  j->ticket = s->next_ticket++;
  j->t_submit = now_s();
  s->pending.push_back(j);
  s->all[j->ticket] = j;
  *ticket = j->ticket;
  s->cv.notify_one();
  return SPN_OK;
}

int spn_poll(spn_server s, uint64_t ticket, int* done, spn_result* out) {
  if (!s || !done) return sfail(SPN_E_ARG, "NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return sfail(SPN_E_NOTFOUND, "unknown ticket");
  const Job& j = *it->second;
  *done = j.state == kDone || j.state == kFailed;
  if (out) {
    std::memset(out, 0, sizeof *out);
    out->status = j.status;
    out->state = j.state;
    out->sweeps = j.done;
    if (j.state == kDone) {  // written by the scheduler before the state changes
      out->E = j.E;
      out->M = j.M;
    }
    out->t_submit = j.t_submit;
    out->t_admit = j.t_admit;
    out->t_done = j.t_done;
  }
  return SPN_OK;
}

int spn_server_fetch(spn_server s, uint64_t ticket, void* out, size_t bytes) {
  if (!s || !out) return sfail(SPN_E_ARG, "NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return sfail(SPN_E_NOTFOUND, "unknown ticket");
  Job& j = *it->second;
  if (j.state != kDone) return sfail(SPN_E_STATE, "the job is not done");
  if (j.req.model == SPN_EA3D_PMJ) {
    const size_t need = j.words.size() * 4 + 32;
    if (bytes != need) return sfail(SPN_E_ARG, "EA results are N uint32 words followed by 32 slot bytes");
    std::memcpy(out, j.words.data(), j.words.size() * 4);
    std::memcpy(static_cast<uint8_t*>(out) + j.words.size() * 4, j.slots.data(), 32);
  } else {
    if (bytes != j.spins.size()) return sfail(SPN_E_ARG, "bytes must be N");
    std::memcpy(out, j.spins.data(), bytes);
  }
  return SPN_OK;
}

int spn_server_stats(spn_server s, uint64_t* attempts, double* busy_seconds, uint64_t* rounds, size_t* used_bytes) {
  if (!s) return sfail(SPN_E_ARG, "NULL argument");
  std::lock_guard<std::mutex> lock(s->mu);
  if (attempts) *attempts = s->attempts.load();
  if (busy_seconds) *busy_seconds = s->busy;
  if (rounds) *rounds = s->rounds.load();
  if (used_bytes) *used_bytes = s->used;
  return SPN_OK;
}

int spn_server_destroy(spn_server s) {
  if (!s) return sfail(SPN_E_ARG, "NULL argument");
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
    s->pending.clear();
    s->cv.notify_one();
  }
  if (s->worker.joinable()) s->worker.join();
  {  // the scheduler has handed over its last finished jobs; the reader drains them
    std::lock_guard<std::mutex> lock(s->mu);
    s->rb_stop = true;
  }
  s->rb_cv.notify_one();
  if (s->reader.joinable()) s->reader.join();
  for (auto& kv : s->all) release(*kv.second, s->aux);
  cudaStreamSynchronize(s->main);
  cudaStreamSynchronize(s->aux);
  cudaStreamSynchronize(s->rb);
  for (size_t i = 0; i < s->pool.size(); ++i) {
    cudaStreamDestroy(s->pool[i]);
    cudaEventDestroy(s->pool_done[i]);
  }
  cudaFree(s->d_inst);
  cudaFree(s->d_ea);
  cudaFree(s->d_order);
  cudaFree(s->d_counters);
  cudaFree(s->d_tns);
  cudaFreeHost(s->h_tns);
  cudaFree(s->d_err);
  cudaEventDestroy(s->fork);
  cudaEventDestroy(s->aux_ev);
  cudaFreeHost(s->h_err);
  if (s->trace) std::fclose(s->trace);
  for (cudaEvent_t ev : s->tev) cudaEventDestroy(ev);
  if (s->tstart) cudaEventDestroy(s->tstart);
  cudaStreamDestroy(s->main);
  cudaStreamDestroy(s->aux);
  cudaStreamDestroy(s->rb);
  delete s;
  return SPN_OK;
}

}  // extern "C"
