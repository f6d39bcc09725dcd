// Internal declarations of libspn: handle layout, kernel parameter blocks and
// launchers shared by the translation units of the library.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "philox.cuh"

struct spn_ctx;  // the handle (global, as in spn.h)
struct EaBatch;  // forward: multi-spin coded EA batch (ea_msc.cu)

namespace spn {

// Metropolis thresholds of Eq. 2 for the classes q = dE / 4 = 1 .. 3: a move
// of class q is accepted iff u < t[q], or always when bit q of `always` is set
// (floor(exp(-beta dE) 2^32) = 2^32, beta ~ 0).
struct DevThr {
  uint32_t t[4];
  uint32_t always;
};

// floor(exp(-beta * dE) * 2^32) in [0, 2^32] (host, IEEE double).
uint64_t boltzmann_threshold(double beta, int dE);
DevThr make_thresholds(double beta);

// Kernel paths of a single lattice.
enum Path : int { kPathGeneric = 0, kPathStream = 1, kPathResident = 2, kPathPacked = 3 };

// Streaming-kernel geometry (stream.cu): TY rows per band (3D), R slices per
// step, nseg segments along the streamed axis, raw / bit slice buffers; packed:
// the lattice is stored as bit words (rows of packed_row_words(Lx) words).
struct StreamGeom {
  int packed;
  int wave;  // 1: the 2D band-parallel kernel (wave.cu), nseg row segments; 2: the 3D wavefront kernel (wave3.cu);
            // 3: the 2D band-parallel kernel on a bit-packed lattice (wave.cu); 4: the 3D wavefront kernel on a
            // bit-packed lattice (wave3.cu)
  int TY, R, nseg, threads, nraw, nbit;
  int roundsC, roundsA, roundsB, qcap;  // words per thread per phase; tie-queue entries per warp
  size_t smem;
};

struct Lattice {
  int nd = 2;
  int Lx = 0, Ly = 0, Lz = 1;
  int64_t N = 0;
  const uint8_t* bonds = nullptr;  // per-site byte, bit d set iff J(n, d) = -1 (null: J = +1)
  int pitch = 0;                   // streaming sweep only: bytes per row in memory (0: Lx, dense)
};

// A site's random planes come from the Philox counter whose first word is the
// 32-bit 8 g + call, g = j + ceil(Lx / 64) r the site's 64-site word of row r.
// Past 2^29 such words the first word would wrap and sites far apart would draw
// the same numbers, so no lattice holds more (this also keeps N <= 2^35).
constexpr int64_t kMaxRowWords = (int64_t)1 << 29;
inline bool counter_range_ok(int Lx, int Ly, int Lz) {
  return (int64_t)((Lx + 63) / 64) * Ly * Lz <= kMaxRowWords;
}

// Launchers (all asynchronous on `st`).  acc points at two int64 (dE, dM) that
// the sweep adds its accepted moves to; err is a device error word.
cudaError_t launch_init_hot(const Lattice& g, int8_t* s, uint64_t seed, uint32_t stream_id, cudaStream_t st);
cudaError_t launch_observables(const Lattice& g, const int8_t* s, unsigned long long* out2, int* bad, cudaStream_t st);
cudaError_t launch_sweep_generic(const Lattice& g, int8_t* s, const DevThr& T, const PhiloxKeys& K,
                                 uint32_t stream_id, uint32_t sweep, unsigned long long* acc, cudaStream_t st);
bool stream_path_supported(const Lattice& g, int TY, bool packed = false);
// Bit-packed storage: row r (= y + Ly z) holds W = ceil(Lx / 64) words of the
// even-x sites (bit i of word j: x = 64 j + 2 i, set iff the spin is -1), then W
// words of the odd-x sites (x = 64 j + 2 i + 1), then zero words up to a
// multiple of 4 words; bits beyond Lx are 0.
int packed_row_words(int Lx);
cudaError_t launch_pack(const Lattice& g, const int8_t* s, uint32_t* w, cudaStream_t st);
cudaError_t launch_unpack(const Lattice& g, const uint32_t* w, int8_t* s, cudaStream_t st);
// Double-checkerboard sweep (tiles Tx x Ty (x Tz), Tx a multiple of 64, an even
// number of tiles per axis, dense int8 lattice, no bonds): both tile parities
// of one sweep, `hits` updates of each colour per tile.
bool dc_supported(const Lattice& g, int Tx, int Ty, int Tz);
// the band-parallel form of the double checkerboard (dcwave.cu): 2D rows of >= 2048 sites in whole words, one hit
bool dcwave_supported(const Lattice& g, int Tx, int Ty, int hits);
int dcwave_default_segments(const Lattice& g, int hits);
cudaError_t launch_sweep_dcwave(const Lattice& g, const int8_t* in, int8_t* out, int Tx, int Ty, int hits, int nseg,
                                const DevThr& T, const PhiloxKeys& K, uint32_t stream_id, uint32_t sweep,
                                unsigned long long* acc, int* err, cudaStream_t st, uint32_t expire_polls = 0);
cudaError_t launch_sweep_dc(const Lattice& g, int8_t* s, int Tx, int Ty, int Tz, int hits, const DevThr& T,
                            const PhiloxKeys& K, uint32_t stream_id, uint32_t sweep, unsigned long long* acc,
                            cudaStream_t st);
// Band-parallel sweep (wave.cu): 2D int8 lattices whose Lx is a multiple of 64
// and at least 2048, dense rows, no bonds; a warp per (band of 30 words, segment
// of rows), nseg segments.
bool wave_supported(const Lattice& g);
int wave_default_segments(const Lattice& g);
size_t wave_smem_bytes(const Lattice& g);
bool wave_packed_supported(const Lattice& g);
size_t wave_packed_smem_bytes();
cudaError_t launch_sweep_wave_packed(const Lattice& g, const uint32_t* in, uint32_t* out, int nseg, const DevThr& T,
                                     const PhiloxKeys& K, uint32_t stream_id, uint32_t sweep,
                                     unsigned long long* acc, cudaStream_t st);
int wave_cta_threads();
cudaError_t launch_sweep_wave(const Lattice& g, const int8_t* in, int8_t* out, int nseg, const DevThr& T,
                              const PhiloxKeys& K, uint32_t stream_id, uint32_t sweep, unsigned long long* acc,
                              int* err, cudaStream_t st, uint32_t expire_polls);
// Wavefront 3D sweep (wave3.cu): int8 lattices with Lx = 64, 128, 256 or 512,
// dense rows, no bonds, band height TY a multiple of 32 / (Lx / 64) with at most
// eight compute warps, dividing Ly; nseg segments along z.
bool wave3_supported(const Lattice& g, int TY);
int wave3_default_segments(const Lattice& g, int TY, bool packed = false);
size_t wave3_smem_bytes(const Lattice& g, int TY, bool packed = false);  // of one CTA
int wave3_cta_threads(const Lattice& g, int TY, bool packed = false);
cudaError_t launch_sweep_wave3(const Lattice& g, const int8_t* in, int8_t* out, int TY, int nseg, const DevThr& T,
                               const PhiloxKeys& K, uint32_t stream_id, uint32_t sweep, unsigned long long* acc,
                               int* err, cudaStream_t st, uint32_t expire_polls);
cudaError_t launch_sweep_wave3_packed(const Lattice& g, const uint32_t* in, uint32_t* out, int TY, int nseg,
                                      const DevThr& T, const PhiloxKeys& K, uint32_t stream_id, uint32_t sweep,
                                      unsigned long long* acc, int* err, cudaStream_t st);
StreamGeom stream_geometry(const Lattice& g, int TY, int R, int nseg, bool packed = false);
bool stream_geometry_ok(const Lattice& g, const StreamGeom& geo);
// expire_polls (test support, 0 otherwise): the copy of each CTA's first slice
// is never issued and every bounded wait of the launch gives up after that many
// polls, so the launch reports a timeout without any device fault.
cudaError_t launch_sweep_stream(const Lattice& g, const void* in, void* out, const StreamGeom& geo,
                                const DevThr& T, const PhiloxKeys& K, uint32_t stream_id, uint32_t sweep,
                                unsigned long long* acc, int* err, cudaStream_t st, uint32_t expire_polls = 0);

// One instance of a batched resident run (batched.cu).
struct ResInst {
  int8_t* spins;               // device int8 lattice, result written back
  unsigned long long* trace;   // [nsweeps][2] per-sweep (dE, dM), zeroed by the caller; may be null
  unsigned long long* em0;     // [2] start (E, M), zeroed by the caller; may be null
  uint64_t seed;
  uint32_t stream;
  uint32_t sweep0;
  int nsweeps;
  int init_hot;                // 1: hot start from Philox; 0: start from `spins`
  int Lx, Ly, Lz;              // extents (Lz = 1 in 2D); the launch's shared memory fits the largest
  DevThr T;
  unsigned long long* tns;     // [2] device clock (ns) at the instance's start and end; may be null
};

struct ResArgs {
  const ResInst* inst;  // all instances of one launch share nd and the cluster size
  int ninst;
  const int* order;     // queue order (longest first)
  int* counter;         // queue head, zeroed by the caller
  int* err;
  // set by a caller that knows no instance has a class with dE > 0 that is
  // always accepted (DevThr.always & 14 == 0): the kernel is then compiled
  // without that test; left false, the general kernel runs
  bool no_always;
};

// true iff no class with dE > 0 of these thresholds is always accepted
inline bool no_always_class(const DevThr& T) { return (T.always & 14u) == 0; }

bool resident_supported(int nd, int Lx, int Ly, int Lz, int cs);
size_t resident_smem(int nd, int Lx, int Ly, int Lz, int cs);
constexpr int kMaxResidentCluster = 16;  // 9 .. 16: non-portable cluster sizes
// smallest cluster size (1, 2, 4, ..., max_cs) whose CTAs hold the lattice; 0: none
int resident_cluster_size(int nd, int Lx, int Ly, int Lz, int max_cs = 8);
int resident_max_ctas(int nd, int cs, int threads, size_t smem);  // CTAs resident at once (whole clusters)
cudaError_t launch_resident(const ResArgs& a, int nd, int cs, int threads, int ctas, size_t smem, cudaStream_t st);

int device_sm_count();
void count_launches(uint64_t n);
void set_last_error(const char* msg);  // the thread's spn_last_error() message
uint64_t launch_count();

}  // namespace spn

namespace spn {

// Exact division by a launch-invariant 32-bit divisor (Granlund-Montgomery
// round-up method): q = (t + ((n - t) >> 1)) >> s with t = umulhi(n, m).
struct FastDiv {
  uint32_t d, m, s;
};

struct EaArgs {
  uint64_t* words;            // [pairs][N] uint64
  const uint8_t* bonds;       // [S][N] bond bytes (site order)
  uint8_t* temp_of_slot;      // [S][32]
  unsigned long long* xacc;   // [S][32] accepted exchanges per pair
  const uint32_t* xtab;       // concatenated exchange tables
  int xoff[32];               // offset of pair k's table in xtab
  int xlen[32];               // its length (d = 1 .. xlen), 0 with xalways[k]
  uint32_t xalways;           // bit k: pair k has equal betas (always accept)
  uint32_t thr[3][32];        // thr[q-1][t] for dE = 4q, non-decreasing in t
  int nd;                     // 2: square lattice (Lz = 1), 3: simple cubic
  int Lx, Ly, Lz, N;
  FastDiv div_h, div_ly;      // by Lx / 2 and by Ly
  uint32_t sweep0;
  int nsweeps;
  int exchange_every;
  int nsamples;
  int u_per_slot;             // 1: every temperature slot draws its own u (32 bit planes per site)
  PhiloxKeys K;
  int* err;
};

// Disorder-parallel EA batches (ea_dp.cu): word lattice 32 g + t holds the 32
// samples of group g at temperature t, N uint32 words in colour-separated row
// order; bonds [g][d][N] words (bit j: J(n, d) = -1 for sample j of the group).
struct EaDpArgs {
  uint32_t* dp;          // [32 ngroups][N]
  const uint32_t* bdp;   // [ngroups][nd][N]
  uint32_t* U;           // [32 ngroups][32] unsatisfied forward bonds per sample (need_u)
  int nd, Lx, Ly, Lz, N;
  FastDiv div_h, div_ly;  // by Lx / 2 and by Ly
  uint32_t sweep0;
  int nsweeps;
  int need_u;             // count unsatisfied bonds after the last sweep (an exchange follows)
  uint32_t thr[32][3];    // thr[t][lv] for dE = 4 (lv + 1), beta of temperature t
  PhiloxKeys K;
};
struct EaDpExchangeArgs {
  const uint32_t* U;
  uint32_t* X;                // [ngroups][32] swap masks of the step's pairs (k, k + 1)
  unsigned long long* xacc;   // [nsamples][32]
  const uint32_t* xtab;
  int xoff[32], xlen[32];
  uint32_t xalways;
  int nsamples;
  uint32_t e;                 // exchange step
  PhiloxKeys K;
};
size_t dp_smem(int N);
cudaError_t launch_dp_from_words(const uint64_t* pairs, uint32_t* dp, int Lx, int N, int nsamples, int ngroups,
                                 cudaStream_t st);
cudaError_t launch_dp_to_words(const uint32_t* dp, uint64_t* pairs, int Lx, int N, int nsamples, int ngroups,
                               cudaStream_t st);
cudaError_t launch_dp_bonds(const uint64_t* packed, uint32_t* bdp, int nd, int Lx, int N, int nsamples, int ngroups,
                            cudaStream_t st);
cudaError_t launch_dp_sweep(const EaDpArgs& a, int nwl, int threads, cudaStream_t st);
cudaError_t launch_dp_exchange(const EaDpExchangeArgs& a, int ngroups, cudaStream_t st);
cudaError_t launch_dp_swap(uint32_t* dp, const uint32_t* X, int N, int ngroups, cudaStream_t st);

// Served multi-spin coded EA jobs (single-sample batch handles): the
// parameter block of the next `nsweeps` sweeps of h (its sweep counter
// advances), and one launch running many such blocks, one CTA each.
int ea_window_args(struct spn_ctx* h, int64_t nsweeps, EaArgs* out, size_t* smem, int* threads);
int ea_job_per_sm(struct spn_ctx* h);  // CTAs of a one-sample EA handle's job kernel resident per SM
cudaError_t launch_ea_jobs(const EaArgs* d_list, int n, int nd, bool ps, int threads, size_t smem, cudaStream_t st);
// Server admissions of single-sample EA batches in two parts: the host part
// (validation, bond bytes, exchange tables; no CUDA call, any thread) and the
// device part, whose allocations, copies and hot start are ordered on st and
// never wait for the device (the handle's stream is st).
struct EaPrep {
  int model = 0;
  struct ::EaBatch* b = nullptr;  // host fields filled; owned until uploaded
  std::vector<uint8_t> bb;         // per-site bond bytes
  std::vector<uint32_t> tab;       // exchange tables
  ~EaPrep();
};
int ea_prepare_single(EaPrep& p, int model, const int32_t* dims, const void* couplings, const double* betas,
                      uint64_t seed, int exchange_every);
int ea_upload_async(struct ::spn_ctx** out, EaPrep& p, cudaStream_t st);

}  // namespace spn

struct EaBatch;                // multi-spin coded EA batch (ea_msc.cu)
void spn_ea_free(EaBatch* b);
struct HeisState;              // Heisenberg lattice of a handle (heis.cu)

namespace spn {
// Heisenberg handles: model SPN_HEIS2D / SPN_HEIS3D; dims checked there.
bool is_heis_model(int model);
bool heis_dims_ok(int nd, const int32_t* dims);
int heis_create(::spn_ctx* h, const int32_t* dims, int init);
int heis_sweep(::spn_ctx* h, double beta, int64_t nsweeps);
int heis_reinit(::spn_ctx* h, int init);
void heis_free(HeisState* s);
cudaError_t launch_heis_init(float4* s, int nd, const int* L, int64_t N, uint64_t seed, uint32_t stream, bool cold,
                             cudaStream_t st);
cudaError_t launch_heis_sweep(float4* s, int nd, const int* L, int64_t N, float beta, uint64_t seed,
                              uint32_t stream, uint32_t sweep, unsigned long long* acc, unsigned long long* work,
                              unsigned long long* work_base, cudaStream_t st);
cudaError_t launch_heis_observables(const float4* s, int nd, const int* L, int64_t N, double* out4,
                                    cudaStream_t st);
cudaError_t launch_heis_exp(const float* x, float* y, int n, cudaStream_t st);
}  // namespace spn

struct spn_ctx {
  int model = 0;
  EaBatch* ea = nullptr;  // set for batch handles (spn_create_batch)
  HeisState* heis = nullptr;  // set for Heisenberg handles
  spn::Lattice g;
  uint64_t seed = 0;
  uint32_t stream_id = 0;
  uint32_t expire_polls = 0;  // test support: the next streaming launch of this handle gives up its waits
  int8_t* spins[2] = {nullptr, nullptr};
  int cur = 0;
  // streaming sweep of a lattice whose Lx is not a multiple of 64: the lattice
  // is staged into rows padded to 64 bytes for the sweeps of one spn_sweep call
  int8_t* staged[2] = {nullptr, nullptr};
  // bit-packed path: the lattice lives in packed[pcur] while packed_live (the
  // int8 buffer is then stale until the next call that needs it)
  uint32_t* packed[2] = {nullptr, nullptr};
  int pcur = 0;
  bool packed_live = false;
  uint8_t* d_bonds = nullptr;
  cudaStream_t st = nullptr;
  int path = spn::kPathGeneric;
  int tile_y = 0, step_slices = 0, seg = 0;
  uint64_t sweeps = 0;
  // incremental bookkeeping: device deltas (dE, dM) per sweep since `folded`
  unsigned long long* d_acc = nullptr;
  int64_t acc_cap = 0;
  uint64_t folded = 0;  // sweeps already folded into the host trace
  int64_t E = 0, M = 0;  // observables after `folded` sweeps
  std::vector<int64_t> traceE, traceM;
  int* d_err = nullptr;
  int* d_bad = nullptr;
  unsigned long long* d_obs = nullptr;
  // resident path: the one-instance work list of the persistent kernel
  spn::ResInst* d_res = nullptr;
  int* d_resq = nullptr;  // [0] queue order (0), [1] queue head
};
