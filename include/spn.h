/*
 * spn.h -- C ABI of libspn, checkerboard Metropolis sweeps of nearest-neighbour
 * Ising-type lattices on one NVIDIA GB300 (sm_103a).
 *
 * The method is the single-spin-flip Metropolis simulation of the Ising model
 * (M. Weigel, "Simulating spin models on GPU", Sec. 3): Hamiltonian Eq. 1,
 * H = -J sum_<ij> s_i s_j with s_i = +-1 on square (2D) and simple-cubic (3D)
 * lattices with periodic boundaries; acceptance Eq. 2, p = min[1, exp(-beta dE)];
 * the two sub-lattices of the checkerboard decomposition are updated one after
 * the other because the sites of one colour are independent.  Sec. 4 extends it
 * to the 3D model and to the +-J Edwards-Anderson spin glass with many disorder
 * samples multi-spin coded into machine words.
 *
 * Conventions shared by every entry point
 *   - Return value: SPN_OK (0) on success, a negative SPN_E_* code on failure.
 *     spn_last_error() gives a message for the calling thread's last failure.
 *     No C++ exception crosses this boundary.
 *   - dims: int32[2] (2D) or int32[3] (3D), x fastest; every extent even, >= 2.
 *     Site n = x + Lx*(y + Ly*z); colour c(n) = (x+y+z) & 1; m = n >> 1.
 *     An Ising or EA lattice holds at most 2^29 row words, ceil(Lx / 64) * Ly
 *     * Lz <= 2^29 (so N <= 2^35), because 8 g + q / 4 below is one 32-bit
 *     counter word; spn_create(_ex), spn_multi_create and spn_submit refuse a
 *     larger one with SPN_E_ARG before any device work.  An extent of 2 is
 *     allowed, but there each pair of sites is joined by two bonds, and with
 *     +-J couplings the checkerboard chain can then be reducible (averages that
 *     depend on the start); extents >= 4 avoid it.
 *   - Spins on the host are int8 +-1 in site order.  Couplings ("bonds") are
 *     bit-packed uint64 words [sample][dir][ceil(N/64)], bit (n % 64) of word
 *     n / 64 set iff J(n, dir) = -1 for the bond from n to n + e_dir.
 *   - Memory: the library owns every device buffer it allocates; host buffers
 *     passed in are read (or written) during the call only.  The device-pointer
 *     entry point spn_sweep_noalloc never allocates and never frees.
 *   - Randomness: Philox4x32-10 keyed by the 64-bit seed.  Each row of the
 *     lattice is cut into 64-site words; the sites of one colour in word j of
 *     row r = y + Ly z form group g = j + ceil(Lx / 64) r, site x at lane
 *     (x & 63) >> 1.  Plane q (0..31) of a group is word q & 3 of
 *     R(8 g + q / 4, sweep, colour | purpose << 1, stream); bit 31 - q of a
 *     site's 32-bit number is its lane's bit of plane q (purpose 0: Metropolis,
 *     1: hot start, which takes bit 31 as "spin -1").  A move with dE > 0 is
 *     accepted iff u < floor(exp(-beta dE) * 2^32) (Eq. 2).  The multi-spin
 *     coded EA sweep of a batch with replica exchange gives every temperature
 *     slot j of the site with within-colour index m its own u: bit 31 - p of
 *     it is bit j of plane p = word p & 3 of R(m, sweep, colour | 3 << 1 |
 *     (p / 4 + 1) << 4, sample).  A batch without exchange (or one switched by
 *     spn_batch_set_u_per_slot(h, 0)) shares one u per site among the slots:
 *     word m & 3 of R(m >> 2, sweep, colour | 3 << 1, sample).  Replica
 *     exchange uses word k & 3 of R(k >> 2, step, 2 << 1, sample).  Results
 *     are bit-identical for a given (seed, stream, sweep index, beta) on every
 *     path.
 *   - A handle is not thread-safe; a server is.
 */
#ifndef SPN_H
#define SPN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum spn_status {
  SPN_OK = 0,
  SPN_E_ARG = -1,      /* invalid argument (null pointer, odd extent, wrong size ...) */
  SPN_E_NOMEM = -2,    /* device or host allocation failed */
  SPN_E_BUDGET = -3,   /* a served job does not fit the server's HBM budget */
  SPN_E_CUDA = -4,     /* a CUDA runtime call failed (message in spn_last_error) */
  SPN_E_TIMEOUT = -5,  /* a bounded device wait ran out (no hang, state preserved) */
  SPN_E_STATE = -6,    /* call not valid for this handle's model or state */
  SPN_E_NOTFOUND = -7  /* unknown ticket */
};

enum spn_model {
  SPN_ISING2D = 1,   /* square lattice, J = +1 (Eq. 1) */
  SPN_ISING3D = 2,   /* simple cubic, J = +1 (Sec. 4) */
  SPN_EA3D_PMJ = 3,  /* simple cubic, J = +-1 per bond (Sec. 4, spin glass) */
  SPN_EA2D_PMJ = 4,  /* square lattice, J = +-1 per bond (batches only: spn_create_batch) */
  SPN_HEIS2D = 5,    /* square lattice, classical Heisenberg (O(3)) spins, J = +1 (Sec. 4 outlook) */
  SPN_HEIS3D = 6     /* simple cubic, classical Heisenberg spins */
};

enum spn_init { SPN_INIT_HOT = 0, SPN_INIT_COLD = 1 };

typedef struct spn_ctx* spn_handle;

/* Thread-local message of the last failure on this thread ("" if none). */
const char* spn_last_error(void);

/* Library version string and the device it runs on (prints nothing). */
const char* spn_version(void);

/* ------------------------------------------------------------------------
 * Single lattice (Sec. 3 procedure; Eq. 1-2)
 * ---------------------------------------------------------------------- */

/* Create a lattice of `model` with extents `dims`, hot start from Philox
 * (stream 0).  couplings: NULL for the Ising models; for SPN_EA3D_PMJ one
 * sample of bit-packed bonds [3][ceil(N/64)] (copied).  Errors: SPN_E_ARG for
 * odd/too small extents, a lattice past the counter range (above), or a
 * missing/unexpected coupling array, SPN_E_NOMEM, SPN_E_CUDA. */
int spn_create(spn_handle* out, int model, const int32_t* dims, const void* couplings, uint64_t seed);

/* As spn_create with an explicit Philox stream id and start (SPN_INIT_HOT or
 * SPN_INIT_COLD = all +1). */
int spn_create_ex(spn_handle* out, int model, const int32_t* dims, const void* couplings, uint64_t seed,
                  uint32_t stream, int init);

/* Run nsweeps sweeps at inverse temperature beta >= 0 (may be +inf) on the
 * handle's stream, asynchronously.  Sweep k of the handle's life uses sweep
 * counter k.  Each sweep updates colour 0, then colour 1 (Sec. 3); energy and
 * magnetisation change by the accepted moves and are recorded per sweep. */
int spn_sweep(spn_handle h, double beta, int64_t nsweeps);

/* Current integer energy E = -sum J s_i s_j (Eq. 1, each bond once) and
 * magnetisation M = sum s_i (synchronises the handle's stream). */
/* The paper's own update order (Sec. 3): the double-checkerboard sweep with
 * the generalised multi-hit.  The lattice is cut into tiles of
 * tile[0] x tile[1] (x tile[2]) sites, tile[0] a multiple of 64 and an even
 * number of tiles along every axis; a sweep takes the tiles of even, then odd
 * tile parity, and in each updates the colour-0 sites, then the colour-1 sites,
 * `hits` times over.  Random numbers are the bit-plane words of purpose 4 at
 * counter sweep * hits + hit.  Each call appends nsweeps entries to the trace
 * and advances the sweep counter like spn_sweep.  Ising lattices without bonds
 * whose Lx is a multiple of 64; SPN_E_ARG otherwise. */
int spn_sweep_dc(spn_handle h, double beta, int64_t nsweeps, const int32_t* tile, int32_t hits);

int spn_observables(spn_handle h, int64_t* E, int64_t* M);

/* Recompute E and M from the spins with a full reduction (independent of the
 * incremental bookkeeping; synchronises). */
int spn_recompute(spn_handle h, int64_t* E, int64_t* M);

/* Per-sweep trace of (E, M) after every sweep since creation, oldest first:
 * writes min(cap, total) entries and the total count to *n (synchronises). */
int spn_trace(spn_handle h, int64_t* E, int64_t* M, int64_t cap, int64_t* n);

/* Copy the spins (int8 +-1, site order) into host_out; bytes must be N. */
int spn_get_spins(spn_handle h, int8_t* host_out, size_t bytes);

/* Replace the spins from a host buffer of N int8 +-1 values (pinned memory
 * makes the copy asynchronous-fast); E and M are recomputed on the device, which
 * also rejects values other than +-1 with SPN_E_ARG.  The sweep counter is
 * kept. */
int spn_set_spins(spn_handle h, const int8_t* host_in, size_t bytes);

/* Start a new run on the same handle: re-initialise the spins (hot start from
 * Philox with the given seed and stream, or cold), reset the sweep counter to
 * 0 and clear the trace.  Device memory is reused (no allocation). */
int spn_reinit(spn_handle h, uint64_t seed, uint32_t stream, int init);

/* Number of sweeps done so far (the next sweep's counter). */
int spn_sweep_count(spn_handle h, uint64_t* count);

/* Make the handle use an existing CUDA stream (cudaStream_t as void*; NULL =
 * the legacy default stream).  The caller keeps ownership of the stream. */
int spn_set_stream(spn_handle h, void* cuda_stream);

/* Wait for the handle's queued work. */
int spn_sync(spn_handle h);

/* Release the handle and its device memory (synchronises first). */
int spn_destroy(spn_handle h);

/* Geometry of the streaming sweep kernel for this handle: tile_y = rows per
 * band in 3D (divides Ly; ignored in 2D), step_slices = slices (2D rows, 3D
 * planes) advanced per pipeline step (0 = automatic), seg = number of segments
 * the streamed axis is cut into, one CTA each per band (0 = automatic).  The
 * results never depend on it.  SPN_E_ARG if it does not fit one CTA. */
int spn_set_tiling(spn_handle h, int32_t tile_y, int32_t step_slices, int32_t seg);

/* Autotuner of the streaming sweep (Sec. 4 tunes its tile to L): for the
 * handle's streaming path (1 or 3), time every fitting combination of band
 * height (3D: even divisors of Ly up to 32), slices per step (automatic, 1, 2,
 * 4) and segment count (automatic, or 2, 4, 6, 8 CTAs per SM) on trial_sweeps
 * sweeps of a scratch copy of the lattice at beta, and set the fastest as the
 * handle's tiling (the default tiling, timed first, is replaced only by one
 * more than 1% faster).  The handle's spins, counters and trace are untouched and
 * results never depend on the tiling.  Choices are cached per (shape, path,
 * device) for the process.  chosen (optional, 3 ints): tile_y, step_slices,
 * seg as for spn_set_tiling.  SPN_E_STATE if the handle is not on a streaming
 * path. */
int spn_autotune(spn_handle h, double beta, int32_t trial_sweeps, int32_t* chosen);

/* Which kernel path the handle uses: 0 = generic global-memory sweep,
 * 1 = streaming shared-memory sweep, 2 = shared-memory-resident sweep,
 * 3 = bit-packed streaming sweep.  Path 3 keeps the lattice in HBM as one bit
 * per spin between sweeps (row r = y + Ly z: ceil(Lx/64) words of the even-x
 * sites, as many of the odd-x sites, zero words up to a multiple of 4; a set
 * bit is spin -1); spn_sweep packs the int8 lattice on entry when needed, and
 * the calls that read spins (spn_get_spins, spn_recompute, the other paths)
 * unpack it first.  Path 2 runs every sweep of one spn_sweep call in a single
 * launch, the lattice held as bits in the shared memory of one CTA or of a
 * cluster of up to 8 (at most 200 KB each, Ising only); it is the default for
 * lattices of at most 65536 sites that fit one CTA, path 1 for larger ones.
 * Results never depend on the path.  spn_set_path fails with SPN_E_ARG if the
 * path does not support the lattice (bonds, a band that does not divide Ly, a
 * lattice too large for path 2). */
int spn_get_path(spn_handle h, int32_t* path);
int spn_set_path(spn_handle h, int32_t path);

/* Number of kernels this library has launched in the process so far (all
 * handles); a diagnostic for benchmarks. */
int spn_launch_count(uint64_t* count);

/* ------------------------------------------------------------------------
 * Classical Heisenberg spins (the continuous-spin generalisation Sec. 4 names
 * for single-precision GPU arithmetic): H = -sum_<ij> S_i . S_j, |S| = 1.
 * spn_create_ex(model SPN_HEIS2D / SPN_HEIS3D, couplings NULL) makes the
 * handle (dims even, N < 2^31; hot start: every site a uniform direction, cold
 * start: all (0, 0, 1)); spn_sweep, spn_reinit, spn_sweep_count,
 * spn_set_stream, spn_sync and spn_destroy work on it, the int8 calls return
 * SPN_E_STATE.  A sweep updates colour 0, then colour 1: a site proposes a
 * direction uniform on the sphere (Marsaglia's method) and takes it iff
 * dE = -(S' - S) . h <= 0 or u < exp(-beta dE), h the sum of its neighbours.
 * Spins are binary32; every step is a correctly rounded binary32 operation in
 * a fixed order and exp is Cody-Waite reduction plus a degree-7 Taylor
 * polynomial of those operations, so lattices are reproducible bit for bit;
 * beta is rounded to binary32.  Random words (Philox, key = seed): proposal
 * call k = 0..7 is R(m, sweep, c | 5 << 1 | k << 4, stream), m = n >> 1,
 * tries 2k and 2k+1 from words (0, 1) and (2, 3), a word w giving
 * (w >> 8) 2^-23 - 1; no move after 16 failed tries; the hot start uses
 * purpose 7 with sweep 0; u = (w >> 8) 2^-24 with w = word m & 3 of
 * R(m >> 2, sweep, c | 6 << 1, stream).  E and M start from a binary64
 * recompute and add, per sweep, the exact sum of the accepted moves' binary32
 * dE and dS each rounded to a multiple of 2^-40 (so they are reproducible).
 * ---------------------------------------------------------------------- */

/* Spins as binary32 [N][3] (x, y, z) in site order; count = 3 N.  Set copies
 * the vectors as given (callers pass unit vectors) and recomputes E and M. */
int spn_heis_get_spins(spn_handle h, float* xyz, size_t count);
int spn_heis_set_spins(spn_handle h, const float* xyz, size_t count);

/* E and M[3] after the sweeps so far (synchronises). */
int spn_heis_observables(spn_handle h, double* E, double* M);

/* E = -sum_n sum_d S_n . S_{n+e_d} and M recomputed from the spins on the
 * device in binary64. */
int spn_heis_recompute(spn_handle h, double* E, double* M);

/* Per-sweep trace: E[s], M[3 s + i] after sweep s; *n = sweeps so far. */
int spn_heis_trace(spn_handle h, double* E, double* M, int64_t cap, int64_t* n);

/* Test support: the device exp of the acceptance on n host floats. */
int spn_test_heis_exp(const float* x, float* y, size_t n);

/* ------------------------------------------------------------------------
 * Batched runs of many independent lattices (uneven sizes, temperatures and
 * sweep counts; Sec. 3 procedure for each)
 * ---------------------------------------------------------------------- */

/* One lattice of a batched run: model SPN_ISING2D or SPN_ISING3D, extents
 * dims (dims[2] ignored in 2D), inverse temperature beta >= 0, nsweeps sweeps
 * from the hot start of Philox (seed, stream). */
typedef struct spn_job {
  int32_t model;
  int32_t dims[3];
  double beta;
  int64_t nsweeps;
  uint64_t seed;
  uint32_t stream;
  int32_t reserved; /* 0 */
} spn_job;

typedef struct spn_multi_ctx* spn_multi;

enum spn_run_mode {
  SPN_RUN_BATCHED = 0, /* one persistent resident launch per lattice shape, all shapes concurrent, CUDA graph */
  SPN_RUN_LOOP = 1     /* the plain per-instance launch loop (one launch per sweep) */
};

/* Allocate the lattices and traces of njobs jobs (copied).  Every lattice must
 * fit the resident kernel: its bits (2 ceil(Lx / 64) words per row) in a cluster
 * of at most 8 CTAs x 200 KB, the rows split among the cluster's CTAs;
 * SPN_E_ARG otherwise. */
int spn_multi_create(spn_multi* out, const spn_job* jobs, int njobs);

/* Run every job from its hot start (asynchronous on the run's stream).  Both
 * modes give bit-identical lattices and traces; the first batched run captures
 * a CUDA graph that later runs replay. */
int spn_multi_run(spn_multi m, int mode);

/* Wait for the run; SPN_E_TIMEOUT if a bounded device wait ran out. */
int spn_multi_sync(spn_multi m);

/* Result of job `job` after a run (synchronises): its int8 lattice (bytes =
 * N, or spins = NULL) and E, M after each of its first min(cap, nsweeps)
 * sweeps (or E = M = NULL). */
int spn_multi_result(spn_multi m, int job, int8_t* spins, size_t bytes, int64_t* E, int64_t* M, int64_t cap);

/* Use an existing CUDA stream for the runs (the graph is captured again). */
int spn_multi_set_stream(spn_multi m, void* cuda_stream);

/* Autotuner of the batched run (Sec. 4 observes that the best tile depends on
 * L).  A trial runs the whole batch at reduced length (every job from its hot
 * start, its sweeps scaled so that the longest job has trial_sweeps) with all
 * lattice shapes launched together, as in a real run.  Starting from the
 * current launch shapes, each lattice shape in turn tries every cluster size
 * (CTAs sharing one lattice: 1, 2, 4 or 8 that fit) and thread count (64 ..
 * 512) and keeps the one with the fastest trial (a change must win by 1%).
 * Results never depend on the launch shape.  The choice is remembered per
 * (shape, device) for the process, so later batches start from it.  rates
 * (optional, count = number of shapes): the batch's trial attempts/ns after
 * each shape was tuned.  Synchronises; the next SPN_RUN_BATCHED run captures
 * a new graph. */
int spn_multi_autotune(spn_multi m, int32_t trial_sweeps, double* rates, size_t count);

/* Launch shapes, 7 ints per lattice shape (in the batch's own order): nd, Lx,
 * Ly, Lz, cluster size, threads per CTA, CTAs of the launch.  count = 7 x the
 * number of shapes. */
int spn_multi_groups(spn_multi m, int32_t* out, size_t count);

/* Set the launch shape of lattice shape `group` by hand (cluster size 1, 2, 4
 * or 8 that fits, threads a multiple of 32 up to 512); SPN_E_ARG otherwise. */
int spn_multi_set_launch(spn_multi m, int32_t group, int32_t cs, int32_t threads);

int spn_multi_destroy(spn_multi m);

/* ------------------------------------------------------------------------
 * Batched +-J Edwards-Anderson samples, multi-spin coded, with replica
 * exchange (Sec. 4: many disorder realisations at once, asynchronous
 * multi-spin coding; the exchange rule is Hukushima-Nemoto parallel tempering)
 * ---------------------------------------------------------------------- */

/* Create a batch of nsamples +-J samples, simple cubic (SPN_EA3D_PMJ, dims
 * int32[3]) or square (SPN_EA2D_PMJ, dims int32[2]), of extents dims, each
 * holding 32 replicas at the 32 inverse temperatures betas
 * (nbeta = 32, non-increasing, i.e. ascending temperature, each >= 1e-6).
 * Replica j of sample i lives in bit j (its temperature slot) of the sample's
 * 32-bit site words; on the device two samples share one uint64 word (64
 * replicas per word).  couplings: bit-packed bonds [sample][d][ceil(N/64)], d = 3 or 2
 * (copied).  The replica bits start from the hot-start words of Philox stream
 * i; slot j starts at temperature j.  exchange_every = X > 0 exchanges the
 * temperature pairs (k, k+1), k = e mod 2, e mod 2 + 2, ..., after every X-th
 * sweep (step e), accepting iff (beta_k - beta_k+1)(E_k - E_k+1) >= 0 or
 * u < floor(exp(that) 2^32); 0 = never.  A sample must fit one CTA's shared
 * memory (5 bytes per site, about 44,000 sites: L <= 34).  SPN_E_ARG otherwise. */
int spn_create_batch(spn_handle* out, int model, const int32_t* dims, int nsamples, const void* couplings,
                     const double* betas, int nbeta, uint64_t seed, int exchange_every);

/* A batch in the disorder-parallel layout (Sec. 4: many disorder realisations
 * at once with asynchronous multi-spin coding, the bits of a word being
 * different samples).  Same arguments and results as spn_create_batch, but
 * Lx must be a multiple of 8 (SPN_E_ARG otherwise), and the device keeps one
 * 32-bit word per (site, temperature, group of 32 samples): sample s belongs to
 * group g = 2 (s >> 6) + (s & 1) (so the replicas 2p and 2p + 1 of a
 * realisation never share a word) and the samples of a group share the
 * Metropolis u of the site at each temperature t: word m & 3 of
 * R(m >> 2, sweep, colour | 3 << 1, 32 g + t) for within-colour index m.  A
 * sample's 32 temperatures draw independent numbers, so the ladder is exact
 * under replica exchange, and a word lattice has one temperature, so the
 * acceptance is a scalar compare per site.  Replica exchange swaps the two
 * configurations of an accepted pair (u as in spn_create_batch), so the slot
 * map stays the identity: bit t of a sample's word is always temperature t.
 * spn_batch_* calls work on it as on any batch, except
 * spn_batch_set_u_per_slot (SPN_E_STATE) and spn_batch_set_slots, which
 * accepts only identity maps.  Reading words, energies or overlaps converts
 * the word lattices on the device first. */
int spn_create_batch_dp(spn_handle* out, int model, const int32_t* dims, int nsamples, const void* couplings,
                        const double* betas, int nbeta, uint64_t seed, int exchange_every);

/* Run nsweeps multi-spin coded sweeps (colour 0, then colour 1) with the
 * exchanges due; every slot draws its own u, or the 32 replicas of a site share
 * its Philox word, as spn_batch_set_u_per_slot says. */
int spn_batch_sweep(spn_handle h, int64_t nsweeps);

/* Random numbers of the temperature slots (Sec. 4's multi-spin coding puts
 * many replicas in one word; which of them share random numbers is a choice).
 * on = 1 (the default of a batch with exchange_every > 0): every slot draws its
 * own u, bit 31 - p of slot j's u being bit j of plane p, plane p = word p & 3
 * of Philox(m, sweep, colour | 3 << 1 | (p / 4 + 1) << 4, sample) for site m of
 * its colour, compared most significant plane first until every slot is
 * decided; replica exchange then keeps every temperature Boltzmann-distributed.
 * on = 0 (the default without exchange): the 32 slots of a site share one u,
 * word m & 3 of Philox(m >> 2, sweep, colour | 3 << 1, sample), about eight
 * times fewer Philox calls.  Each replica is still an exact Metropolis chain,
 * but the replicas of a sample are correlated, and with replica exchange the
 * temperature marginals then drift (about 1% of E at the hottest temperature
 * of a 4 x 4 ladder): choose it with exchange only knowingly.  Takes effect
 * from the next spn_batch_sweep.  SPN_E_STATE if h is not a batch handle,
 * SPN_E_ARG if on is not 0 or 1. */
int spn_batch_set_u_per_slot(spn_handle h, int32_t on);

/* Site words [sample][N] (bit j = replica in slot j, 1 = spin -1). */
int spn_batch_get_words(spn_handle h, uint32_t* out, size_t count);
int spn_batch_set_words(spn_handle h, const uint32_t* in, size_t count);

/* Temperature index of every slot, [sample][32]; set requires permutations. */
int spn_batch_get_slots(spn_handle h, uint8_t* temp_of_slot, size_t count);
int spn_batch_set_slots(spn_handle h, const uint8_t* temp_of_slot, size_t count);

/* Energy (Eq. 1 with J = +-1) and magnetisation of every replica by slot,
 * [sample][32], recomputed from the words on the device. */
int spn_batch_energies(spn_handle h, int64_t* E, int64_t* M, size_t count);

/* Accepted exchanges of pair (k, k+1) per sample, [sample][32] (entry 31 = 0). */
int spn_batch_exchange_counts(spn_handle h, int64_t* acc, size_t count);

/* Spin-glass overlap of replica pairs (Sec. 4's many disorder realisations;
 * two replicas of one realisation give its overlap).  Samples 2p and 2p+1 of
 * the batch are the two replicas of pair p: the batch needs an even number of
 * samples, and the couplings of 2p and 2p+1 must be identical (SPN_E_STATE
 * otherwise).  Enqueues one measurement on the handle's stream (asynchronous,
 * one kernel): for every pair p and temperature index t,
 *   q = sum_n s_n^(2p)(t) s_n^(2p+1)(t),
 * s^(i)(t) being the replica of sample i at temperature t; the device keeps q
 * and adds q^2 and q^4 to per-(pair, t) sums. */
int spn_batch_measure_overlap(spn_handle h);

/* The measurements so far (synchronises).  count = nsamples / 2 * 32; any
 * output may be NULL.  nmeas: measurements taken; q_last[p*32 + t]: q of the
 * last one; q2_sum[p*32 + t]: sum of q^2 (exact, uint64); q4_sum[2*(p*32 + t)]
 * and [2*(p*32 + t) + 1]: low and high 64 bits of the exact sum of q^4.  The
 * Binder cumulant g(t) = (3 - [<q^4>] / [<q^2>]^2) / 2 follows from these
 * (<.> = mean over measurements, [.] = mean over pairs). */
int spn_batch_overlap(spn_handle h, int64_t* nmeas, int64_t* q_last, uint64_t* q2_sum, uint64_t* q4_sum,
                      size_t count);

/* Clear the overlap sums and the measurement count (synchronises). */
int spn_batch_overlap_reset(spn_handle h);

/* ------------------------------------------------------------------------
 * Served requests with continuous batching (the paper serves nothing: each job
 * is the Sec. 3 procedure, or the Sec. 4 multi-spin coded ladder, run to
 * completion bit for bit as it would run alone)
 * ---------------------------------------------------------------------- */

/* A simulation request.  Ising (SPN_ISING2D / SPN_ISING3D): beta, nsweeps from
 * the hot start of (seed, stream).  EA (SPN_EA3D_PMJ, one disorder sample):
 * betas = 32 ladder betas, couplings = [3][ceil(N/64)] bond words, replica
 * exchange every exchange_every sweeps, seed; stream is ignored (sample 0).
 * Everything pointed to is copied by spn_submit. */
typedef struct spn_request {
  int32_t model;
  int32_t dims[3];
  double beta;
  const double* betas;
  int64_t nsweeps;
  uint64_t seed;
  uint32_t stream;
  int32_t exchange_every;
  const void* couplings;
} spn_request;

/* state: 0 queued, 1 admitted (running), 2 done, 3 failed (status = error code).
 * E, M: final energy and magnetisation (EA: the replica at the lowest
 * temperature).  Times in seconds on the server's monotonic clock. */
typedef struct spn_result {
  int32_t status;
  int32_t state;
  int64_t sweeps;
  int64_t E;
  int64_t M;
  double t_submit;
  double t_admit;
  double t_done;
} spn_result;

typedef struct spn_server_ctx* spn_server;

/* Start a server that admits jobs while their device memory (lattices, ping-
 * pong buffers, accumulators) fits hbm_budget_bytes.  A scheduler thread runs
 * rounds: each job chosen for a round (least recently run first, while their
 * SM equivalents fit the GPU) advances by a window of about 30 ms of its own run
 * time.  Ising lattices whose bits fit a cluster of up to 16 CTAs share
 * persistent resident launches, larger ones stream, EA jobs take one CTA each;
 * the launches run on a pool of streams, and jobs arriving during a round join
 * a later one.  Loading the library sets CUDA_DEVICE_MAX_CONNECTIONS to 32
 * unless the process has set it (effective only before a CUDA context exists):
 * a round runs more concurrent launches than the default 8 hardware queues. */
int spn_server_create(spn_server* out, size_t hbm_budget_bytes);

/* Queue a request (copied) and return its ticket at once; never waits for the
 * GPU.  SPN_E_BUDGET if the job alone exceeds the budget; SPN_E_ARG for odd
 * extents or a lattice past the counter range.  An EA sample must fit one
 * CTA's shared memory, as in spn_create_batch (about 44,000 sites); a larger
 * one is queued and then fails at admission (state 3, status SPN_E_ARG). */
int spn_submit(spn_server s, const spn_request* req, uint64_t* ticket);

/* Non-blocking: *done = 1 once the ticket's job is finished or failed; out
 * (may be NULL) receives its state and times. */
int spn_poll(spn_server s, uint64_t ticket, int* done, spn_result* out);

/* The result of a finished job: Ising N int8 spins; EA N uint32 replica words
 * followed by 32 bytes temp_of_slot. */
int spn_server_fetch(spn_server s, uint64_t ticket, void* out, size_t bytes);

/* Aggregate counters: attempted spin flips done, seconds the scheduler spent in
 * rounds, rounds, device bytes currently charged to the budget. */
int spn_server_stats(spn_server s, uint64_t* attempts, double* busy_seconds, uint64_t* rounds, size_t* used_bytes);

/* Stop accepting work, finish the admitted jobs, release everything. */
int spn_server_destroy(spn_server s);

/* ------------------------------------------------------------------------
 * Sweeps without device allocation
 * ---------------------------------------------------------------------- */

/* The paper has no counterpart of this entry point: it exists for callers that
 * must not let a library allocate device memory -- a host framework whose
 * caching allocator has reserved the device memory (a raw cudaMalloc would fail
 * or fragment its pool), plugin hosts that only hand out buffers, and
 * latency-critical loops in which cudaMalloc / cudaFree would synchronise the
 * device.
 *
 * Runs nsweeps sweeps (model SPN_ISING2D or SPN_ISING3D, J = +1) of the lattice
 * d_spins (device, N int8 +-1 in site order, updated in place) at inverse
 * temperature beta, with Philox seed / stream id and sweep counters sweep0 ..
 * sweep0 + nsweeps - 1 -- the same results as a handle created with this seed
 * and stream that has done sweep0 sweeps.  d_trace (device, 2 * nsweeps int64)
 * receives the change (dE, dM) of every sweep.  cuda_stream: cudaStream_t as
 * void* (NULL = legacy default stream).  Returns when the sweeps are done.
 *
 * It allocates nothing: its scratch (a second lattice for the ping-pong
 * streaming kernel and an error word) is a fixed 16 MiB static device array
 * that every GPU loading the library holds until the process exits, so N is
 * limited to 16,777,216 sites (SPN_E_ARG beyond).  A 16-byte aligned lattice
 * whose rows are whole multiples of 64 sites takes the streaming sweep; any other
 * lattice (including a pointer into the middle of a caller's buffer) takes the
 * generic sweep, with identical results.  The first call on a device
 * looks up that array's device address; make it before any stream capture.
 * All calls share the array: calls that overlap on the GPU (other threads or
 * streams) race and corrupt each other's results. */
int spn_sweep_noalloc(int model, const int32_t* dims, int8_t* d_spins, double beta, uint64_t seed,
                      uint32_t stream, uint32_t sweep0, int64_t nsweeps, int64_t* d_trace, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* SPN_H */
