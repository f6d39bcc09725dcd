/*
 * spn_oracle.c -- CPU oracle for the checkerboard Metropolis sweep of
 * nearest-neighbour Ising-type lattices (M. Weigel, "Simulating spin models on
 * GPU", Sec. 3 Eq. 1-2 and the sub-lattice procedure; Sec. 4 for the 3D model and
 * the +-J Edwards-Anderson spin glass with multi-spin coding).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the tests, the smoke check and
 * the CPU-baseline / reference legs of the benchmark load this library.  It
 * shares no code, header, table or helper with the CUDA library: both sides are
 * written independently from the same definitions.
 *
 * Plain, slow, obviously correct: every site is visited by a straight loop, the
 * local field is summed from its 2*d neighbours, the Metropolis probability is
 * the integer threshold of Eq. 2, and random numbers come from Philox4x32-10
 * (Salmon, Moraes, Dror, Shaw, SC'11) written from its published definition.
 * The only parallelism is an OpenMP loop over the sites of one colour; sites of
 * one colour are independent (Sec. 3), so the result does not depend on the
 * thread count.
 *
 * Definitions fixed here where the paper is silent (each one is a reading that
 * the GPU library follows too):
 *   lattice   extents L[0..d-1], all even; site n = x + Lx*(y + Ly*z);
 *             colour c(n) = (x+y+z) & 1; within-colour index m = n >> 1.
 *   energy    E = -sum_n sum_dir J(n,dir) s_n s_{n+e_dir}   (Eq. 1, each bond once)
 *             M = sum_n s_n.
 *   bonds     optional; bit (n % 64) of word [dir*nw + n/64] set <=> J(n,dir) = -1,
 *             nw = ceil(N/64).  Without bonds J = +1 (the ferromagnet of Eq. 1).
 *   threshold thr(beta, dE) = floor(exp(-beta*dE) * 2^32) for dE > 0 (Eq. 2),
 *             a value in [0, 2^32]; dE <= 0 is always accepted.
 *   random    R(c0,c1,c2,c3) = Philox4x32-10 with key (seed lo32, seed hi32).
 *             Each row (y, z) of the lattice is cut into words of 64 sites,
 *             x = 64 j .. 64 j + 63 (the last word of a row is shorter when
 *             Lx is not a multiple of 64); the sites of one colour in word j
 *             of row r = y + Ly z form group g = j + ceil(Lx / 64) r, site x
 *             at lane i = (x & 63) >> 1.  The site key is k = 32 g + i; when
 *             Lx is a multiple of 64 it equals the within-colour index m.  The
 *             group owns 32 "planes": plane q (0..31) is
 *             word q & 3 of R(8g + (q >> 2), t, c | (p << 1), stream).  Bit
 *             31 - q of the site word is bit i of plane q, so plane 0 carries the
 *             most significant bits of the group's sites.  Purposes p:
 *               0  Metropolis u at sweep t, colour c
 *               1  hot start (t = 0)
 *               4  Metropolis u of the double-checkerboard order at hit h of
 *                  sweep t (counter word 1 = t * hits + h)
 *             The 32-bit u is uniform; storing it across planes lets a GPU
 *             thread compare 32 sites at once, most significant plane first,
 *             and stop drawing planes as soon as every site is decided.
 *             Purpose 3 (multi-spin coded EA) uses plain words instead: the u
 *             of within-colour index m is word m & 3 of R(m >> 2, t, c | 3 << 1,
 *             stream), one word per site shared by the sample's 32 replicas.
 *   hot start s_n = -1 if bit 31 of the hot-start word is set, else +1.
 *   sweep t   colour 0, then colour 1; a site of colour c flips iff dE <= 0 or
 *             u < thr(beta, dE); E and M are updated by every accepted flip.
 *
 * Multi-spin coded EA (Sec. 4, "asynchronous multi-spin coding"), on the
 *   square (nd = 2) or simple cubic (nd = 3) lattice:
 *   one uint32 per (sample, site); bit j is the replica held in temperature slot
 *   j (1 <=> spin -1).  Without u_per_slot all 32 replicas of a sample share the
 *   site's u (purpose 3 words, stream = sample); with it every slot draws its
 *   own (orc_msc_slot_planes), which replica exchange needs.  Slot j
 *   runs at beta[temp_of_slot[j]]; betas are indexed by ascending temperature
 *   (non-increasing beta).  Hot start: the replica bits are the hot-start word.
 *   Replica exchange after every X-th sweep (step e = (t+1)/X - 1): for the
 *   temperature pairs (k, k+1) with k = e mod 2, 4, ... accept iff
 *   D = (beta_k - beta_{k+1}) * (E_k - E_{k+1}) >= 0 or
 *   u < floor(exp(D) * 2^32) with u = word k & 3 of R(k >> 2, e, 2 << 1, stream);
 *   an accepted pair swaps the slots of the two temperatures.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TWO32 4294967296.0

#if FLT_EVAL_METHOD != 0
#error "the Heisenberg oracle needs float expressions evaluated in float"
#endif

/* ---------------------------------------------------------------- Philox */

/* Philox4x32 with 10 rounds, Salmon et al. SC'11: each round multiplies words 0
 * and 2 by two fixed odd constants, swaps the words and mixes the high halves of
 * the products with the other two words and the round key; the key is bumped by
 * the two Weyl constants between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
    uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
    uint32_t y1 = (uint32_t)p1;
    uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
    uint32_t y3 = (uint32_t)p0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += W0; k1 += W1;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* The random-number reading of the header: the paper's per-thread LCG (Sec. 4)
 * is replaced by Philox4x32-10 (Salmon et al.) keyed by site, sweep and stream.
 * Site word of site key m for purpose p: bit 31 - q is bit (m & 31) of plane q
 * = word q & 3 of R(8 (m >> 5) + (q >> 2), t, c | (p << 1), stream). */
uint32_t orc_site_word(uint64_t seed, uint32_t stream, uint32_t t, int colour, int purpose, uint64_t m) {
  const uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  const uint32_t lane = (uint32_t)(m & 31);
  uint32_t u = 0;
  for (uint32_t call = 0; call < 8; ++call) {
    uint32_t ctr[4] = {(uint32_t)(8 * (m >> 5) + call), t, (uint32_t)colour | ((uint32_t)purpose << 1), stream};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    for (uint32_t j = 0; j < 4; ++j) {
      const uint32_t q = 4 * call + j;
      u |= ((w[j] >> lane) & 1u) << (31 - q);
    }
  }
  return u;
}

/* The u compared with the threshold of Eq. 2 (purpose 0). */
uint32_t orc_metropolis_u(uint64_t seed, uint32_t stream, uint32_t sweep, int colour, uint64_t m) {
  return orc_site_word(seed, stream, sweep, colour, 0, m);
}

/* The word of the seeded hot start (purpose 1; the paper does not state its start). */
uint32_t orc_hot_word(uint64_t seed, uint32_t stream, int colour, uint64_t m) {
  return orc_site_word(seed, stream, 0, colour, 1, m);
}

/* Multi-spin coded Metropolis u (Sec. 4: one random number for all bits of a
 * word): word m & 3 of R(m >> 2, sweep, c | 3 << 1, stream). */
uint32_t orc_msc_u(uint64_t seed, uint32_t stream, uint32_t sweep, int colour, uint64_t m) {
  const uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  uint32_t ctr[4] = {(uint32_t)(m >> 2), sweep, (uint32_t)colour | (3u << 1), stream};
  uint32_t w[4];
  orc_philox4x32_10(ctr, key, w);
  return w[m & 3];
}

/* Per-slot u of the multi-spin coded sweep when every slot draws its own
 * number (the remedy of the shared u: with replica exchange the 32 slots must
 * be independent for the ladder to keep its Boltzmann marginals): bit 31 - p
 * of slot j's u is bit j of plane p, plane p = word p & 3 of the Philox call
 * (m, sweep, colour | 3 << 1 | (p / 4 + 1) << 4, stream).  planes[32] out. */
void orc_msc_slot_planes(uint64_t seed, uint32_t stream, uint32_t sweep, int colour, uint64_t m, uint32_t planes[32]) {
  const uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  for (uint32_t call = 0; call < 8; ++call) {
    uint32_t ctr[4] = {(uint32_t)m, sweep, (uint32_t)colour | (3u << 1) | ((call + 1u) << 4), stream};
    orc_philox4x32_10(ctr, key, planes + 4 * call);
  }
}

static uint32_t slot_u(const uint32_t planes[32], int j) {
  uint32_t u = 0;
  for (int p = 0; p < 32; ++p) u |= ((planes[p] >> j) & 1u) << (31 - p);
  return u;
}

/* ------------------------------------------------------- Metropolis rule */

/* Eq. 2: p_acc = min[1, exp(-beta dE)], as the integer threshold
 * floor(exp(-beta dE) 2^32); a move with dE > 0 is accepted iff u < thr. */
uint64_t orc_threshold(double beta, int dE) {
  if (dE <= 0) return (uint64_t)1 << 32;
  double a = beta * (double)dE;
  double x = exp(-a) * ORC_TWO32;
  return (uint64_t)floor(x);
}

int orc_accept(double beta, int dE, uint32_t u) {
  if (dE <= 0) return 1;
  return (uint64_t)u < orc_threshold(beta, dE);
}

/* ---------------------------------------------------------- the lattice */

typedef struct {
  int nd;
  int64_t L[3];
  int64_t N;
  int64_t nw;
} lat_t;

static int lat_make(lat_t* g, int nd, const int64_t* L) {
  if (nd < 2 || nd > 3) return -1;
  g->nd = nd;
  g->N = 1;
  for (int d = 0; d < 3; ++d) {
    g->L[d] = d < nd ? L[d] : 1;
    if (d < nd && (g->L[d] < 2 || (g->L[d] & 1))) return -1;
    g->N *= g->L[d];
  }
  g->nw = (g->N + 63) / 64;
  return 0;
}

static void lat_coords(const lat_t* g, int64_t n, int64_t x[3]) {
  x[0] = n % g->L[0];
  x[1] = (n / g->L[0]) % g->L[1];
  x[2] = n / (g->L[0] * g->L[1]);
}

static int64_t lat_index(const lat_t* g, const int64_t x[3]) {
  return x[0] + g->L[0] * (x[1] + g->L[1] * x[2]);
}

/* Neighbour of n one step along direction d, forward (dir = +1) or back. */
static int64_t lat_step(const lat_t* g, int64_t n, int d, int dir) {
  int64_t x[3];
  lat_coords(g, n, x);
  x[d] = (x[d] + dir + g->L[d]) % g->L[d];
  return lat_index(g, x);
}

/* Site key of n: 32 (word of its row, counted over all rows) + lane. */
static uint64_t lat_key(const lat_t* g, int64_t n) {
  const int64_t x = n % g->L[0], row = n / g->L[0];
  const int64_t words = (g->L[0] + 63) / 64;
  return (uint64_t)(32 * ((x >> 6) + words * row) + ((x & 63) >> 1));
}

static int lat_colour(const lat_t* g, int64_t n) {
  int64_t x[3];
  lat_coords(g, n, x);
  return (int)((x[0] + x[1] + x[2]) & 1);
}

static int bond_J(const lat_t* g, const uint64_t* bonds, int64_t n, int d) {
  if (!bonds) return 1;
  uint64_t w = bonds[(int64_t)d * g->nw + (n >> 6)];
  return ((w >> (n & 63)) & 1) ? -1 : 1;
}

/* Local field h_n = sum_d [J(n,d) s_{n+e_d} + J(n-e_d,d) s_{n-e_d}]. */
static int local_field(const lat_t* g, const int8_t* s, const uint64_t* bonds, int64_t n) {
  int h = 0;
  for (int d = 0; d < g->nd; ++d) {
    int64_t f = lat_step(g, n, d, +1);
    int64_t b = lat_step(g, n, d, -1);
    h += bond_J(g, bonds, n, d) * s[f];
    h += bond_J(g, bonds, b, d) * s[b];
  }
  return h;
}

/* Energy change of flipping s_n under Eq. 1: dE = 2 s_n h_n (Sec. 3). */
int orc_delta_e(int nd, const int64_t* L, const int8_t* s, const uint64_t* bonds, int64_t n) {
  lat_t g;
  if (lat_make(&g, nd, L)) return 0;
  return 2 * s[n] * local_field(&g, s, bonds, n);
}

/* Eq. 1: E = -sum over bonds J s_i s_j (each bond once, through the forward
 * direction of its first site), M = sum s. */
int orc_observables(int nd, const int64_t* L, const int8_t* s, const uint64_t* bonds, int64_t* E,
                    int64_t* M) {
  lat_t g;
  if (lat_make(&g, nd, L)) return -1;
  int64_t e = 0, m = 0;
#pragma omp parallel for reduction(+ : e, m) schedule(static)
  for (int64_t n = 0; n < g.N; ++n) {
    m += s[n];
    for (int d = 0; d < g.nd; ++d) e -= (int64_t)bond_J(&g, bonds, n, d) * s[n] * s[lat_step(&g, n, d, +1)];
  }
  *E = e;
  *M = m;
  return 0;
}

/* Seeded hot start of every site from its hot-start word (the header's reading). */
int orc_init_hot(int nd, const int64_t* L, uint64_t seed, uint32_t stream, int8_t* s) {
  lat_t g;
  if (lat_make(&g, nd, L)) return -1;
#pragma omp parallel for schedule(static)
  for (int64_t n = 0; n < g.N; ++n) {
    uint32_t w = orc_hot_word(seed, stream, lat_colour(&g, n), lat_key(&g, n));
    s[n] = (w >> 31) ? -1 : 1;
  }
  return 0;
}

/* One half-sweep: every site of colour c decides from the state at the start of
 * the half-sweep.  Its neighbours all have the other colour, so an in-place loop
 * is the same as a simultaneous update (Sec. 3). */
static void half_sweep(const lat_t* g, int8_t* s, const uint64_t* bonds, const uint64_t* thr,
                       uint64_t seed, uint32_t stream, uint32_t sweep, int c, int umode, int64_t* dEsum,
                       int64_t* dMsum) {
  int64_t de = 0, dm = 0;
#pragma omp parallel for reduction(+ : de, dm) schedule(static)
  for (int64_t n = 0; n < g->N; ++n) {
    if (lat_colour(g, n) != c) continue;
    int dE = 2 * s[n] * local_field(g, s, bonds, n);
    int acc;
    if (dE <= 0) {
      acc = 1;
    } else {
      uint32_t u = umode ? orc_msc_u(seed, stream, sweep, c, (uint64_t)(n >> 1))
                         : orc_metropolis_u(seed, stream, sweep, c, lat_key(g, n));
      acc = (uint64_t)u < thr[dE / 4];
    }
    if (acc) {
      dm += -2 * s[n];
      s[n] = (int8_t)(-s[n]);
      de += dE;
    }
  }
  *dEsum += de;
  *dMsum += dm;
}

/* The sub-lattice procedure of Sec. 3 with the acceptance of Eq. 2:
 * nsweeps sweeps starting at global sweep index sweep0.  E and M are the running
 * sums (in/out); traceE/traceM, if given, receive E and M after each sweep.
 * umode 0 draws u from the Ising bit planes (purpose 0), umode 1 from the
 * multi-spin coded words (purpose 3) -- the latter lets a scalar run reproduce
 * one replica of a multi-spin coded sample. */
int orc_sweeps_ex(int nd, const int64_t* L, int8_t* s, const uint64_t* bonds, double beta, uint64_t seed,
                  uint32_t stream, uint32_t sweep0, int64_t nsweeps, int umode, int64_t* E, int64_t* M,
                  int64_t* traceE, int64_t* traceM) {
  lat_t g;
  if (lat_make(&g, nd, L)) return -1;
  uint64_t thr[4];
  for (int k = 0; k < 4; ++k) thr[k] = orc_threshold(beta, 4 * k);
  for (int64_t t = 0; t < nsweeps; ++t) {
    uint32_t sweep = sweep0 + (uint32_t)t;
    int64_t de = 0, dm = 0;
    half_sweep(&g, s, bonds, thr, seed, stream, sweep, 0, umode, &de, &dm);
    half_sweep(&g, s, bonds, thr, seed, stream, sweep, 1, umode, &de, &dm);
    *E += de;
    *M += dm;
    if (traceE) traceE[t] = *E;
    if (traceM) traceM[t] = *M;
  }
  return 0;
}

/* orc_sweeps_ex (Sec. 3, Eq. 2) drawing u from the Ising bit planes. */
int orc_sweeps(int nd, const int64_t* L, int8_t* s, const uint64_t* bonds, double beta, uint64_t seed,
               uint32_t stream, uint32_t sweep0, int64_t nsweeps, int64_t* E, int64_t* M,
               int64_t* traceE, int64_t* traceM) {
  return orc_sweeps_ex(nd, L, s, bonds, beta, seed, stream, sweep0, nsweeps, 0, E, M, traceE, traceM);
}

/* ------------------------------------------- double checkerboard (Sec. 3) */

/* Tile parity of site n for tiles of T[0] x T[1] (x T[2]) sites: the parity of
 * the tile's coordinates (the "coarse" checkerboard). */
static int dc_tile_parity(const lat_t* g, const int64_t* T, int64_t n) {
  int64_t x[3];
  lat_coords(g, n, x);
  return (int)((x[0] / T[0] + x[1] / T[1] + (g->nd == 3 ? x[2] / T[2] : 0)) & 1);
}

/* Sec. 3, the double-checkerboard procedure with the generalised multi-hit:
 * the lattice is cut into coarse tiles, coloured like a checkerboard; a sweep
 * takes the tiles of parity 0, then those of parity 1, and within them runs
 * `hits` times over: every site of colour 0 (the fine checkerboard), then every
 * site of colour 1.  Sites updated together are never neighbours: they share a
 * colour, and a tile's boundary layer belongs to tiles of the other parity.
 * The u of a site at hit h of sweep t is its purpose-4 plane word with counter
 * word 1 = t hits + h.  Every extent must be a multiple of its tile edge, with
 * an even number of tiles along each axis. */
int orc_sweeps_dc(int nd, const int64_t* L, int8_t* s, const int64_t* T, int hits, double beta, uint64_t seed,
                  uint32_t stream, uint32_t sweep0, int64_t nsweeps, int64_t* E, int64_t* M, int64_t* traceE,
                  int64_t* traceM) {
  lat_t g;
  if (lat_make(&g, nd, L) || hits < 1) return -1;
  for (int d = 0; d < nd; ++d)
    if (T[d] < 1 || L[d] % T[d] || (L[d] / T[d]) % 2) return -1;
  uint64_t thr[4];
  for (int k = 0; k < 4; ++k) thr[k] = orc_threshold(beta, 4 * k);
  for (int64_t t = 0; t < nsweeps; ++t) {
    const uint64_t sweep = (uint64_t)sweep0 + (uint64_t)t;
    int64_t de = 0, dm = 0;
    for (int P = 0; P < 2; ++P)
      for (int h = 0; h < hits; ++h)
        for (int c = 0; c < 2; ++c) {
          const uint32_t ctr = (uint32_t)(sweep * (uint64_t)hits + (uint64_t)h);
#pragma omp parallel for reduction(+ : de, dm) schedule(static)
          for (int64_t n = 0; n < g.N; ++n) {
            if (lat_colour(&g, n) != c || dc_tile_parity(&g, T, n) != P) continue;
            const int dE = 2 * s[n] * local_field(&g, s, NULL, n);
            int acc = 1;
            if (dE > 0) acc = (uint64_t)orc_site_word(seed, stream, ctr, c, 4, lat_key(&g, n)) < thr[dE / 4];
            if (acc) {
              dm += -2 * s[n];
              s[n] = (int8_t)(-s[n]);
              de += dE;
            }
          }
        }
    *E += de;
    *M += dm;
    if (traceE) traceE[t] = *E;
    if (traceM) traceM[t] = *M;
  }
  return 0;
}

/* ------------------------------------------------- multi-spin coded EA */

/* Replica bit j of a site word, as a spin +-1. */
static int rep_spin(uint32_t w, int j) { return ((w >> j) & 1) ? -1 : 1; }

/* Seeded hot start of the multi-spin coded samples: every replica bit of a site
 * word is the hot-start word (sample i uses stream stream0 + i). */
int orc_ea_init_hot(int nd, const int64_t* L, int nsamples, uint64_t seed, uint32_t stream0, uint32_t* sp) {
  lat_t g;
  if (lat_make(&g, nd, L)) return -1;
  for (int i = 0; i < nsamples; ++i)
    for (int64_t n = 0; n < g.N; ++n)
      sp[(int64_t)i * g.N + n] = orc_hot_word(seed, stream0 + (uint32_t)i, lat_colour(&g, n), lat_key(&g, n));
  return 0;
}

/* Eq. 1 with the +-J bonds of the Sec. 4 spin glass, for every replica of
 * every sample, indexed by slot: E[i*32 + j], M[i*32 + j]. */
int orc_ea_observables(int nd, const int64_t* L, int nsamples, const uint32_t* sp, const uint64_t* bonds,
                       int64_t* E, int64_t* M) {
  lat_t g;
  if (lat_make(&g, nd, L)) return -1;
  for (int i = 0; i < nsamples; ++i) {
    const uint32_t* w = sp + (int64_t)i * g.N;
    const uint64_t* J = bonds + (int64_t)i * nd * g.nw;
    for (int j = 0; j < 32; ++j) {
      int64_t e = 0, m = 0;
      for (int64_t n = 0; n < g.N; ++n) {
        int sn = rep_spin(w[n], j);
        m += sn;
        for (int d = 0; d < nd; ++d) e -= (int64_t)bond_J(&g, J, n, d) * sn * rep_spin(w[lat_step(&g, n, d, +1)], j);
      }
      E[i * 32 + j] = e;
      M[i * 32 + j] = m;
    }
  }
  return 0;
}

/* One exchange step e for one sample (temperatures indexed by ascending T).
 * Eslot: energies by slot; slot_of_temp / temp_of_slot: the permutation (in/out);
 * acc: per-pair acceptance counters (may be NULL). */
static void exchange_step(const double* betas, const int64_t* Eslot, uint8_t* slot_of_temp,
                          uint8_t* temp_of_slot, uint64_t seed, uint32_t stream, uint32_t e, int64_t* acc) {
  int64_t Et[32];
  for (int t = 0; t < 32; ++t) Et[t] = Eslot[slot_of_temp[t]];
  for (int k = (int)(e & 1); k + 1 < 32; k += 2) {
    double D = (betas[k] - betas[k + 1]) * (double)(Et[k] - Et[k + 1]);
    int accept;
    if (D >= 0) {
      accept = 1;
    } else {
      uint32_t ctr[4] = {(uint32_t)k >> 2, e, 2u << 1, stream};
      uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
      uint32_t w[4];
      orc_philox4x32_10(ctr, key, w);
      uint64_t thr = (uint64_t)floor(exp(D) * ORC_TWO32);
      accept = (uint64_t)w[k & 3] < thr;
    }
    if (accept) {
      uint8_t a = slot_of_temp[k], b = slot_of_temp[k + 1];
      slot_of_temp[k] = b;
      slot_of_temp[k + 1] = a;
      temp_of_slot[b] = (uint8_t)k;
      temp_of_slot[a] = (uint8_t)(k + 1);
      if (acc) acc[k] += 1;
    }
  }
}

/* Sec. 4's multi-spin coded sweep (Eq. 2 per replica bit) with replica exchange:
 * nsweeps multi-spin coded sweeps of nsamples samples (sample i uses stream
 * stream0 + i), from global sweep index sweep0, with replica exchange after every
 * exchange_every-th sweep (0 = never).  temp_of_slot / slot_of_temp: [sample][32],
 * in/out.  acc: [sample][32] exchange acceptance counters (may be NULL). */
int orc_ea_sweeps_ex(int nd, const int64_t* L, int nsamples, uint32_t* sp, const uint64_t* bonds, const double* betas,
                     uint8_t* temp_of_slot, uint8_t* slot_of_temp, uint64_t seed, uint32_t stream0,
                     uint32_t sweep0, int64_t nsweeps, int exchange_every, int64_t* acc, int u_per_slot) {
  lat_t g;
  if (lat_make(&g, nd, L)) return -1;
  uint64_t thr[32][4];
  for (int t = 0; t < 32; ++t)
    for (int k = 0; k < 4; ++k) thr[t][k] = orc_threshold(betas[t], 4 * k);
  int64_t* Eslot = (int64_t*)malloc(sizeof(int64_t) * 32);
  int64_t* Mslot = (int64_t*)malloc(sizeof(int64_t) * 32);
  for (int i = 0; i < nsamples; ++i) {
    uint32_t* w = sp + (int64_t)i * g.N;
    const uint64_t* J = bonds + (int64_t)i * nd * g.nw;
    uint8_t* pi = temp_of_slot + 32 * i;
    uint8_t* tau = slot_of_temp + 32 * i;
    uint32_t stream = stream0 + (uint32_t)i;
    for (int64_t t = 0; t < nsweeps; ++t) {
      uint32_t sweep = sweep0 + (uint32_t)t;
      for (int c = 0; c < 2; ++c) {
#pragma omp parallel for schedule(static)
        for (int64_t n = 0; n < g.N; ++n) {
          if (lat_colour(&g, n) != c) continue;
          uint32_t u = orc_msc_u(seed, stream, sweep, c, (uint64_t)(n >> 1));
          uint32_t planes[32];
          if (u_per_slot) orc_msc_slot_planes(seed, stream, sweep, c, (uint64_t)(n >> 1), planes);
          uint32_t flip = 0;
          for (int j = 0; j < 32; ++j) {
            if (u_per_slot) u = slot_u(planes, j);
            int sn = rep_spin(w[n], j);
            int h = 0;
            for (int d = 0; d < nd; ++d) {
              int64_t f = lat_step(&g, n, d, +1), b = lat_step(&g, n, d, -1);
              h += bond_J(&g, J, n, d) * rep_spin(w[f], j);
              h += bond_J(&g, J, b, d) * rep_spin(w[b], j);
            }
            int dE = 2 * sn * h;
            int a = dE <= 0 || (uint64_t)u < thr[pi[j]][dE / 4];
            if (a) flip |= 1u << j;
          }
          w[n] ^= flip;
        }
      }
      if (exchange_every > 0 && ((int64_t)sweep + 1) % exchange_every == 0) {
        uint32_t e = (uint32_t)(((int64_t)sweep + 1) / exchange_every - 1);
        orc_ea_observables(nd, L, 1, w, J, Eslot, Mslot);
        exchange_step(betas, Eslot, tau, pi, seed, stream, e, acc ? acc + 32 * i : NULL);
      }
    }
  }
  free(Eslot);
  free(Mslot);
  return 0;
}

/* orc_ea_sweeps_ex (Sec. 4) with the shared u of every slot. */
int orc_ea_sweeps(int nd, const int64_t* L, int nsamples, uint32_t* sp, const uint64_t* bonds, const double* betas,
                  uint8_t* temp_of_slot, uint8_t* slot_of_temp, uint64_t seed, uint32_t stream0,
                  uint32_t sweep0, int64_t nsweeps, int exchange_every, int64_t* acc) {
  return orc_ea_sweeps_ex(nd, L, nsamples, sp, bonds, betas, temp_of_slot, slot_of_temp, seed, stream0, sweep0,
                          nsweeps, exchange_every, acc, 0);
}

/* ------------------------------------- disorder-parallel multi-spin coding */

/* Sec. 4 runs many disorder realisations at once with asynchronous multi-spin
 * coding: the bits of a machine word are different samples, updated with one
 * random number.  Here 32 samples form a group and share the site's u at each
 * temperature; a sample's 32 temperatures draw independent u (other groups of
 * the Philox stream), so replica exchange within a sample sees independent
 * replicas.
 *
 *   group     sample s belongs to group g(s) = 2 (s >> 6) + (s & 1); samples 2p
 *             and 2p + 1 (a replica pair of one realisation, when their
 *             couplings are equal) fall in different groups.
 *   random    the Metropolis u of group g at temperature index t, site n of
 *             colour c, sweep: word m & 3 of R(m >> 2, sweep, c | 3 << 1,
 *             32 g + t), m = n >> 1 (the multi-spin coded word of stream 32 g + t).
 *   state     sp[s*N + n], bit t = the configuration at temperature t (1 <=>
 *             spin -1); bit t runs at beta[t] (ascending temperature).
 *   sweep     colour 0, then colour 1; bit t of a site of colour c flips iff
 *             dE <= 0 or u < thr(beta_t, dE).
 *   exchange  after every X-th sweep (step e = (sweep + 1) / X - 1), for each
 *             sample the pairs (k, k+1), k = e mod 2, e mod 2 + 2, ...: with
 *             E_k the energy of the configuration at temperature k, accept iff
 *             D = (beta_k - beta_{k+1}) (E_k - E_{k+1}) >= 0 or
 *             u < floor(exp(D) 2^32), u = word k & 3 of R(k >> 2, e, 2 << 1, s);
 *             an accepted pair swaps the two configurations (bits k and k + 1 of
 *             every site word) and counts in acc[s*32 + k].
 *   sample0   row i of sp (and of bonds, acc) is sample sample0 + i of the batch,
 *             so a subset of a batch can be run alone. */
int orc_ea_dp_group(int sample) { return 2 * (sample >> 6) + (sample & 1); }

int orc_ea_dp_sweeps(int nd, const int64_t* L, int nsamples, uint32_t* sp, const uint64_t* bonds, const double* betas,
                     uint64_t seed, uint32_t sweep0, int64_t nsweeps, int exchange_every, int64_t* acc,
                     int sample0) {
  lat_t g;
  if (lat_make(&g, nd, L)) return -1;
  uint64_t thr[32][4];
  for (int t = 0; t < 32; ++t)
    for (int k = 0; k < 4; ++k) thr[t][k] = orc_threshold(betas[t], 4 * k);
  const uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  for (int i = 0; i < nsamples; ++i) {
    uint32_t* w = sp + (int64_t)i * g.N;
    const uint64_t* J = bonds + (int64_t)i * nd * g.nw;
    const int sample = sample0 + i;  /* the batch index of row i of sp */
    const uint32_t group = (uint32_t)orc_ea_dp_group(sample);
    for (int64_t it = 0; it < nsweeps; ++it) {
      uint32_t sweep = sweep0 + (uint32_t)it;
      for (int c = 0; c < 2; ++c) {
#pragma omp parallel for schedule(static)
        for (int64_t n = 0; n < g.N; ++n) {
          if (lat_colour(&g, n) != c) continue;
          uint32_t flip = 0;
          for (int t = 0; t < 32; ++t) {
            uint32_t u = orc_msc_u(seed, 32u * group + (uint32_t)t, sweep, c, (uint64_t)(n >> 1));
            int sn = rep_spin(w[n], t);
            int h = 0;
            for (int d = 0; d < nd; ++d) {
              int64_t f = lat_step(&g, n, d, +1), b = lat_step(&g, n, d, -1);
              h += bond_J(&g, J, n, d) * rep_spin(w[f], t);
              h += bond_J(&g, J, b, d) * rep_spin(w[b], t);
            }
            int dE = 2 * sn * h;
            if (dE <= 0 || (uint64_t)u < thr[t][dE / 4]) flip |= 1u << t;
          }
          w[n] ^= flip;
        }
      }
      if (exchange_every > 0 && ((int64_t)sweep + 1) % exchange_every == 0) {
        uint32_t e = (uint32_t)(((int64_t)sweep + 1) / exchange_every - 1);
        int64_t E[32], M[32];
        orc_ea_observables(nd, L, 1, w, J, E, M);  /* bit t: the configuration at temperature t */
        for (int k = (int)(e & 1); k + 1 < 32; k += 2) {
          double D = (betas[k] - betas[k + 1]) * (double)(E[k] - E[k + 1]);
          int accept;
          if (D >= 0) {
            accept = 1;
          } else {
            uint32_t ctr[4] = {(uint32_t)k >> 2, e, 2u << 1, (uint32_t)sample};
            uint32_t r[4];
            orc_philox4x32_10(ctr, key, r);
            accept = (uint64_t)r[k & 3] < (uint64_t)floor(exp(D) * ORC_TWO32);
          }
          if (accept) {
            for (int64_t n = 0; n < g.N; ++n) {
              uint32_t d = ((w[n] >> k) ^ (w[n] >> (k + 1))) & 1u;
              w[n] ^= (d << k) | (d << (k + 1));
            }
            if (acc) acc[32 * (int64_t)i + k] += 1;
          }
        }
      }
    }
  }
  return 0;
}

/* Spin-glass overlap of replica pairs (Sec. 4: many disorder realisations at
 * once; two replicas of one realisation give its overlap): samples 2p and
 * 2p + 1 are two replicas of pair p.  For every temperature index t,
 * q[p*32 + t] = sum_n s_n^(2p)(t) s_n^(2p+1)(t), where s^(i)(t) is the replica of
 * sample i held in slot slot_of_temp[i*32 + t].  A plain double loop. */
int orc_ea_overlap(int nd, const int64_t* L, int npairs, const uint32_t* sp, const uint8_t* slot_of_temp,
                   int64_t* q) {
  lat_t g;
  if (lat_make(&g, nd, L)) return -1;
  for (int p = 0; p < npairs; ++p) {
    const uint32_t* wa = sp + (int64_t)(2 * p) * g.N;
    const uint32_t* wb = sp + (int64_t)(2 * p + 1) * g.N;
    for (int t = 0; t < 32; ++t) {
      const int ja = slot_of_temp[(2 * p) * 32 + t], jb = slot_of_temp[(2 * p + 1) * 32 + t];
      int64_t sum = 0;
      for (int64_t n = 0; n < g.N; ++n) sum += (int64_t)rep_spin(wa[n], ja) * rep_spin(wb[n], jb);
      q[p * 32 + t] = sum;
    }
  }
  return 0;
}

/* ------------------------------------------ Heisenberg spins (Sec. 4 outlook) */

/* The classical O(3) Heisenberg model H = -sum_<ij> S_i . S_j (J = 1, |S| = 1),
 * the continuous-spin generalisation the paper names for single-precision GPU
 * arithmetic, with the same checkerboard Metropolis sweep: a site of colour c
 * proposes a new direction S' uniformly on the sphere and takes it iff
 * dE = -(S' - S) . h <= 0 or u < exp(-beta dE), h the sum of its 2 nd
 * neighbours.  Spins are binary32 (x, y, z) per site.  Every floating-point step
 * is one IEEE-754 binary32 operation (+, -, *, sqrt, round-to-integral), rounded
 * to nearest, in the order written (left to right), never fused (this file is
 * built with -ffp-contract=off and evaluates float expressions in float); no
 * library transcendental is called, so any implementation doing the same
 * operations gets the same bits.
 *   random  proposals: call k = 0..7 is R(m, t, c | 5 << 1 | k << 4, stream),
 *           m = n >> 1; tries 2k and 2k+1 take words (0, 1) and (2, 3); hot
 *           start: the same with purpose 7 and t = 0.  Metropolis u: word m & 3
 *           of R(m >> 2, t, c | 6 << 1, stream).  A word w gives the binary32
 *           value (w >> 8) 2^-24 in [0, 1) exactly.
 *   beta    rounded once to binary32. */

static float f32_bits_pow2(int k) { /* 2^k for -126 <= k <= 127, exactly */
  uint32_t b = (uint32_t)(127 + k) << 23;
  float f;
  memcpy(&f, &b, sizeof f);
  return f;
}

/* exp(x) for x <= 0: Cody-Waite reduction (Cody and Waite, "Software Manual for
 * the Elementary Functions", 1980) x = k ln2 + r, k the nearest integer to
 * x log2(e) and ln 2 split into a 16-bit high part (so k ln2_hi is exact) and
 * the rest; e^r by its Taylor polynomial of degree 7 in Horner form; times 2^k.
 * x < -87 gives 0 (the result would leave the normal range). */
float orc_heis_exp(float x) {
  const float log2e = (float)(1.0 / 0.6931471805599453);
  const float ln2_hi = 45426.0f / 65536.0f;
  const float ln2_lo = (float)(0.6931471805599453 - 45426.0 / 65536.0);
  const float c[8] = {1.0f, 1.0f, 0.5f, (float)(1.0 / 6.0), (float)(1.0 / 24.0), (float)(1.0 / 120.0),
                      (float)(1.0 / 720.0), (float)(1.0 / 5040.0)};
  if (x < -87.0f) return 0.0f;
  if (x > 0.0f) return 1.0f; /* not used: the sweep only asks for dE > 0 */
  const float kf = rintf(x * log2e);
  const float r = (x - kf * ln2_hi) - kf * ln2_lo;
  float p = c[7];
  for (int i = 6; i >= 0; --i) p = p * r + c[i];
  return p * f32_bits_pow2((int)kf);
}

static float word_unit(uint32_t w) { return (float)(w >> 8) * (1.0f / 16777216.0f); }

/* Marsaglia's uniform point on the sphere (Ann. Math. Stat. 43, 645 (1972)) from
 * the purpose-p words of site m: v1, v2 = 2 (w >> 8) 2^-24 - 1 in [-1, 1); the
 * first try with s = v1^2 + v2^2 < 1 gives S = (2 v1 sqrt(1-s), 2 v2 sqrt(1-s),
 * 1 - 2 s).  Returns 0 if all 16 tries fail (then there is no proposal). */
int orc_heis_proposal(uint64_t seed, uint32_t stream, uint32_t t, int colour, int purpose, uint64_t m, float out[3]) {
  const uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  for (uint32_t k = 0; k < 8; ++k) {
    uint32_t ctr[4] = {(uint32_t)m, t, (uint32_t)colour | ((uint32_t)purpose << 1) | (k << 4), stream};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    for (int j = 0; j < 2; ++j) {
      const float v1 = (float)(w[2 * j] >> 8) * (1.0f / 8388608.0f) - 1.0f;
      const float v2 = (float)(w[2 * j + 1] >> 8) * (1.0f / 8388608.0f) - 1.0f;
      const float ss = v1 * v1 + v2 * v2;
      if (ss < 1.0f) {
        const float f = 2.0f * sqrtf(1.0f - ss);
        out[0] = v1 * f;
        out[1] = v2 * f;
        out[2] = 1.0f - 2.0f * ss;
        return 1;
      }
    }
  }
  return 0;
}

/* Seeded hot start of Heisenberg spins: each site a uniform point on the sphere
 * from orc_heis_proposal with purpose 7 at t = 0, or (0, 0, 1) if its 16 tries
 * all miss. */
int orc_heis_init_hot(int nd, const int64_t* L, uint64_t seed, uint32_t stream, float* S) {
  lat_t g;
  if (lat_make(&g, nd, L)) return -1;
  for (int64_t n = 0; n < g.N; ++n) {
    float v[3] = {0.0f, 0.0f, 1.0f};
    orc_heis_proposal(seed, stream, 0, lat_colour(&g, n), 7, (uint64_t)(n >> 1), v);
    S[3 * n] = v[0];
    S[3 * n + 1] = v[1];
    S[3 * n + 2] = v[2];
  }
  return 0;
}

/* Eq. 1 for the continuous spins of Sec. 4's outlook (classical Heisenberg):
 * E = -sum_n sum_d S_n . S_{n+e_d} and M = sum_n S_n, in binary64 in site order
 * (products of two binary32 values are exact in binary64). */
int orc_heis_observables(int nd, const int64_t* L, const float* S, double* E, double* M) {
  lat_t g;
  if (lat_make(&g, nd, L)) return -1;
  double e = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
  for (int64_t n = 0; n < g.N; ++n) {
    for (int d = 0; d < nd; ++d) {
      const int64_t f = lat_step(&g, n, d, +1);
      e -= (double)S[3 * n] * S[3 * f] + (double)S[3 * n + 1] * S[3 * f + 1] + (double)S[3 * n + 2] * S[3 * f + 2];
    }
    mx += S[3 * n];
    my += S[3 * n + 1];
    mz += S[3 * n + 2];
  }
  *E = e;
  M[0] = mx;
  M[1] = my;
  M[2] = mz;
  return 0;
}

/* The sub-lattice procedure of Sec. 3 and Eq. 2 for Heisenberg spins:
 * nsweeps sweeps from global sweep index sweep0.  E and M (in/out) are advanced
 * by the accepted moves, in site order; traceE[s], traceM[3 s ..] after sweep s. */
int orc_heis_sweeps(int nd, const int64_t* L, float* S, double beta, uint64_t seed, uint32_t stream, uint32_t sweep0,
                    int64_t nsweeps, double* E, double* M, double* traceE, double* traceM) {
  lat_t g;
  if (lat_make(&g, nd, L)) return -1;
  const float bf = (float)beta;
  const uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  double* dE = (double*)malloc(sizeof(double) * 4 * (size_t)g.N);
  if (!dE) return -1;
  for (int64_t t = 0; t < nsweeps; ++t) {
    const uint32_t sweep = sweep0 + (uint32_t)t;
    for (int c = 0; c < 2; ++c) {
#pragma omp parallel for schedule(static)
      for (int64_t n = 0; n < g.N; ++n) {
        double* rec = dE + 4 * n;
        rec[0] = rec[1] = rec[2] = rec[3] = 0.0;
        if (lat_colour(&g, n) != c) continue;
        float h[3] = {0.0f, 0.0f, 0.0f};
        for (int d = 0; d < nd; ++d) {
          const int64_t b = lat_step(&g, n, d, -1), f = lat_step(&g, n, d, +1);
          for (int i = 0; i < 3; ++i) {
            h[i] = h[i] + S[3 * b + i];
            h[i] = h[i] + S[3 * f + i];
          }
        }
        float p[3];
        if (!orc_heis_proposal(seed, stream, sweep, c, 5, (uint64_t)(n >> 1), p)) continue;
        float ds[3];
        for (int i = 0; i < 3; ++i) ds[i] = p[i] - S[3 * n + i];
        float dot = ds[0] * h[0];
        dot = dot + ds[1] * h[1];
        dot = dot + ds[2] * h[2];
        const float de = -dot;
        int accept = de <= 0.0f;
        if (!accept) {
          const uint64_t m = (uint64_t)(n >> 1);
          uint32_t ctr[4] = {(uint32_t)(m >> 2), sweep, (uint32_t)c | (6u << 1), stream};
          uint32_t w[4];
          orc_philox4x32_10(ctr, key, w);
          accept = word_unit(w[m & 3]) < orc_heis_exp(-(bf * de));
        }
        if (accept) {
          rec[0] = de;
          for (int i = 0; i < 3; ++i) {
            rec[1 + i] = ds[i];
            S[3 * n + i] = p[i];
          }
        }
      }
      for (int64_t n = 0; n < g.N; ++n) {
        *E += dE[4 * n];
        for (int i = 0; i < 3; ++i) M[i] += dE[4 * n + 1 + i];
      }
    }
    if (traceE) traceE[t] = *E;
    if (traceM)
      for (int i = 0; i < 3; ++i) traceM[3 * t + i] = M[i];
  }
  free(dE);
  return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the OpenMP loops from now on (timing support: 1 gives the serial
 * figure); no effect without OpenMP. */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
  extern void omp_set_num_threads(int);
  omp_set_num_threads(n > 0 ? n : 1);
#else
  (void)n;
#endif
}
