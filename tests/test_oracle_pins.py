"""Pins of the CPU oracle against results fixed by the paper and by mathematics.

Each test checks one part of the oracle against something other than itself:
a library implementation of Philox, closed forms (Kaufman, Onsager, the exact
threshold), brute-force enumeration, exact invariants (gauge symmetry, beta = 0
and beta = infinity dynamics) and exact stationarity of the half-sweep kernel.
"""

from __future__ import annotations

import os
import subprocess
import sys
import textwrap

import mpmath as mp
import numpy as np
import pytest

import oracle
from exact_lattice import energy, neighbours, reachable
from exact_ising import (binned_mean_err, binned_variance_err, energy_histogram_pvalue, enumerate_2d, exact_averages,
                         kaufman_energy, kaufman_energy_variance, kaufman_log_z, log_z_enumerated,
                         onsager_energy_per_spin)
from paper_1006_3865_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


# ----------------------------------------------------------------- Philox

def test_philox_matches_library_implementation():
    """Philox4x32-10 (Salmon et al. SC'11) against Triton's implementation of the
    same generator, run on the CPU through Triton's interpreter."""
    pytest.importorskip("triton")
    code = textwrap.dedent(
        """
        import os, sys
        os.environ["TRITON_INTERPRET"] = "1"
        import numpy as np, torch, triton, triton.language as tl

        @triton.jit
        def k(out_ptr, c0_ptr, c1_ptr, c2_ptr, c3_ptr, seed, N: tl.constexpr):
            i = tl.arange(0, N)
            a, b, c, d = tl.philox(seed, tl.load(c0_ptr + i), tl.load(c1_ptr + i),
                                   tl.load(c2_ptr + i), tl.load(c3_ptr + i))
            tl.store(out_ptr + 4 * i + 0, a); tl.store(out_ptr + 4 * i + 1, b)
            tl.store(out_ptr + 4 * i + 2, c); tl.store(out_ptr + 4 * i + 3, d)

        N = 64
        rng = np.random.default_rng(7)
        C = rng.integers(0, 2**32, size=(4, N), dtype=np.uint64).astype(np.uint32)
        C[:, 0] = 0
        C[:, 1] = 0xFFFFFFFF
        cs = [torch.from_numpy(C[j].view(np.int32).copy()) for j in range(4)]
        for seed in (0, 0xFFFFFFFFFFFFFFFF, 0x5EED5EED, 0x0123456789ABCDEF):
            out = torch.zeros(4 * N, dtype=torch.int32)
            k[(1,)](out, *cs, seed, N=N)
            np.save(sys.argv[1] + f"_{seed:x}.npy", out.numpy().view(np.uint32).reshape(N, 4))
        np.save(sys.argv[1] + "_ctr.npy", C)
        """)
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        prefix = os.path.join(d, "ph")
        r = subprocess.run([sys.executable, "-c", code, prefix], capture_output=True, text=True, timeout=600)
        if r.returncode != 0:
            pytest.skip("triton interpreter unavailable: " + r.stderr.strip().splitlines()[-1][:200])
        C = np.load(prefix + "_ctr.npy")
        for seed in (0, 0xFFFFFFFFFFFFFFFF, 0x5EED5EED, 0x0123456789ABCDEF):
            ref = np.load(prefix + f"_{seed:x}.npy")
            key = [seed & 0xFFFFFFFF, seed >> 32]
            for i in range(C.shape[1]):
                got = oracle.philox4x32_10(C[:, i], key)
                assert np.array_equal(got, ref[i]), (seed, i, got, ref[i])


def test_site_word_layout():
    """Bit 31 - q of a site word is bit (m & 31) of plane q = word q & 3 of the
    Philox call 8 (m >> 5) + q >> 2 (most significant plane first)."""
    seed, stream, t, c = 0xABCDEF0123, 5, 17, 1
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for m in (0, 1, 2, 31, 32, 63, 1023, 12345):
        planes = [oracle.philox4x32_10([8 * (m >> 5) + call, t, c | (0 << 1), stream], key) for call in range(8)]
        bits = [(int(planes[q >> 2][q & 3]) >> (m & 31)) & 1 for q in range(32)]
        u = sum(b << (31 - q) for q, b in enumerate(bits))
        assert oracle.metropolis_u(seed, stream, t, c, m) == u
    # hot start draws purpose 1
    planes = [oracle.philox4x32_10([8 * 3 + call, 0, 0 | (1 << 1), stream], key) for call in range(8)]
    u = sum(((int(planes[q >> 2][q & 3]) >> 7) & 1) << (31 - q) for q in range(32))
    assert oracle.hot_word(seed, stream, 0, 3 * 32 + 7) == u


def test_msc_u_layout():
    """The multi-spin coded u of index m is word m & 3 of the call m >> 2 (purpose 3)."""
    seed, stream, t, c = 0x1234, 9, 3, 1
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for m in (0, 1, 3, 4, 1000, 77777):
        w = oracle.philox4x32_10([m >> 2, t, c | (3 << 1), stream], key)
        assert oracle.msc_u(seed, stream, t, c, m) == int(w[m & 3])


def test_site_words_are_uniform():
    """Bits of the Metropolis words are balanced (5 sigma) across sites and sweeps."""
    seed = inputs.unit_seed(3)
    us = np.array([oracle.metropolis_u(seed, 0, t, c, m) for t in range(4) for c in (0, 1)
                   for m in range(2048)], dtype=np.uint64)
    n = len(us)
    for b in range(32):
        ones = int(((us >> np.uint64(b)) & np.uint64(1)).sum())
        assert abs(ones - n / 2) < 5 * np.sqrt(n / 4), b


# ----------------------------------------------------------- thresholds

@pytest.mark.parametrize("beta", [0.0, 1e-12, 0.05, 0.2216544, 0.3, 1 / 2.269185, 0.5, 1.0, 2.0, 5.0, 30.0])
def test_threshold_is_floor_of_boltzmann_factor(beta):
    """Eq. 2: thr = floor(exp(-beta dE) 2^32), checked against a 50-digit evaluation."""
    for dE in (4, 8, 12):
        thr = oracle.threshold(beta, dE)
        with mp.workdps(50):
            x = mp.exp(-mp.mpf(beta) * dE) * mp.mpf(2) ** 32
            exact = int(mp.floor(x))
            frac = x - exact
        if 1e-6 < frac < 1 - 1e-6:  # double rounding cannot move the floor
            assert thr == exact, (beta, dE, thr, exact)
        else:
            assert abs(thr - exact) <= 1
        assert 0 <= thr <= 1 << 32
    for dE in (0, -4, -8, -12):
        assert oracle.threshold(beta, dE) == 1 << 32


def test_threshold_limits_and_accept():
    assert oracle.threshold(0.0, 8) == 1 << 32
    assert oracle.threshold(float("inf"), 4) == 0
    assert oracle.threshold(40.0, 4) == 0
    t = oracle.threshold(0.4, 8)
    assert oracle.accept(0.4, 8, t - 1) and not oracle.accept(0.4, 8, t)
    assert oracle.accept(0.4, 0, 0xFFFFFFFF) and oracle.accept(0.4, -8, 0xFFFFFFFF)


# ------------------------------------------------------------ energies

def _all_states(N):
    idx = np.arange(1 << N, dtype=np.uint64)
    return (1 - 2 * ((idx[:, None] >> np.arange(N, dtype=np.uint64)) & np.uint64(1)).astype(np.int8)).astype(np.int8)


@pytest.mark.parametrize("dims", [(4, 4), (2, 6), (4, 2)])
def test_energy_spectrum_matches_kaufman(dims):
    """The oracle's Eq. 1 energy over all states gives Kaufman's exact Z(beta)."""
    Lx, Ly = dims
    S = _all_states(Lx * Ly)
    E = np.array([oracle.observables(dims, s)[0] for s in S], dtype=np.int64)
    M = S.astype(np.int64).sum(axis=1)
    En, Mn = enumerate_2d(Lx, Ly)
    assert np.array_equal(np.sort(E), np.sort(En))
    for beta in (0.1, 0.3, 0.4406868, 0.6, 1.0):
        lz = log_z_enumerated(E, beta)
        assert abs(lz - float(kaufman_log_z(Ly, Lx, beta))) < 1e-11 * max(1.0, abs(lz))
    assert all(oracle.observables(dims, s)[1] == int(s.sum()) for s in S[::97])


@pytest.mark.parametrize("dims,bonded", [((2, 2, 4), False), ((2, 2, 2), True), ((4, 2, 2), True)])
def test_3d_energy_of_every_state_matches_numpy(dims, bonded):
    """E and M of every state of a tiny simple cubic torus (Ising, or +-J bonds
    as the input generator draws them) against Eq. 1 written out in numpy over
    the three forward bonds of each site."""

    N = int(np.prod(dims))
    packed = inputs.ea_bonds(dims, 1, 77) if bonded else None
    J = (inputs.unpack_bonds(packed, N)[0] if bonded else np.ones((3, N))).astype(np.int64)
    S = (1 - 2 * ((np.arange(1 << N)[:, None] >> np.arange(N)) & 1)).astype(np.int8)
    E = energy(S, J, neighbours(dims))
    for i in range(len(S)):
        assert oracle.observables(dims, S[i], bonds=packed) == (int(E[i]), int(S[i].sum()))


def test_3d_energy_reduces_to_2d_planes():
    """A z-uniform 3D state has E = Lz * E_2D(plane) - N (all z-bonds satisfied)."""
    rng = np.random.default_rng(11)
    for dims in ((4, 4, 2), (4, 6, 4), (2, 2, 2)):
        Lx, Ly, Lz = dims
        for _ in range(5):
            plane = rng.choice(np.array([-1, 1], np.int8), size=Lx * Ly)
            s = np.tile(plane, Lz)
            E3, M3 = oracle.observables(dims, s)
            E2, M2 = oracle.observables((Lx, Ly), plane)
            assert E3 == Lz * E2 - Lx * Ly * Lz and M3 == Lz * M2


def test_ea_energy_symmetries():
    """J = +1 reproduces Ising; J = -1 on the bipartite torus equals Ising of the
    staggered state; a gauge transformation leaves E invariant."""
    rng = np.random.default_rng(5)
    for dims in ((4, 4), (4, 2, 6), (2, 2, 2)):
        N = int(np.prod(dims))
        nd = len(dims)
        coords = np.indices(dims[::-1]).reshape(nd, -1)[::-1]
        stag = (1 - 2 * (coords.sum(axis=0) & 1)).astype(np.int8)
        for _ in range(4):
            s = rng.choice(np.array([-1, 1], np.int8), size=N)
            Jp = inputs.uniform_bonds(dims, 1, +1)[0]
            Jm = inputs.uniform_bonds(dims, 1, -1)[0]
            assert oracle.observables(dims, s, Jp) == oracle.observables(dims, s)
            assert oracle.observables(dims, s, Jm)[0] == oracle.observables(dims, (s * stag).astype(np.int8))[0]
            J = inputs.ea_bonds(dims, 1, int(rng.integers(1 << 30)))[0]
            eps = rng.choice(np.array([-1, 1], np.int8), size=N)
            Jm_ = inputs.unpack_bonds(J, N).astype(np.int64)
            Jg = Jm_.copy()
            for d in range(nd):
                idx = np.arange(N).reshape(dims[::-1])
                nbr = np.roll(idx, -1, axis=nd - 1 - d).reshape(-1)
                Jg[d] = eps * Jm_[d] * eps[nbr]
            Jg = inputs.pack_bonds(Jg.astype(np.int8))
            assert oracle.observables(dims, (s * eps).astype(np.int8), Jg)[0] == oracle.observables(dims, s, J)[0]


@pytest.mark.parametrize("dims,bonded", [((4, 4), False), ((4, 6), True), ((4, 2, 4), False), ((2, 4, 2), True)])
def test_delta_e_is_energy_difference(dims, bonded):
    rng = np.random.default_rng(9)
    N = int(np.prod(dims))
    J = inputs.ea_bonds(dims, 1, 77)[0] if bonded else None
    for _ in range(3):
        s = rng.choice(np.array([-1, 1], np.int8), size=N)
        E0, _ = oracle.observables(dims, s, J)
        for n in range(N):
            f = s.copy()
            f[n] = -f[n]
            assert oracle.delta_e(dims, s, n, J) == oracle.observables(dims, f, J)[0] - E0


# ------------------------------------------------------- exact dynamics

def test_half_sweep_kernel_is_exactly_stationary():
    """The half-sweep transition built from the oracle's dE and acceptance rule
    keeps the Boltzmann distribution of the 4x4 torus stationary, up to the
    2^-32 quantisation of the acceptance probability."""
    dims = (4, 4)
    N = 16
    beta = 0.37
    S = _all_states(N)
    E = np.array([oracle.observables(dims, s)[0] for s in S], dtype=np.float64)
    pi = np.exp(-beta * (E - E.min()))
    pi /= pi.sum()
    colour = np.array([(n % 4 + n // 4) & 1 for n in range(N)])
    thr = {dE: oracle.threshold(beta, dE) for dE in (4, 8)}
    for c in (0, 1):
        sites = np.nonzero(colour == c)[0]
        P = np.zeros((len(S), len(sites)))
        for i, s in enumerate(S):
            for j, n in enumerate(sites):
                dE = oracle.delta_e(dims, s, int(n))
                P[i, j] = 1.0 if dE <= 0 else thr[dE] / 2.0**32
        new = np.zeros(len(S))
        idx = np.arange(len(S), dtype=np.int64)
        for F in range(1 << len(sites)):
            flip = np.array([(F >> j) & 1 for j in range(len(sites))], dtype=bool)
            prob = np.prod(np.where(flip, P, 1.0 - P), axis=1)
            mask = int(sum(1 << int(sites[j]) for j in range(len(sites)) if flip[j]))
            np.add.at(new, idx ^ mask, pi * prob)
        # each of the 8 sites carries a relative quantisation error below 2^-32 / p_min
        p_min = thr[8] / 2.0**32
        assert np.max(np.abs(new - pi) / pi) < 16 * 2.0**-32 / p_min


def test_half_sweep_kernel_is_exactly_stationary_3d_pmj():
    """The same on a 4 x 2 x 2 +-J cube with the couplings on which the
    checkerboard chain splits into closed classes: every half-sweep still keeps
    the Boltzmann distribution, so the split is a failure of irreducibility,
    not of the update."""
    dims, N, beta = (4, 2, 2), 16, 0.37
    packed = inputs.ea_bonds(dims, 1, inputs.unit_seed(0x5A))
    S = _all_states(N)
    E = np.array([oracle.observables(dims, s, bonds=packed)[0] for s in S], dtype=np.float64)
    pi = np.exp(-beta * (E - E.min()))
    pi /= pi.sum()
    colour = np.array([(n % 4 + (n // 4) % 2 + n // 8) & 1 for n in range(N)])
    thr = {dE: oracle.threshold(beta, dE) for dE in (4, 8, 12)}
    for c in (0, 1):
        sites = np.nonzero(colour == c)[0]
        P = np.zeros((len(S), len(sites)))
        for i, s in enumerate(S):
            for j, n in enumerate(sites):
                dE = oracle.delta_e(dims, s, int(n), bonds=packed)
                P[i, j] = 1.0 if dE <= 0 else thr[dE] / 2.0**32
        new = np.zeros(len(S))
        idx = np.arange(len(S), dtype=np.int64)
        for F in range(1 << len(sites)):
            flip = np.array([(F >> j) & 1 for j in range(len(sites))], dtype=bool)
            prob = np.prod(np.where(flip, P, 1.0 - P), axis=1)
            mask = int(sum(1 << int(sites[j]) for j in range(len(sites)) if flip[j]))
            np.add.at(new, idx ^ mask, pi * prob)
        assert np.max(np.abs(new - pi) / pi) < 16 * 2.0**-32 / (thr[12] / 2.0**32)


def test_beta_zero_flips_every_spin():
    """beta = 0: every proposal is accepted, so each sweep maps s -> -s."""
    for dims in ((8, 6), (4, 4, 6)):
        s = oracle.init_hot(dims, 99)
        s0 = s.copy()
        E0, M0 = oracle.observables(dims, s)
        E, M, tE, tM = oracle.sweeps(dims, s, 0.0, 3, 99)
        assert np.array_equal(s, -s0)
        assert list(tE) == [E0] * 3 and list(tM) == [-M0, M0, -M0]


def test_beta_infinite_freezes_ground_state():
    for dims in ((8, 8), (4, 4, 4)):
        s = np.ones(int(np.prod(dims)), np.int8)
        E, M, tE, tM = oracle.sweeps(dims, s, float("inf"), 5, 3)
        assert (s == 1).all() and M == s.size


def test_acceptance_is_strict_at_the_threshold():
    """u = thr is rejected and u = thr - 1 accepted (strict u < thr of Eq. 2): a
    cold 8x8 lattice has dE = 8 at every site; beta is tuned so that the
    threshold lands exactly on the u of site 0."""
    dims, seed = (8, 8), 4242
    u0 = oracle.metropolis_u(seed, 0, 0, 0, 0)
    assert 1000 < u0 < (1 << 32) - 1000
    for target, flips in ((u0, False), (u0 + 1, True)):
        lo, hi = 0.0, 10.0
        for _ in range(200):  # bisection on the monotone threshold
            mid = 0.5 * (lo + hi)
            if oracle.threshold(mid, 8) > target:
                lo = mid
            else:
                hi = mid
        beta = hi if oracle.threshold(hi, 8) == target else lo
        assert oracle.threshold(beta, 8) == target
        s = np.ones(64, np.int8)
        oracle.sweeps(dims, s, beta, 1, seed)
        assert (s[0] == -1) == flips


def test_trace_matches_recomputed_observables():
    for dims, bonds in (((16, 8), None), ((6, 4, 8), None), ((4, 4, 4), inputs.ea_bonds((4, 4, 4), 1, 5)[0])):
        s = oracle.init_hot(dims, 1234, 3)
        E, M, tE, tM = oracle.sweeps(dims, s, 0.35, 20, 1234, stream=3, bonds=bonds)
        assert (E, M) == oracle.observables(dims, s, bonds)
        assert tE[-1] == E and tM[-1] == M


def test_result_independent_of_thread_count():
    code = textwrap.dedent(
        """
        import sys, numpy as np
        sys.path.insert(0, sys.argv[1])
        import oracle
        s = oracle.init_hot((64, 32), 42)
        E, M, tE, tM = oracle.sweeps((64, 32), s, 0.44, 30, 42)
        print(E, M, int(tE.sum()), int(np.abs(s.astype(np.int64) * np.arange(s.size)).sum()))
        """)
    outs = set()
    for nt in ("1", "3"):
        env = dict(os.environ, OMP_NUM_THREADS=nt)
        r = subprocess.run([sys.executable, "-c", code, ROOT], capture_output=True, text=True, env=env, timeout=300)
        assert r.returncode == 0, r.stderr
        outs.add(r.stdout)
    assert len(outs) == 1


def test_hot_start_is_balanced():
    s = oracle.init_hot((128, 128), inputs.unit_seed(1))
    n = s.size
    assert abs(int((s < 0).sum()) - n / 2) < 5 * np.sqrt(n / 4)


# ------------------------------------------------ statistical physics

@pytest.mark.parametrize("T", [1.5, 2.269185, 3.5])
def test_long_run_matches_enumeration_L4(T):
    """<E> and <|M|> of the 4x4 torus match exact enumeration (4 sigma, binned)."""
    dims, beta = (4, 4), 1.0 / T
    s = oracle.init_hot(dims, 2024)
    _, _, tE, tM = oracle.sweeps(dims, s, beta, 60000, 2024)
    En, Mn = enumerate_2d(4, 4)
    e, am, _ = exact_averages(En, Mn, beta)
    me, ee = binned_mean_err(tE[1000:])
    mm, em = binned_mean_err(np.abs(tM[1000:]))
    assert abs(me - e) < 4 * ee, (me, e, ee)
    assert abs(mm - am) < 4 * em, (mm, am, em)


def test_long_run_matches_kaufman_L16():
    """<E> of the 16x16 torus at T = 2.5 matches Kaufman's exact finite-size value."""
    dims, beta = (16, 16), 1.0 / 2.5
    s = oracle.init_hot(dims, 77)
    _, _, tE, _ = oracle.sweeps(dims, s, beta, 30000, 77)
    me, ee = binned_mean_err(tE[2000:])
    ex = kaufman_energy(16, 16, beta)
    assert abs(me - ex) < 4 * ee, (me, ex, ee)


@pytest.mark.parametrize("T", [1.5, 2.269185, 3.5])
def test_kaufman_variance_matches_enumeration(T):
    """Var(E) from the second beta-derivative of Kaufman's ln Z equals the
    variance over all 2^16 states of the 4x4 torus."""
    En, Mn = enumerate_2d(4, 4)
    e, _, e2 = exact_averages(En, Mn, 1.0 / T)
    v = kaufman_energy_variance(4, 4, 1.0 / T)
    assert abs(v - (e2 - e * e)) < 1e-9 * v, (v, e2 - e * e)


@pytest.mark.parametrize("T", [2.269185, 2.5])
def test_long_run_specific_heat_matches_kaufman_L16(T):
    """The paper finds its 2D runs consistent with the exact internal energy and
    specific heat of the finite lattice (Sec. 4): c = beta^2 Var(E) / N of a
    16x16 run matches Kaufman's value (4 jackknife sigma)."""
    dims, beta = (16, 16), 1.0 / T
    s = oracle.init_hot(dims, 3)
    _, _, tE, _ = oracle.sweeps(dims, s, beta, 100000, 3)
    v, ev = binned_variance_err(tE[5000:])
    ex = kaufman_energy_variance(16, 16, beta)
    assert abs(v - ex) < 4 * ev, (v, ex, ev)
    c, cex = beta ** 2 * v / 256, beta ** 2 * ex / 256
    assert abs(c - cex) < 0.05 * cex, (c, cex)


@pytest.mark.parametrize("T,cold", [(3.0, False), (2.0, True)])
def test_onsager_energy_large_lattice(T, cold):
    """u(T) of a 96x96 lattice (L >> correlation length) matches Onsager."""
    dims = (96, 96)
    s = np.ones(96 * 96, np.int8) if cold else oracle.init_hot(dims, 5)
    _, _, tE, _ = oracle.sweeps(dims, s, 1.0 / T, 2500, 5)
    me, ee = binned_mean_err(tE[500:] / s.size, nbins=20)
    assert abs(me - onsager_energy_per_spin(T)) < 4 * ee + 2e-3, (me, onsager_energy_per_spin(T), ee)


def test_3d_energy_matches_the_high_temperature_series():
    """3D Ising at small beta against the high-temperature expansion of the
    simple cubic lattice: with t = tanh(beta), ln Z / N = ln 2 + 3 ln cosh(beta)
    + 3 t^4 + O(t^6) (3N bonds; the smallest closed graphs are the 3N
    plaquettes), so u = E / N = -3 t - 12 t^3 (1 - t^2) + O(t^5).  At
    beta = 0.05 the plaquette term (1.5e-3) is about nine standard errors of
    8000 sweeps, so a lattice that misses a neighbour or a bond fails."""
    dims, beta = (32, 32, 32), 0.05
    t = np.tanh(beta)
    series = -3 * t - 12 * t ** 3 * (1 - t * t)
    s = oracle.init_hot(dims, 11)
    _, _, tE, _ = oracle.sweeps(dims, s, beta, 8200, 11)
    me, ee = binned_mean_err(tE[200:] / s.size, nbins=20)
    assert abs(me - series) < 4 * ee + 2e-5, (me, series, ee)
    assert abs(me - (-3 * t)) > 4 * ee  # the plaquette term is seen


def test_3d_energy_matches_the_low_temperature_series():
    """3D Ising deep in the ordered phase against the low-temperature expansion
    of the simple cubic lattice.  From the all-up ground state (E = -3N), the
    excitations up to 14 broken bonds are: one flipped spin (6 broken bonds, N
    ways), two flipped neighbours (10, 3N ways), two flipped non-neighbours (12,
    N(N-1)/2 - 3N ways) and a flipped path of three sites (14, 15N ways: two of
    the centre's six neighbours).  With x = exp(-2 beta) the logarithm of the
    polymer sum gives ln Z / N = 3 beta + x^6 + 3 x^10 - 7/2 x^12 + 15 x^14 +
    O(x^16), hence u = E / N = -3 + 12 e^(-12 beta) + 60 e^(-20 beta)
    - 84 e^(-24 beta) + 420 e^(-28 beta).  At beta = 0.6 from a cold start the
    single-flip term (9.0e-3) is far beyond the error bar and the neighbour-pair
    term (3.7e-4) is several standard errors, so a sweep that drops or doubles
    a neighbour, or maps dE = 12 to the wrong threshold, fails."""
    dims, beta = (24, 24, 24), 0.6
    N = 24 ** 3
    e = lambda a: np.exp(-a * beta)
    series = -3 + 12 * e(12) + 60 * e(20) - 84 * e(24) + 420 * e(28)
    s = np.ones(N, np.int8)
    _, _, tE, _ = oracle.sweeps(dims, s, beta, 8200, 23)
    me, ee = binned_mean_err(tE[200:] / N, nbins=20)
    assert abs(me - series) < 4 * ee + 1e-5, (me, series, ee)
    assert abs(me - (-3 + 12 * e(12))) > 4 * ee  # the neighbour-pair excitations are seen
    assert abs(me + 3) > 100 * ee  # single flips are seen


@pytest.mark.parametrize("beta", [0.221654, 0.4])
def test_3d_long_run_matches_enumeration_4x2x2(beta):
    """<E> and <|M|> of a 4 x 2 x 2 simple cubic torus (16 sites, every state
    enumerated in numpy; the extent-2 axes join each pair by two bonds) match a
    long oracle run within 4 binned sigma.  The checkerboard chain from a hot
    start cannot leave its class; the states outside it (eight zero-field
    two-state cycles) carry under 1e-4 of the Boltzmann weight here."""

    dims, N = (4, 2, 2), 16
    J = inputs.unpack_bonds(inputs.uniform_bonds(dims, 1, +1), N)[0].astype(np.int64)
    S = 1 - 2 * ((np.arange(1 << N)[:, None] >> np.arange(N)) & 1)
    E, M = energy(S, J, neighbours(dims)), S.sum(axis=1)
    w = np.exp(-beta * (E - E.min()))
    s = oracle.init_hot(dims, 11)
    start = int(((s < 0).astype(np.int64) << np.arange(N)).sum())  # bit n set iff spin n is -1
    assert w[~reachable(dims, J, start)].sum() / w.sum() < 1e-4
    _, _, tE, tM = oracle.sweeps(dims, s, beta, 100000, 11)
    me, ee = binned_mean_err(tE[2000:])
    mm, em = binned_mean_err(np.abs(tM[2000:]))
    e, am = (w * E).sum() / w.sum(), (w * np.abs(M)).sum() / w.sum()
    assert abs(me - e) < 4 * ee, (me, e, ee)
    assert abs(mm - am) < 4 * em, (mm, am, em)


@pytest.mark.parametrize("T", [1.5, 2.269185, 3.5])
def test_energy_histogram_matches_exact_density_of_states_L4(T):
    """The whole energy distribution of a 4 x 4 run, not only its mean: energies
    of every 20th sweep (about ten autocorrelation times apart) against
    P(E) = g(E) e^(-beta E) / Z with g(E) counted over all 2^16 states (Pearson
    chi-square).  The same samples fail against the distribution at a beta 5%
    off (p <= 1e-8 at all three temperatures; 3% off is resolved at T = 2.27
    and 3.5, not in the mostly frozen run at T = 1.5)."""
    En, _ = enumerate_2d(4, 4)
    levels, g = np.unique(En, return_counts=True)

    def probs(b):
        w = g * np.exp(-b * (levels - levels.min()))
        return w / w.sum()

    s = oracle.init_hot((4, 4), 1)
    _, _, tE, _ = oracle.sweeps((4, 4), s, 1.0 / T, 200000, 1)
    samples = tE[1000::20]
    assert energy_histogram_pvalue(levels, probs(1.0 / T), samples) > 1e-3
    assert energy_histogram_pvalue(levels, probs(1.05 / T), samples) < 1e-4


def test_energy_histogram_matches_exact_density_of_states_3d_4x2x2():
    """The same on the 4 x 2 x 2 simple cubic torus at the bulk critical coupling."""

    dims, N, beta = (4, 2, 2), 16, 0.221654
    J = inputs.unpack_bonds(inputs.uniform_bonds(dims, 1, +1), N)[0].astype(np.int64)
    S = 1 - 2 * ((np.arange(1 << N)[:, None] >> np.arange(N)) & 1)
    levels, g = np.unique(energy(S, J, neighbours(dims)), return_counts=True)
    w = g * np.exp(-beta * (levels - levels.min()))
    s = oracle.init_hot(dims, 2)
    _, _, tE, _ = oracle.sweeps(dims, s, beta, 200000, 2)
    assert energy_histogram_pvalue(levels, w / w.sum(), tE[1000::20]) > 1e-3


def test_acceptance_rate_matches_threshold():
    """Across a run, the flip frequency of colour-0 sites with dE = 8 and dE = 4
    equals thr/2^32 within 5 sigma (the sweep applies the rule of Eq. 2)."""
    dims, beta, seed = (32, 32), 0.3, 8
    s = oracle.init_hot(dims, seed)
    oracle.sweeps(dims, s, beta, 20, seed)
    colour0 = [n for n in range(s.size) if ((n % 32) + n // 32) % 2 == 0]
    counts = {4: [0, 0], 8: [0, 0]}
    for t in range(20, 60):
        before = s.copy()
        dEs = [(n, oracle.delta_e(dims, before, n)) for n in colour0]
        # colour-0 sites are not touched by the colour-1 half, so after the sweep
        # they hold the outcome of the colour-0 half-sweep
        oracle.sweeps(dims, s, beta, 1, seed, sweep0=t)
        for n, dE in dEs:
            if dE in counts:
                counts[dE][0] += 1
                counts[dE][1] += int(s[n] != before[n])
    for dE, (n, f) in counts.items():
        p = oracle.threshold(beta, dE) / 2.0**32
        assert n > 100
        assert abs(f - n * p) < 5 * np.sqrt(n * p * (1 - p)) + 1, (dE, n, f, p)


# -------------------------------------------------------- EA dynamics

def test_ea_gauge_invariance_of_trajectories():
    """s -> eps s, J_ij -> eps_i J_ij eps_j leaves every dE unchanged, so the
    gauge-transformed run is exactly the transformed trajectory."""
    rng = np.random.default_rng(3)
    dims = (6, 4, 4)
    N = int(np.prod(dims))
    J = inputs.ea_bonds(dims, 1, 31)[0]
    s = oracle.init_hot(dims, 8)
    eps = rng.choice(np.array([-1, 1], np.int8), size=N)
    Jm = inputs.unpack_bonds(J, N).astype(np.int64)
    idx = np.arange(N).reshape(dims[::-1])
    Jg = np.stack([eps * Jm[d] * eps[np.roll(idx, -1, axis=2 - d).reshape(-1)] for d in range(3)])
    Jg = inputs.pack_bonds(Jg.astype(np.int8))
    g = (s * eps).astype(np.int8)
    E1, M1, tE1, _ = oracle.sweeps(dims, s, 0.7, 25, 8, bonds=J)
    E2, M2, tE2, _ = oracle.sweeps(dims, g, 0.7, 25, 8, bonds=Jg)
    assert np.array_equal(g, (s * eps).astype(np.int8))
    assert np.array_equal(tE1, tE2)


def _ea_setup(dims, nsamples, seed, ferro=False):
    bonds = inputs.uniform_bonds(dims, nsamples, +1) if ferro else inputs.ea_bonds(dims, nsamples, seed)
    words = oracle.ea_init_hot(dims, nsamples, seed)
    pi = np.tile(np.arange(32, dtype=np.uint8), (nsamples, 1))
    return bonds, words, pi, pi.copy()


@pytest.mark.parametrize("ferro", [False, True])
def test_msc_replicas_equal_scalar_runs(ferro):
    """Without exchange, the replica in slot j of the multi-spin coded run is
    exactly the int8 run at beta[temp_of_slot[j]] started from bit j (the same u
    drives both); the slot map starts as a random permutation."""
    dims, ns, seed = (4, 4, 6), 2, 1357
    betas = inputs.geometric_ladder(0.5, 5.0)
    bonds, words, pi, tau = _ea_setup(dims, ns, seed, ferro)
    rng = np.random.default_rng(4)
    for i in range(ns):
        pi[i] = rng.permutation(32).astype(np.uint8)
        tau[i][pi[i]] = np.arange(32, dtype=np.uint8)
    w0 = words.copy()
    oracle.ea_sweeps(dims, words, bonds, betas, pi, tau, 7, seed)
    for i in range(ns):
        for j in (0, 5, 17, 31):
            s = (1 - 2 * ((w0[i] >> np.uint32(j)) & np.uint32(1)).astype(np.int8)).astype(np.int8)
            oracle.sweeps(dims, s, betas[pi[i][j]], 7, seed, stream=i, bonds=None if ferro else bonds[i],
                          msc_u_words=True)
            got = (1 - 2 * ((words[i] >> np.uint32(j)) & np.uint32(1)).astype(np.int8)).astype(np.int8)
            assert np.array_equal(got, s), (i, j)


def test_exchange_with_equal_betas_always_accepts():
    dims, ns, seed = (4, 4, 4), 2, 99
    betas = np.full(32, 0.8)
    bonds, words, pi, tau = _ea_setup(dims, ns, seed)
    acc = np.zeros((ns, 32), np.int64)
    oracle.ea_sweeps(dims, words, bonds, betas, pi, tau, 40, seed, exchange_every=10, acc=acc)
    # 4 steps: even pairs (16) at e = 0, 2 and odd pairs (15) at e = 1, 3
    assert acc[:, 0::2].sum(axis=1).tolist() == [32, 32] and acc[:, 1::2].sum(axis=1).tolist() == [30, 30]
    for i in range(ns):
        assert sorted(pi[i].tolist()) == list(range(32))
        assert all(tau[i][pi[i][j]] == j for j in range(32))


def test_exchange_keeps_permutation_and_energy_order():
    """With a wide ladder the slot maps stay inverse permutations and the energy of
    each temperature's replica is that of the slot assigned to it."""
    dims, ns, seed = (4, 4, 4), 3, 2468
    betas = inputs.geometric_ladder(0.2, 2.0)
    bonds, words, pi, tau = _ea_setup(dims, ns, seed)
    acc = np.zeros((ns, 32), np.int64)
    oracle.ea_sweeps(dims, words, bonds, betas, pi, tau, 200, seed, exchange_every=10, acc=acc)
    assert acc.sum() > 0
    for i in range(ns):
        assert sorted(pi[i].tolist()) == list(range(32))
        assert all(tau[i][pi[i][j]] == j for j in range(32))
    E, _ = oracle.ea_observables(dims, words, bonds)
    # low temperatures hold lower energies on average after equilibration
    Et = np.array([[E[i][tau[i][t]] for t in range(32)] for i in range(ns)])
    assert Et[:, :8].mean() < Et[:, -8:].mean()


def test_exchange_acceptance_follows_the_replica_exchange_rule():
    """Every attempted pair with D = (beta_k - beta_k+1)(E_k - E_k+1) >= 0 swaps,
    and pairs with D < 0 swap with total frequency sum(exp(D)) within 5 sigma.
    The energies before each exchange come from an identical run without
    exchange (the dynamics is a deterministic function of the counters; both
    runs draw a u per slot, the default of runs with exchange)."""
    dims, ns, seed, X = (4, 4, 4), 8, 97531, 10
    betas = inputs.geometric_ladder(0.6, 3.0)
    bonds, words, pi, tau = _ea_setup(dims, ns, seed)
    must, expect, var, got = 0, 0.0, 0.0, 0
    for e in range(30):
        w2, pi2, tau2 = words.copy(), pi.copy(), tau.copy()
        oracle.ea_sweeps(dims, w2, bonds, betas, pi2, tau2, X, seed, sweep0=X * e, exchange_every=0, u_per_slot=True)
        Eslot, _ = oracle.ea_observables(dims, w2, bonds)
        before = tau.copy()
        oracle.ea_sweeps(dims, words, bonds, betas, pi, tau, X, seed, sweep0=X * e, exchange_every=X)
        assert np.array_equal(words, w2)
        for i in range(ns):
            for k in range(e & 1, 31, 2):
                D = (betas[k] - betas[k + 1]) * float(Eslot[i][before[i][k]] - Eslot[i][before[i][k + 1]])
                swapped = tau[i][k] == before[i][k + 1] and tau[i][k + 1] == before[i][k]
                if not swapped:
                    assert tau[i][k] == before[i][k] and tau[i][k + 1] == before[i][k + 1]
                if D >= 0:
                    assert swapped
                    must += 1
                else:
                    p = float(np.exp(D))
                    expect += p
                    var += p * (1 - p)
                    got += int(swapped)
    assert must > 50 and var > 50
    assert abs(got - expect) < 5 * np.sqrt(var), (got, expect, var)
