"""Pins of the oracle's double-checkerboard sweep with generalised multi-hit
(Sec. 3): the special case beta = 0, a plain restatement of the update order on
tiny lattices, exact stationarity of one tile-parity / colour step, long runs
against exact enumeration (2D, and the 3D 4 x 2 x 2 torus) and Kaufman's
finite-lattice energy, and the 32 x 32 decomposition of Fig. 1 from its text
fixture under golden/."""

from __future__ import annotations

from pathlib import Path

import numpy as np
import pytest

import oracle
from exact_lattice import energy, neighbours
from exact_ising import binned_mean_err, enumerate_2d, exact_averages, kaufman_energy


def _coords(dims, n):
    x = n % dims[0]
    y = (n // dims[0]) % dims[1]
    z = n // (dims[0] * dims[1]) if len(dims) == 3 else 0
    return x, y, z


def _restated(dims, s, tile, hits, beta, nsweeps, seed, stream=0):
    """The procedure of Sec. 3 written out site by site: tiles of parity 0 then
    1; within them `hits` times colour 0 then colour 1; u from the purpose-4
    plane word of the site at counter sweep * hits + hit."""
    N = s.size
    nd = len(dims)
    words = (dims[0] + 63) // 64
    thr = {dE: oracle.threshold(beta, dE) for dE in (4, 8, 12)}
    E, M = oracle.observables(dims, s)
    tE, tM = [], []
    for t in range(nsweeps):
        for P in (0, 1):
            for h in range(hits):
                for c in (0, 1):
                    for n in range(N):
                        x, y, z = _coords(dims, n)
                        if (x + y + z) & 1 != c:
                            continue
                        tp = x // tile[0] + y // tile[1] + (z // tile[2] if nd == 3 else 0)
                        if tp & 1 != P:
                            continue
                        nb = []
                        for d, ext in enumerate(dims):
                            for step in (-1, 1):
                                q = [x, y, z][:nd]
                                q[d] = (q[d] + step) % ext
                                m = q[0] + dims[0] * (q[1] + (dims[1] * q[2] if nd == 3 else 0))
                                nb.append(int(s[m]))
                        dE = 2 * int(s[n]) * sum(nb)
                        row = n // dims[0]
                        key = 32 * (x // 64 + words * row) + (x % 64) // 2
                        u = oracle.site_word(seed, stream, t * hits + h, c, 4, key)
                        if dE <= 0 or u < thr[dE]:
                            M -= 2 * int(s[n])
                            E += dE
                            s[n] = -s[n]
        tE.append(E)
        tM.append(M)
    return E, M, np.array(tE), np.array(tM)


@pytest.mark.parametrize("hits", [1, 2, 3])
def test_beta_zero_flips_every_site_hits_times(hits):
    for dims, tile in (((8, 6), (2, 3)), ((4, 4, 8), (2, 2, 4))):
        s = oracle.init_hot(dims, 5)
        s0 = s.copy()
        oracle.sweeps_dc(dims, s, tile, hits, 0.0, 1, 5)
        assert np.array_equal(s, s0 if hits % 2 == 0 else -s0)


@pytest.mark.parametrize("dims,tile,hits,beta", [((8, 8), (2, 2), 1, 0.44), ((8, 8), (4, 2), 3, 0.3),
                                                 ((6, 4), (3, 2), 2, 0.5), ((4, 4, 4), (2, 2, 2), 2, 0.25)])
def test_matches_restated_procedure(dims, tile, hits, beta):
    s1 = oracle.init_hot(dims, 21, 2)
    s2 = s1.copy()
    a = oracle.sweeps_dc(dims, s1, tile, hits, beta, 3, 21, stream=2)
    b = _restated(dims, s2, tile, hits, beta, 3, 21, stream=2)
    assert np.array_equal(s1, s2)
    assert a[0] == b[0] and a[1] == b[1]
    assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])


def test_one_step_is_exactly_stationary():
    """Updating the colour-c sites of the parity-P tiles of a 4x4 torus with 2x2
    tiles (an independent set) keeps the Boltzmann distribution stationary, up
    to the 2^-32 quantisation of the acceptance probability."""
    dims, N, beta = (4, 4), 16, 0.41
    S = ((np.arange(1 << N)[:, None] >> np.arange(N)) & 1).astype(np.int8) * -2 + 1
    E = np.array([oracle.observables(dims, s)[0] for s in S], dtype=np.float64)
    pi = np.exp(-beta * (E - E.min()))
    pi /= pi.sum()
    thr = {dE: oracle.threshold(beta, dE) for dE in (4, 8)}
    for P in (0, 1):
        for c in (0, 1):
            sites = [n for n in range(N) if (n % 4 + n // 4) & 1 == c and ((n % 4) // 2 + (n // 4) // 2) & 1 == P]
            assert len(sites) == 4
            prob = np.zeros((len(S), len(sites)))
            for i, s in enumerate(S):
                for j, n in enumerate(sites):
                    dE = oracle.delta_e(dims, s, n)
                    prob[i, j] = 1.0 if dE <= 0 else thr[dE] / 2.0**32
            new = np.zeros(len(S))
            idx = np.arange(len(S), dtype=np.int64)
            for F in range(1 << len(sites)):
                flip = np.array([(F >> j) & 1 for j in range(len(sites))], dtype=bool)
                p = np.prod(np.where(flip, prob, 1.0 - prob), axis=1)
                mask = sum(1 << sites[j] for j in range(len(sites)) if flip[j])
                np.add.at(new, idx ^ mask, pi * p)
            assert np.max(np.abs(new - pi) / pi) < 16 * 2.0**-32 / (thr[8] / 2.0**32)


def test_long_run_matches_enumeration_L4():
    dims, beta = (4, 4), 1.0 / 2.269185
    s = oracle.init_hot(dims, 99)
    _, _, tE, tM = oracle.sweeps_dc(dims, s, (2, 2), 3, beta, 40000, 99)
    En, Mn = enumerate_2d(4, 4)
    e, am, _ = exact_averages(En, Mn, beta)
    me, ee = binned_mean_err(tE[1000:])
    mm, em = binned_mean_err(np.abs(tM[1000:]))
    assert abs(me - e) < 4 * ee, (me, e, ee)
    assert abs(mm - am) < 4 * em, (mm, am, em)


def test_long_run_matches_kaufman_L16():
    dims, beta = (16, 16), 1.0 / 2.5
    s = oracle.init_hot(dims, 8)
    _, _, tE, _ = oracle.sweeps_dc(dims, s, (4, 4), 2, beta, 20000, 8)
    me, ee = binned_mean_err(tE[2000:])
    ex = kaufman_energy(16, 16, beta)
    assert abs(me - ex) < 4 * ee, (me, ex, ee)


@pytest.mark.parametrize("hits,beta", [(1, 0.3), (3, 0.221654)])
def test_3d_long_run_matches_enumeration_4x2x2(hits, beta):
    """<E> and <|M|> of the 4 x 2 x 2 simple cubic torus with 2 x 1 x 1 tiles
    (two tiles along every axis) against all 2^16 states enumerated in numpy."""

    dims, N = (4, 2, 2), 16
    S = 1 - 2 * ((np.arange(1 << N)[:, None] >> np.arange(N)) & 1)
    E, M = energy(S, np.ones((3, N), np.int64), neighbours(dims)), S.sum(axis=1)
    w = np.exp(-beta * (E - E.min()))
    s = oracle.init_hot(dims, 5)
    _, _, tE, tM = oracle.sweeps_dc(dims, s, (2, 1, 1), hits, beta, 60000, 5)
    me, ee = binned_mean_err(tE[2000:])
    mm, em = binned_mean_err(np.abs(tM[2000:]))
    e, am = (w * E).sum() / w.sum(), (w * np.abs(M)).sum() / w.sum()
    assert abs(me - e) < 4 * ee, (me, e, ee)
    assert abs(mm - am) < 4 * em, (mm, am, em)


def test_rejects_tilings_without_an_even_tile_count():
    s = oracle.init_hot((12, 8), 1)
    with pytest.raises(ValueError):
        oracle.sweeps_dc((12, 8), s, (4, 2), 1, 0.4, 1, 1)  # three tiles along x
    with pytest.raises(ValueError):
        oracle.sweeps_dc((12, 8), s, (5, 2), 1, 0.4, 1, 1)


def _fig1_map():
    """The phase map of Fig. 1 (Sec. 3), read from its text fixture."""
    path = Path(__file__).parent / "golden" / "fig1_double_checkerboard_32x32.txt"
    rows = [ln.strip() for ln in path.read_text().splitlines() if ln.strip() and not ln.startswith("#")]
    return np.array([[int(ch) for ch in r] for r in rows], dtype=np.int64)


def test_fig1_decomposition_counts():
    """Fig. 1 has B^2 / 2 = 8 even and 8 odd tiles, and the procedure of Sec. 3
    gives each tile T^2 / 2 = 32 sites of either sub-lattice."""
    ph = _fig1_map()
    assert ph.shape == (32, 32)
    for P in (0, 1):
        tiles = [(ty, tx) for ty in range(4) for tx in range(4)
                 if np.all(ph[8 * ty:8 * ty + 8, 8 * tx:8 * tx + 8] // 2 == P)]
        assert len(tiles) == 8
        for ty, tx in tiles:
            blk = ph[8 * ty:8 * ty + 8, 8 * tx:8 * tx + 8] % 2
            assert np.count_nonzero(blk == 0) == 32 and np.count_nonzero(blk == 1) == 32
    # the two sub-lattices of the fine level are each an independent set of the torus
    for c in (0, 1):
        m = (ph % 2) == c
        assert not np.any(m & np.roll(m, 1, 0)) and not np.any(m & np.roll(m, 1, 1))


@pytest.mark.parametrize("hits,beta", [(1, 0.44), (3, 0.3)])
def test_fig1_lattice_follows_the_figure(hits, beta):
    """The oracle's sweep of the 32 x 32 lattice of Fig. 1 with 8 x 8 tiles equals a
    site-by-site sweep in the order the figure's phase map gives."""
    ph = _fig1_map()
    dims = (32, 32)
    s1 = oracle.init_hot(dims, 77, 1)
    s2 = s1.copy()
    a = oracle.sweeps_dc(dims, s1, (8, 8), hits, beta, 2, 77, stream=1)
    thr = {dE: oracle.threshold(beta, dE) for dE in (4, 8)}
    for t in range(2):
        for P in (0, 1):
            for h in range(hits):
                for c in (0, 1):
                    for y, x in zip(*np.nonzero(ph == 2 * P + c)):
                        n = int(x) + 32 * int(y)
                        nb = s2[(x + 1) % 32 + 32 * y] + s2[(x - 1) % 32 + 32 * y] \
                            + s2[x + 32 * ((y + 1) % 32)] + s2[x + 32 * ((y - 1) % 32)]
                        dE = 2 * int(s2[n]) * int(nb)
                        u = oracle.site_word(77, 1, t * hits + h, c, 4, 32 * int(y) + int(x) // 2)
                        if dE <= 0 or u < thr[dE]:
                            s2[n] = -s2[n]
    assert np.array_equal(s1, s2)
    E, M = oracle.observables(dims, s2)
    assert a[0] == E and a[1] == M
