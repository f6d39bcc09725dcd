"""Pins of the oracle's 2D +-J Edwards-Anderson path and of the replica
overlap / Binder observables (Sec. 4: many disorder realisations at once,
multi-spin coded).

* Each replica of the 2D multi-spin coded run is the plain int8 2D EA run at
  its temperature (the same u drives both).
* Long parallel-tempering runs of a 4 x 4 sample reproduce, at several
  temperatures, the exact <E>, <q^2> and <q^4> of two independent replicas,
  computed by enumerating all 2^16 states (energies written from Eq. 1 with
  numpy) and the XOR autocorrelation of the Boltzmann weights (a Walsh-Hadamard
  transform): P(x) = sum_s p(s) p(s ^ x), q = N - 2 popcount(x).
* The overlap's special cases (identical replicas, a globally flipped replica)
  and the Binder cumulant's limits (a two-peaked q gives 1, a Gaussian q 0)."""

from __future__ import annotations

import numpy as np
import pytest

import oracle
from exact_ising import binned_mean_err
from paper_1006_3865_gb300 import inputs


def _ea_setup(dims, nsamples, seed, bonds=None):
    b = inputs.ea_bonds(dims, nsamples, seed) if bonds is None else bonds
    words = oracle.ea_init_hot(dims, nsamples, seed)
    pi = np.tile(np.arange(32, dtype=np.uint8), (nsamples, 1))
    return b, words, pi, pi.copy()


def test_msc_2d_replicas_equal_scalar_runs():
    dims, ns, seed = (6, 4), 2, 4321
    betas = inputs.geometric_ladder(0.5, 5.0)
    bonds, words, pi, tau = _ea_setup(dims, ns, seed)
    rng = np.random.default_rng(5)
    for i in range(ns):
        pi[i] = rng.permutation(32).astype(np.uint8)
        tau[i][pi[i]] = np.arange(32, dtype=np.uint8)
    w0 = words.copy()
    oracle.ea_sweeps(dims, words, bonds, betas, pi, tau, 9, seed)
    for i in range(ns):
        for j in (0, 7, 20, 31):
            s = (1 - 2 * ((w0[i] >> np.uint32(j)) & np.uint32(1)).astype(np.int8)).astype(np.int8)
            oracle.sweeps(dims, s, betas[pi[i][j]], 9, seed, stream=i, bonds=bonds[i], msc_u_words=True)
            got = (1 - 2 * ((words[i] >> np.uint32(j)) & np.uint32(1)).astype(np.int8)).astype(np.int8)
            assert np.array_equal(got, s), (i, j)


def _enumerate_ea_2d(L, J):
    """Energies of all 2^(L*L) states of one 2D +-J sample (J: int8 [2, N])."""
    N = L * L
    idx = np.arange(1 << N, dtype=np.uint32)
    s = (1 - 2 * ((idx[:, None] >> np.arange(N, dtype=np.uint32)) & np.uint32(1)).astype(np.int32))
    n = np.arange(N)
    x, y = n % L, n // L
    right = (x + 1) % L + L * y
    up = x + L * ((y + 1) % L)
    E = -(s * J[0][None, :] * s[:, right]).sum(axis=1) - (s * J[1][None, :] * s[:, up]).sum(axis=1)
    return E.astype(np.int64)


def _wht(v):
    v = v.copy()
    h = 1
    while h < v.size:
        v = v.reshape(-1, 2, h)
        a, b = v[:, 0, :].copy(), v[:, 1, :].copy()
        v[:, 0, :], v[:, 1, :] = a + b, a - b
        v = v.reshape(-1)
        h *= 2
    return v


def _exact_overlap_moments(E, beta, N):
    w = np.exp(-beta * (E - E.min()).astype(np.float64))
    p = w / w.sum()
    P = _wht(_wht(p) ** 2) / p.size  # XOR autocorrelation of p
    x = np.arange(p.size, dtype=np.uint32)
    pc = np.zeros(p.size, np.int64)
    for k in range(N):
        pc += ((x >> np.uint32(k)) & np.uint32(1)).astype(np.int64)
    q = (N - 2 * pc).astype(np.float64)
    Ef = E.astype(np.float64)
    return {"E": float((p * Ef).sum()), "E2": float((p * Ef ** 2).sum()), "q2": float((P * q ** 2).sum()),
            "q4": float((P * q ** 4).sum()), "q8": float((P * q ** 8).sum())}


def test_wht_autocorrelation_matches_direct_sum():
    """The transform identity used by the exact moments, on 2^8 random weights."""
    rng = np.random.default_rng(1)
    p = rng.random(256)
    P = _wht(_wht(p) ** 2) / 256
    direct = np.array([sum(p[s] * p[s ^ x] for s in range(256)) for x in range(256)])
    assert np.allclose(P, direct)


def test_long_run_matches_exact_energy_and_overlap_moments_4x4():
    L, seed = 4, 777
    dims, N = (L, L), L * L
    bonds1 = inputs.ea_bonds(dims, 1, seed)
    bonds = np.concatenate([bonds1, bonds1])  # two replicas of one disorder realisation
    J = inputs.unpack_bonds(bonds1[0], N)
    E_all = _enumerate_ea_2d(L, J)
    betas = inputs.geometric_ladder(0.8, 4.0)
    _, words, pi, tau = _ea_setup(dims, 2, seed, bonds)
    nsweep, burn, X = 24000, 2000, 10
    ts = (0, 9, 18, 31)
    qs, Es = [], []
    sweep = 0
    chunk = 8
    for _ in range(nsweep // chunk):
        oracle.ea_sweeps(dims, words, bonds, betas, pi, tau, chunk, seed, sweep0=sweep, exchange_every=X)
        sweep += chunk
        if sweep > burn:
            qs.append(oracle.ea_overlap(dims, words, tau)[0])
            E, _ = oracle.ea_observables(dims, words, bonds)
            Es.append([E[0][tau[0][t]] for t in range(32)])
    qs = np.array(qs, dtype=np.float64)
    Es = np.array(Es, dtype=np.float64)
    n = len(qs)
    for t in ts:
        ex = _exact_overlap_moments(E_all, betas[t], N)
        # error bar: the binned estimate, but never below the exact standard error of n independent draws
        for series, mean_ex, var_ex in ((Es[:, t], ex["E"], ex["E2"] - ex["E"] ** 2),
                                        (qs[:, t] ** 2, ex["q2"], ex["q4"] - ex["q2"] ** 2),
                                        (qs[:, t] ** 4, ex["q4"], ex["q8"] - ex["q4"] ** 2)):
            m, e = binned_mean_err(series)
            err = max(e, np.sqrt(var_ex / n))
            assert abs(m - mean_ex) < 4 * err, (t, m, mean_ex, e, np.sqrt(var_ex / n))
    # the low-temperature end is ordered in q, the high-temperature end is not
    g = oracle.binder((qs ** 2).mean(axis=0)[None, :], (qs ** 4).mean(axis=0)[None, :])
    assert g[0] > 0.8 and g[31] < 0.5


def test_overlap_special_cases():
    dims = (8, 6)
    N = 48
    words = oracle.ea_init_hot(dims, 2, 3)
    rng = np.random.default_rng(9)
    sot = np.stack([rng.permutation(32), rng.permutation(32)]).astype(np.uint8)
    # identical replicas (the same replica sits in the slots the maps assign): q = N
    same = words.copy()
    for t in range(32):
        bit = (same[0] >> np.uint32(sot[0][t])) & np.uint32(1)
        same[1] = (same[1] & ~np.uint32(1 << int(sot[1][t]))) | (bit << np.uint32(sot[1][t]))
    assert (oracle.ea_overlap(dims, same, sot) == N).all()
    # flipping every spin of one replica negates q; swapping the replicas keeps it
    q = oracle.ea_overlap(dims, words, sot)
    flipped = words.copy()
    flipped[1] = ~flipped[1]
    assert np.array_equal(oracle.ea_overlap(dims, flipped, sot), -q)
    assert np.array_equal(oracle.ea_overlap(dims, words[::-1].copy(), sot[::-1].copy()), q)
    assert ((q - N) % 2 == 0).all() and (np.abs(q) <= N).all()


def test_binder_limits():
    N = 100
    q = np.where(np.random.default_rng(2).random(4000) < 0.5, -N, N).astype(np.float64)
    g = oracle.binder(np.array([[np.mean(q ** 2)]]), np.array([[np.mean(q ** 4)]]))
    assert g[0] == pytest.approx(1.0)
    z = np.random.default_rng(3).standard_normal(400000) * 7.0
    g = oracle.binder(np.array([[np.mean(z ** 2)]]), np.array([[np.mean(z ** 4)]]))
    assert abs(g[0]) < 0.02
