"""Pins of the oracle's disorder-parallel multi-spin coded ladder (Sec. 4: many
disorder realisations updated at once, the bits of a word being different
samples that share one random number; here 32 samples per group share the
site's u at each temperature, and a sample's 32 temperatures draw independent
u, so replica exchange within a sample sees independent replicas).

* Without exchange, every (sample, temperature) replica is exactly the plain
  int8 Metropolis run of that sample at that temperature with the same random
  words (the scalar sweep is pinned to enumeration, Kaufman and Onsager).
* With exchange, every sample's ladder is Boltzmann-distributed at every
  temperature: 16 samples of a 4 x 4 +-J lattice with 16 different coupling
  sets, eight per group (so they share u), against the exact averages of each
  sample's own couplings from an enumeration of all 2^16 states in numpy.
* The same on the 3D model the EA batches run: 8 samples of a 4 x 2 x 2 +-J
  cube, each sample's couplings first checked to give an irreducible
  checkerboard chain (an extent of 2 can split it into closed classes).
* The exchange follows the replica-exchange rule: pairs with
  D = (beta_k - beta_k+1)(E_k - E_k+1) >= 0 always swap, the others with total
  frequency sum(exp(D)).
"""

from __future__ import annotations

import numpy as np

import oracle
from exact_lattice import energy, neighbours, reachable
from exact_ising import binned_mean_err
from paper_1006_3865_gb300 import inputs

DIMS = (4, 4)
N = 16


def _bit(words, t):
    return (1 - 2 * ((words >> np.uint32(t)) & np.uint32(1)).astype(np.int64)).astype(np.int8)


def test_groups_keep_replica_pairs_apart():
    assert [oracle.ea_dp_group(s) for s in range(6)] == [0, 1, 0, 1, 0, 1]
    assert oracle.ea_dp_group(64) == 2 and oracle.ea_dp_group(129) == 5


def test_replicas_without_exchange_equal_scalar_runs():
    """Bit t of sample s equals the int8 run at beta_t with the words of stream
    32 g(s) + t, from the same start, for 2D and 3D samples."""
    for dims, ns in (((4, 6), 5), ((4, 4, 2), 3)):
        seed = inputs.unit_seed(0xD1)
        betas = inputs.geometric_ladder(0.3, 3.0)
        bonds = inputs.ea_bonds(dims, ns, inputs.unit_seed(0xD2))
        words = oracle.ea_init_hot(dims, ns, seed)
        w0 = words.copy()
        oracle.ea_dp_sweeps(dims, words, bonds, betas, 9, seed)
        for s in range(ns):
            for t in (0, 7, 19, 31):
                x = _bit(w0[s], t).copy()
                oracle.sweeps(dims, x, betas[t], 9, seed, stream=32 * oracle.ea_dp_group(s) + t, bonds=bonds[s],
                              msc_u_words=True)
                assert np.array_equal(_bit(words[s], t), x), (dims, s, t)


def _exact_energies(J):
    """Exact <E> at each of the ladder's temperatures for one 4 x 4 sample; J[d][n]."""
    n = np.arange(N)
    x, y = n % 4, n // 4
    nb = [(x + 1) % 4 + 4 * y, x + 4 * ((y + 1) % 4)]
    states = 1 - 2 * ((np.arange(1 << N)[:, None] >> np.arange(N)) & 1)
    E = -sum((J[d] * states * states[:, nb[d]]).sum(axis=1) for d in range(2))
    betas = inputs.geometric_ladder(0.5, 3.0)
    w = np.exp(-np.outer(betas, E - E.min()))
    return (w * E).sum(axis=1) / w.sum(axis=1)


def test_ladder_with_exchange_is_boltzmann_for_every_sample():
    ns, X, burn, meas = 16, 10, 100, 1500
    seed = inputs.unit_seed(0xD3)
    bonds = inputs.ea_bonds(DIMS, ns, inputs.unit_seed(0xD4))
    J = inputs.unpack_bonds(bonds, N).astype(np.int64)  # [sample][d][n]
    betas = inputs.geometric_ladder(0.5, 3.0)
    words = oracle.ea_init_hot(DIMS, ns, seed)
    series = np.zeros((meas, ns, 32))
    acc = np.zeros((ns, 32), np.int64)
    for it in range(burn + meas):
        oracle.ea_dp_sweeps(DIMS, words, bonds, betas, X, seed, sweep0=X * it, exchange_every=X, acc=acc)
        if it >= burn:
            E, _ = oracle.ea_observables(DIMS, words, bonds)  # bit t: the configuration at temperature t
            series[it - burn] = E
    assert acc.sum() > 0
    z = np.zeros((ns, 32))
    for s in range(ns):
        exact = _exact_energies(J[s])
        for t in range(32):
            m, e = binned_mean_err(series[:, s, t], nbins=15)
            z[s, t] = (m - exact[t]) / max(e, 1e-3)
    assert np.all(np.abs(z) < 5.5), np.round(z, 1)
    assert np.mean(z ** 2) < 1.6, np.mean(z ** 2)


def test_3d_ladder_with_exchange_is_boltzmann_for_every_sample():

    dims, n_sites, ns, X, burn, meas = (4, 2, 2), 16, 8, 10, 100, 1500
    seed = inputs.unit_seed(0xD3)
    bonds = inputs.ea_bonds(dims, ns, inputs.unit_seed(0xD6))
    J = inputs.unpack_bonds(bonds, n_sites).astype(np.int64)  # [sample][d][n]
    for s in range(ns):  # one class: every state reachable from one start (all states are recurrent)
        assert reachable(dims, J[s], 0).all(), s
    betas = inputs.geometric_ladder(0.5, 3.0)
    words = oracle.ea_init_hot(dims, ns, seed)
    series = np.zeros((meas, ns, 32))
    acc = np.zeros((ns, 32), np.int64)
    for it in range(burn + meas):
        oracle.ea_dp_sweeps(dims, words, bonds, betas, X, seed, sweep0=X * it, exchange_every=X, acc=acc)
        if it >= burn:
            series[it - burn] = oracle.ea_observables(dims, words, bonds)[0]
    assert acc.sum() > 0
    S = 1 - 2 * ((np.arange(1 << n_sites)[:, None] >> np.arange(n_sites)) & 1)
    nb = neighbours(dims)
    z = np.zeros((ns, 32))
    for s in range(ns):
        E = energy(S, J[s], nb)
        w = np.exp(-np.outer(betas, E - E.min()))
        exact = (w * E).sum(axis=1) / w.sum(axis=1)
        for t in range(32):
            m, e = binned_mean_err(series[:, s, t], nbins=15)
            z[s, t] = (m - exact[t]) / max(e, 1e-3)
    assert np.all(np.abs(z) < 5.5), np.round(z, 1)
    assert np.mean(z ** 2) < 1.6, np.mean(z ** 2)


def test_exchange_follows_the_replica_exchange_rule():
    dims, ns, X = (4, 4, 4), 8, 10
    seed = inputs.unit_seed(0xD5)
    betas = inputs.geometric_ladder(0.6, 3.0)
    bonds = inputs.ea_bonds(dims, ns, inputs.unit_seed(0xD6))
    words = oracle.ea_init_hot(dims, ns, seed)
    must, expect, var, got = 0, 0.0, 0.0, 0
    for e in range(30):
        w2 = words.copy()
        oracle.ea_dp_sweeps(dims, w2, bonds, betas, X, seed, sweep0=X * e, exchange_every=0)
        E, _ = oracle.ea_observables(dims, w2, bonds)
        acc = np.zeros((ns, 32), np.int64)
        oracle.ea_dp_sweeps(dims, words, bonds, betas, X, seed, sweep0=X * e, exchange_every=X, acc=acc)
        for s in range(ns):
            for k in range(32):
                swapped = acc[s, k] == 1
                if k % 2 != e % 2 or k == 31:
                    assert not swapped
                    continue
                b_k, b_k1 = _bit(w2[s], k), _bit(w2[s], k + 1)
                # an accepted pair swaps the two configurations, a rejected one keeps them
                assert np.array_equal(_bit(words[s], k), b_k1 if swapped else b_k)
                assert np.array_equal(_bit(words[s], k + 1), b_k if swapped else b_k1)
                D = (betas[k] - betas[k + 1]) * float(E[s, k] - E[s, k + 1])
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
