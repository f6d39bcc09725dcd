"""The oracle's multi-spin coded temperature ladder against exact enumeration:
a 4 x 4 +-J lattice (2^16 states), the 32 temperatures of one sample in one
word, 16 independent chains sharing the couplings.  Exact averages come from an
enumeration in numpy over the couplings as the input generator draws them,
independent of the oracle's energy routine, which is checked against the same
enumeration on the final replica states.

* Without exchange every replica is its own Metropolis chain at its
  temperature (the 32 slots share one u per site, which correlates them but
  leaves each one's transition kernel exact): every temperature's mean energy
  matches the Boltzmann average within the statistical error.
* With exchange the shared u matters: replica exchange keeps the product of the
  32 Boltzmann distributions stationary only for independent replicas, and the
  common u makes the replicas of a sample move together, so the marginals drift
  (at the hottest temperature by up to about 1% of E here, about 5 standard
  errors in runs four times longer).  The test bounds that drift.
"""

from __future__ import annotations

import numpy as np

import oracle
from paper_1006_3865_gb300 import inputs

DIMS = (4, 4)
N = 16


def _couplings(seed):
    packed = inputs.ea_bonds(DIMS, 1, seed)
    return packed, inputs.unpack_bonds(packed, N)[0].astype(np.int64)  # J[d][n], d = 0 (x), 1 (y)


def _neighbours():
    n = np.arange(N)
    x, y = n % 4, n // 4
    return np.stack([(x + 1) % 4 + 4 * y, x + 4 * ((y + 1) % 4)])  # forward neighbour along x, y


def _energy(spins, J, nb):
    """E = -sum_n sum_d J[d][n] s_n s_{n + e_d} for spins [..., N] in {+1, -1}."""
    s = spins.astype(np.int64)
    return -sum((J[d] * s * s[..., nb[d]]).sum(axis=-1) for d in range(2))


def _ladder_run(exchange, seed=inputs.unit_seed(0x5A), chains=16, X=10, burn=200, meas=2000):
    """Per-chain mean energy at each temperature, the exact averages, the final
    words and couplings."""
    packed, J = _couplings(seed)
    nb = _neighbours()
    states = 1 - 2 * ((np.arange(1 << N)[:, None] >> np.arange(N)) & 1)
    E_all = _energy(states, J, nb)
    betas = inputs.geometric_ladder(0.5, 3.0)
    w = np.exp(-np.outer(betas, E_all - E_all.min()))
    exact = (w * E_all).sum(axis=1) / w.sum(axis=1)
    bonds = np.repeat(packed, chains, axis=0)  # every chain samples the same couplings
    words = oracle.ea_init_hot(DIMS, chains, seed)
    pi = np.tile(np.arange(32, dtype=np.uint8), (chains, 1))
    tau = pi.copy()
    sums = np.zeros((chains, 32))
    for it in range(burn + meas):
        oracle.ea_sweeps(DIMS, words, bonds, betas, pi, tau, X, seed, sweep0=X * it,
                         exchange_every=X if exchange else 0)
        if it >= burn:
            E, _ = oracle.ea_observables(DIMS, words, bonds)
            sums += np.take_along_axis(E, tau.astype(np.int64), axis=1)  # column t: the replica at temperature t
    return sums / meas, exact, E_all.min(), words, bonds, J, nb


def test_ladder_without_exchange_is_boltzmann_at_every_temperature():
    means, exact, emin, words, bonds, J, nb = _ladder_run(exchange=False)
    err = means.std(axis=0, ddof=1) / np.sqrt(means.shape[0])
    z = (means.mean(axis=0) - exact) / np.maximum(err, 1e-3)
    assert np.all(np.abs(z) < 5.0), np.round(z, 2)
    assert means.mean(axis=0)[0] < emin + 2.5 and means.mean(axis=0)[-1] > emin + 8
    # the oracle's per-replica energies equal the enumeration's energy function
    E, _ = oracle.ea_observables(DIMS, words, bonds)
    for i in range(words.shape[0]):
        spins = 1 - 2 * ((words[i][:, None] >> np.arange(32, dtype=np.uint32)) & 1).astype(np.int64).T  # [slot][site]
        assert np.array_equal(_energy(spins, J, nb), E[i])


def test_exchange_with_shared_u_stays_within_two_percent():
    means, exact, emin, *_ = _ladder_run(exchange=True)
    rel = np.abs(means.mean(axis=0) - exact) / np.abs(exact)
    assert np.all(rel < 0.02), np.round(100 * rel, 2)
    assert means.mean(axis=0)[0] < emin + 2.5 and means.mean(axis=0)[-1] > emin + 8
