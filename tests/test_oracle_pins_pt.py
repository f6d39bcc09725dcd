"""The oracle's multi-spin coded temperature ladder against exact enumeration:
a 4 x 4 +-J lattice (2^16 states), the 32 temperatures of one sample in one
word, 16 independent chains sharing the couplings.  Exact averages come from an
enumeration in numpy over the couplings as the input generator draws them,
independent of the oracle's energy routine, which is checked against the same
enumeration on the final replica states.

* Without exchange every replica is its own Metropolis chain at its
  temperature; by default the 32 slots then share one u per site, which
  correlates them but leaves each one's transition kernel exact, so every
  temperature's mean energy matches the Boltzmann average.
* With exchange the replicas must be independent: replica exchange keeps the
  product of the 32 Boltzmann distributions stationary only when each replica
  moves with its own random numbers (a shared u makes the replicas of a sample
  move together, and the marginals then drift by about 1% of E at the hottest
  temperature).  So a run with exchange draws a u per slot by default, and its
  ladder is exact at every temperature.  The drift of the shared u is shown
  without the oracle by an independent numpy model of the same ladder.
"""

from __future__ import annotations

import numpy as np

import oracle
from exact_lattice import energy, neighbours, reachable
from paper_1006_3865_gb300 import inputs

DIMS = (4, 4)
N = 16


def _couplings(seed, dims=DIMS):
    packed = inputs.ea_bonds(dims, 1, seed)
    return packed, inputs.unpack_bonds(packed, int(np.prod(dims)))[0].astype(np.int64)  # J[d][n], d = x, y (, z)


def _ladder_run(exchange, seed=inputs.unit_seed(0x5A), chains=16, X=10, burn=200, meas=2000, u_per_slot=None,
                dims=DIMS):
    """Per-chain mean energy at each temperature, the exact averages, the final
    words and couplings."""
    packed, J = _couplings(seed, dims)
    nb = neighbours(dims)
    n_sites = int(np.prod(dims))
    states = 1 - 2 * ((np.arange(1 << n_sites)[:, None] >> np.arange(n_sites)) & 1)
    E_all = energy(states, J, nb)
    betas = inputs.geometric_ladder(0.5, 3.0)
    w = np.exp(-np.outer(betas, E_all - E_all.min()))
    exact = (w * E_all).sum(axis=1) / w.sum(axis=1)
    bonds = np.repeat(packed, chains, axis=0)  # every chain samples the same couplings
    words = oracle.ea_init_hot(dims, chains, seed)
    pi = np.tile(np.arange(32, dtype=np.uint8), (chains, 1))
    tau = pi.copy()
    sums = np.zeros((chains, 32))
    for it in range(burn + meas):
        oracle.ea_sweeps(dims, words, bonds, betas, pi, tau, X, seed, sweep0=X * it,
                         exchange_every=X if exchange else 0, u_per_slot=u_per_slot)
        if it >= burn:
            E, _ = oracle.ea_observables(dims, words, bonds)
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
        assert np.array_equal(energy(spins, J, nb), E[i])


def test_default_ladder_with_exchange_is_boltzmann_at_every_temperature():
    """Replica exchange every 10 sweeps with the default random numbers of a run
    with exchange (a u per slot): every temperature's mean energy matches the
    exact Boltzmann average within five standard errors."""
    means, exact, emin, *_ = _ladder_run(exchange=True)
    err = means.std(axis=0, ddof=1) / np.sqrt(means.shape[0])
    z = (means.mean(axis=0) - exact) / np.maximum(err, 1e-3)
    assert np.all(np.abs(z) < 5.0), np.round(z, 2)
    assert means.mean(axis=0)[0] < emin + 2.5 and means.mean(axis=0)[-1] > emin + 8


def numpy_ladder(shared_u, seed=inputs.unit_seed(0x5A), chains=16, X=10, burn=100, meas=1000, rng_seed=12345):
    """Plain numpy parallel tempering of the same lattice, ladder and exchange
    schedule as the oracle run above, independent of the oracle.  Replicas keep
    their slots and the exchange swaps the slots' temperatures, as in the oracle;
    shared_u draws one uniform per site for all 32 slots (the oracle's reading),
    otherwise one per slot and site.  Returns the z-scores of each temperature's
    mean energy against the exact average."""
    packed, J = _couplings(seed)
    nb = neighbours(DIMS)
    states = 1 - 2 * ((np.arange(1 << N)[:, None] >> np.arange(N)) & 1)
    E_all = energy(states, J, nb)
    betas = inputs.geometric_ladder(0.5, 3.0)
    w = np.exp(-np.outer(betas, E_all - E_all.min()))
    exact = (w * E_all).sum(axis=1) / w.sum(axis=1)
    n = np.arange(N)
    x, y = n % 4, n // 4
    back = np.stack([(x - 1) % 4 + 4 * y, x + 4 * ((y - 1) % 4)])  # backward neighbour along x, y
    colour = (x + y) & 1
    rng = np.random.Generator(np.random.PCG64(rng_seed))
    S = np.where(rng.random((chains, 32, N)) < 0.5, -1, 1).astype(np.int64)  # S[c, slot]
    temp_of_slot = np.tile(np.arange(32), (chains, 1))
    sums = np.zeros((chains, 32))
    for blk in range(burn + meas):
        for _ in range(X):
            for c in (0, 1):
                h = sum(J[d] * S[..., nb[d]] + J[d][back[d]] * S[..., back[d]] for d in range(2))
                dE = 2 * S * h
                u = rng.random((chains, 1, N)) if shared_u else rng.random(S.shape)
                b = betas[temp_of_slot][:, :, None]
                flip = ((dE <= 0) | (u < np.exp(-b * np.maximum(dE, 0)))) & (colour == c)
                S = np.where(flip, -S, S)
        E = energy(S, J, nb)  # by slot
        slot_of_temp = np.argsort(temp_of_slot, axis=1)
        Et = np.take_along_axis(E, slot_of_temp, axis=1)
        for k in range(blk & 1, 31, 2):  # the pairs of this exchange step
            D = (betas[k] - betas[k + 1]) * (Et[:, k] - Et[:, k + 1])
            rows = np.nonzero((D >= 0) | (rng.random(chains) < np.exp(np.minimum(D, 0))))[0]
            a, b2 = slot_of_temp[rows, k], slot_of_temp[rows, k + 1]
            temp_of_slot[rows, a], temp_of_slot[rows, b2] = k + 1, k
        if blk >= burn:
            sums += np.take_along_axis(E, np.argsort(temp_of_slot, axis=1), axis=1)
    means = sums / meas
    err = means.std(axis=0, ddof=1) / np.sqrt(chains)
    return (means.mean(axis=0) - exact) / np.maximum(err, 1e-3)


def test_independent_u_per_replica_makes_exchange_exact():
    """The diagnosis above, checked without the oracle: with an independent
    uniform for every slot and site the same exchange schedule keeps every
    temperature Boltzmann-distributed.  (With meas=4000 and rng_seed 1..4 the
    hottest temperature's z is -6.3, -4.4, -3.3, -4.7 for shared_u=True and
    +0.9, +1.9, -0.3, +1.2 for independent u.)"""
    z = numpy_ladder(shared_u=False)
    assert np.all(np.abs(z) < 5.0), np.round(z, 2)


def test_oracle_ladder_with_a_u_per_slot_and_no_exchange_is_boltzmann():
    """The per-slot random numbers chosen for a run without exchange: each
    replica is again its own exact Metropolis chain."""
    means, exact, emin, *_ = _ladder_run(exchange=False, u_per_slot=True, meas=1000)
    err = means.std(axis=0, ddof=1) / np.sqrt(means.shape[0])
    z = (means.mean(axis=0) - exact) / np.maximum(err, 1e-3)
    assert np.all(np.abs(z) < 5.0), np.round(z, 2)


# ---------------------------------------------------------------- 3D ladder

DIMS3 = (4, 2, 2)  # 16 sites of the simple cubic lattice (the EA batches' model), small enough to enumerate
SEED3 = inputs.unit_seed(0x5B)  # couplings on which the checkerboard chain is irreducible (checked below)


def _z(means, exact):
    err = means.std(axis=0, ddof=1) / np.sqrt(means.shape[0])
    return (means.mean(axis=0) - exact) / np.maximum(err, 1e-3)


def test_3d_ladder_energies_match_enumeration():
    """The 3D +-J ladder: the oracle's per-replica energies equal the numpy
    energy of Eq. 1 over the three bond directions, and without exchange every
    temperature's mean energy matches the exact Boltzmann average."""
    _, J = _couplings(SEED3, DIMS3)
    for s0 in (0, 12345):
        assert reachable(DIMS3, J, s0).all()
    means, exact, emin, words, bonds, J, nb = _ladder_run(exchange=False, seed=SEED3, meas=1000, dims=DIMS3)
    E, _ = oracle.ea_observables(DIMS3, words, bonds)
    for i in range(words.shape[0]):
        spins = 1 - 2 * ((words[i][:, None] >> np.arange(32, dtype=np.uint32)) & 1).astype(np.int64).T
        assert np.array_equal(energy(spins, J, nb), E[i])
    z = _z(means, exact)
    assert np.all(np.abs(z) < 5.0), np.round(z, 2)


def test_3d_default_ladder_with_exchange_is_boltzmann_at_every_temperature():
    means, exact, *_ = _ladder_run(exchange=True, seed=SEED3, meas=1000, dims=DIMS3)
    z = _z(means, exact)
    assert np.all(np.abs(z) < 5.0), np.round(z, 2)


def test_checkerboard_chain_can_be_reducible_with_two_site_axes():
    """Why the 3D pins check irreducibility first: with an extent of 2 along y
    and z, each neighbour pair there is joined by two bonds, and on the 0x5A
    couplings the checkerboard sweep (fixed colour order, dE <= 0 always taken)
    splits the 2^16 states into closed classes, so a run's averages depend on its
    start.  Random-site order, or any of twelve other coupling draws, has one
    class; the 2D 4 x 4 lattice of the pins above has one class too."""
    _, J3 = _couplings(inputs.unit_seed(0x5A), DIMS3)
    sizes = {int(reachable(DIMS3, J3, s0).sum()) for s0 in (0, 1, 2, 3, 40000, 65535)}
    assert len(sizes) > 1 and max(sizes) < 1 << 16, sizes
    _, J2 = _couplings(inputs.unit_seed(0x5A))
    assert reachable(DIMS, J2, 0).all()
