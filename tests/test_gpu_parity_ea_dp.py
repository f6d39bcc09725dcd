"""GPU parity of the disorder-parallel multi-spin coded EA batch (Sec. 4: the
bits of a word are samples of one group sharing the site's u at one
temperature; replica exchange swaps configurations between the word lattices
of a pair) against the CPU oracle: words, identity slot maps, exchange counts
and per-replica energies bit for bit, 2D and 3D, groups filled partly, with and
without exchange, and sample subsets of the full 1024-sample L = 32 batch."""

from __future__ import annotations

import numpy as np
import pytest

import oracle
from gpu_util import lib
from paper_1006_3865_gb300 import inputs, spn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lib()


def _oracle(dims, bonds, betas, seed, nsweeps, X, sample0=0, count=None, sweep0=0, words=None):
    ns = bonds.shape[0] if count is None else count
    w = oracle.ea_init_hot(dims, ns, seed, stream0=sample0) if words is None else words
    acc = np.zeros((ns, 32), np.int64)
    oracle.ea_dp_sweeps(dims, w, bonds[sample0:sample0 + ns], betas, nsweeps, seed, sweep0=sweep0, exchange_every=X,
                        acc=acc, sample0=sample0)
    return w, acc


@pytest.mark.parametrize("dims,ns,X,sweeps", [((8, 8, 8), 3, 5, 30), ((16, 8), 70, 10, 40), ((24, 8, 6), 2, 10, 25),
                                             ((8, 4, 6), 4, 0, 15), ((32, 16), 65, 3, 21), ((32, 32, 32), 2, 10, 20)])
def test_dp_batch_matches_oracle(dims, ns, X, sweeps):
    seed = inputs.unit_seed(500 + ns)
    bonds = inputs.ea_bonds(dims, ns, inputs.unit_seed(501))
    betas = inputs.geometric_ladder(0.2, 2.0)
    b = spn.EABatch(dims, bonds, betas, seed, exchange_every=X, disorder_parallel=True)
    b.sweep(sweeps // 2)
    b.sweep(sweeps - sweeps // 2)
    w, acc = _oracle(dims, bonds, betas, seed, sweeps, X)
    assert np.array_equal(b.words(), w)
    assert np.array_equal(b.slots(), np.tile(np.arange(32, dtype=np.uint8), (ns, 1)))
    assert np.array_equal(b.exchange_counts(), acc)
    E, M = b.energies()
    Eo, Mo = oracle.ea_observables(dims, w, bonds)
    assert np.array_equal(E, Eo) and np.array_equal(M, Mo)
    b.close()


def test_dp_set_words_and_cold_ladder():
    """Words set from the host (a cold ladder with equal and crowded betas) are
    swept like the oracle's; a non-identity slot map and the per-slot switch are refused."""
    dims, ns, seed = (8, 6, 4), 3, inputs.unit_seed(510)
    bonds = inputs.ea_bonds(dims, ns, inputs.unit_seed(511))
    betas = inputs.geometric_ladder(0.05, 0.5)
    betas[:8] = betas[0]  # eight equal betas at the cold end (exchanges there always accept)
    rng = np.random.default_rng(5)
    words = rng.integers(0, 2 ** 32, size=(ns, int(np.prod(dims))), dtype=np.uint64).astype(np.uint32)
    b = spn.EABatch(dims, bonds, betas, seed, exchange_every=4, disorder_parallel=True)
    b.set_words(words)
    b.sweep(17)
    w, acc = _oracle(dims, bonds, betas, seed, 17, 4, words=words.copy())
    assert np.array_equal(b.words(), w) and np.array_equal(b.exchange_counts(), acc)
    with pytest.raises(spn.SpnError):
        b.set_slots(np.stack([np.random.default_rng(1).permutation(32).astype(np.uint8) for _ in range(ns)]))
    with pytest.raises(spn.SpnError):
        spn._check(b._lib.spn_batch_set_u_per_slot(b._h, 1))
    b.close()
    with pytest.raises(spn.SpnError):
        spn.EABatch((6, 6, 6), inputs.ea_bonds((6, 6, 6), 1, 1), betas, 1, disorder_parallel=True)


def test_dp_overlap_matches_oracle():
    """Replica pairs (samples 2p, 2p + 1 with equal couplings, in different groups)
    give the oracle's overlaps at every temperature."""
    dims, pairs, seed = (16, 8), 40, inputs.unit_seed(520)
    bonds = np.repeat(inputs.ea_bonds(dims, pairs, inputs.unit_seed(521)), 2, axis=0)
    betas = inputs.geometric_ladder(0.3, 3.0)
    b = spn.EABatch(dims, bonds, betas, seed, exchange_every=10, disorder_parallel=True)
    b.sweep(30)
    b.measure_overlap()
    r = b.overlap()
    w, _ = _oracle(dims, bonds, betas, seed, 30, 10)
    q = oracle.ea_overlap(dims, w, np.tile(np.arange(32, dtype=np.uint8), (2 * pairs, 1)))
    assert np.array_equal(r["q_last"], q)
    b.close()


def test_dp_full_batch_sample_subsets():
    """The 1024-sample L = 32 batch, 20 sweeps with exchange every 10; samples
    0-1, 510-513 and 1022-1023 (different groups and blocks) against the oracle."""
    dims, ns, seed = (32, 32, 32), 1024, inputs.unit_seed(3)
    bonds = inputs.ea_bonds(dims, ns, inputs.unit_seed(4))
    betas = inputs.geometric_ladder(0.2, 2.0)
    b = spn.EABatch(dims, bonds, betas, seed, exchange_every=10, disorder_parallel=True)
    b.sweep(20)
    words, acc = b.words(), b.exchange_counts()
    for s0, cnt in ((0, 2), (510, 4), (1022, 2)):
        w, a = _oracle(dims, bonds, betas, seed, 20, 10, sample0=s0, count=cnt)
        assert np.array_equal(words[s0:s0 + cnt], w), s0
        assert np.array_equal(acc[s0:s0 + cnt], a), s0
    b.close()
