"""GPU parity of the multi-spin coded +-J EA batch (replica bits, slot maps,
exchange counts, per-replica energies) against the CPU oracle, including a
sample subset of the full 1024-sample L = 32 batch."""

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


def _oracle_batch(dims, bonds, betas, seed, nsweeps, X, samples, words0=None, slots0=None, u_per_slot=None):
    out_w, out_pi, out_acc = [], [], []
    for i in samples:
        w = (oracle.ea_init_hot(dims, 1, seed, stream0=i) if words0 is None else words0[i:i + 1].copy())
        pi = (np.arange(32, dtype=np.uint8)[None, :].copy() if slots0 is None else slots0[i:i + 1].copy())
        tau = np.zeros_like(pi)
        tau[0][pi[0]] = np.arange(32, dtype=np.uint8)
        acc = np.zeros((1, 32), np.int64)
        oracle.ea_sweeps(dims, w, bonds[i:i + 1], betas, pi, tau, nsweeps, seed, stream0=i, exchange_every=X, acc=acc,
                         u_per_slot=u_per_slot)
        out_w.append(w[0])
        out_pi.append(pi[0])
        out_acc.append(acc[0])
    return np.array(out_w), np.array(out_pi), np.array(out_acc)


@pytest.mark.parametrize("dims,ns,X,sweeps", [((4, 4, 6), 3, 5, 40), ((8, 8, 8), 4, 10, 60), ((6, 4, 2), 1, 3, 30),
                                             ((16, 16, 16), 2, 10, 40), ((24, 24, 24), 1, 10, 20)])
def test_batch_matches_oracle(dims, ns, X, sweeps):
    seed = inputs.unit_seed(300 + ns)
    bonds = inputs.ea_bonds(dims, ns, inputs.unit_seed(301))
    betas = inputs.geometric_ladder(0.2, 2.0)
    b = spn.EABatch(dims, bonds, betas, seed, exchange_every=X)
    b.sweep(sweeps // 2)
    b.sweep(sweeps - sweeps // 2)
    w, pi, acc = _oracle_batch(dims, bonds, betas, seed, sweeps, X, range(ns))
    assert np.array_equal(b.words(), w)
    assert np.array_equal(b.slots(), pi)
    assert np.array_equal(b.exchange_counts(), acc)
    E, M = b.energies()
    Eo, Mo = oracle.ea_observables(dims, w, bonds)
    assert np.array_equal(E, Eo) and np.array_equal(M, Mo)
    b.close()


@pytest.mark.parametrize("u_per_slot", [False, None])
@pytest.mark.parametrize("dims,ladder", [((8, 8, 8), "equal"), ((16, 8, 4), "pairs"), ((8, 6, 4), "cold")])
def test_tied_and_crowded_thresholds(dims, ladder, u_per_slot):
    """Ladders whose thresholds share buckets of u (equal betas, pairs of equal
    betas, very low temperatures where many thresholds are near 0): with a shared
    u the exact count of thresholds below u then comes from the binary search,
    on both the four-word groups (Lx a multiple of 8) and the per-site loop;
    with the default u per slot, equal thresholds give equal threshold planes."""
    if ladder == "equal":
        betas = np.full(32, 0.35)
    elif ladder == "pairs":
        betas = np.repeat(inputs.geometric_ladder(0.3, 3.0)[::2], 2)
    else:
        betas = inputs.geometric_ladder(0.05, 0.5)
    ns, X, sweeps, seed = 2, 5, 30, inputs.unit_seed(310)
    bonds = inputs.ea_bonds(dims, ns, inputs.unit_seed(311))
    b = spn.EABatch(dims, bonds, betas, seed, exchange_every=X, u_per_slot=u_per_slot)
    b.sweep(sweeps)
    w, pi, acc = _oracle_batch(dims, bonds, betas, seed, sweeps, X, range(ns), u_per_slot=u_per_slot)
    assert np.array_equal(b.words(), w)
    assert np.array_equal(b.slots(), pi)
    assert np.array_equal(b.exchange_counts(), acc)
    b.close()


@pytest.mark.parametrize("dims,ns,X,sweeps,ps", [((8, 8, 8), 3, 5, 30, True), ((6, 4, 2), 2, 3, 20, True),
                                                ((16, 8), 2, 10, 40, True), ((4, 4), 2, 5, 30, True),
                                                ((24, 24, 24), 1, 10, 10, True), ((32, 32, 32), 1, 10, 20, True),
                                                ((40, 32, 34), 1, 5, 10, True), ((8, 8, 8), 2, 0, 20, True),
                                                ((16, 8, 8), 2, 5, 20, False),
                                                ((16, 8), 2, 5, 20, False)])
def test_u_per_slot_matches_oracle(dims, ns, X, sweeps, ps):
    """Every temperature slot with its own u (32 bit planes per site), on the
    four-word groups (Lx a multiple of 8) and the per-site loop, 2D and 3D, with
    and without exchange; and the shared u chosen explicitly for a run with
    exchange: words, slot maps and exchange counts equal the oracle's."""
    seed = inputs.unit_seed(320 + ns)
    bonds = inputs.ea_bonds(dims, ns, inputs.unit_seed(321))
    betas = inputs.geometric_ladder(0.2, 2.0)
    b = spn.EABatch(dims, bonds, betas, seed, exchange_every=X, u_per_slot=ps)
    b.sweep(sweeps // 2)
    b.sweep(sweeps - sweeps // 2)
    w, pi, acc = _oracle_batch(dims, bonds, betas, seed, sweeps, X, range(ns), u_per_slot=ps)
    assert np.array_equal(b.words(), w)
    assert np.array_equal(b.slots(), pi)
    assert np.array_equal(b.exchange_counts(), acc)
    E, M = b.energies()
    Eo, Mo = oracle.ea_observables(dims, w, bonds)
    assert np.array_equal(E, Eo) and np.array_equal(M, Mo)
    b.close()


def test_explicit_state_and_permutation():
    dims, ns, seed = (8, 4, 6), 2, 99
    bonds = inputs.ea_bonds(dims, ns, 5)
    betas = inputs.geometric_ladder(0.5, 5.0)
    rng = np.random.default_rng(3)
    words = rng.integers(0, 2**32, size=(ns, int(np.prod(dims))), dtype=np.uint64).astype(np.uint32)
    slots = np.stack([rng.permutation(32).astype(np.uint8) for _ in range(ns)])
    b = spn.EABatch(dims, bonds, betas, seed, exchange_every=0)
    b.set_words(words)
    b.set_slots(slots)
    b.sweep(15)
    w, pi, acc = _oracle_batch(dims, bonds, betas, seed, 15, 0, range(ns), words0=words, slots0=slots)
    assert np.array_equal(b.words(), w) and np.array_equal(b.slots(), pi)


def test_equal_betas_always_exchange():
    dims, ns = (4, 4, 4), 2
    bonds = inputs.ea_bonds(dims, ns, 6)
    b = spn.EABatch(dims, bonds, np.full(32, 0.8), 12, exchange_every=10)
    b.sweep(40)
    acc = b.exchange_counts()
    assert acc[:, 0::2].sum(axis=1).tolist() == [32, 32] and acc[:, 1::2].sum(axis=1).tolist() == [30, 30]


def test_full_batch_sample_subset():
    """The 1024-sample L = 32 batch (64 replicas per uint64 word), 20 sweeps with
    exchange every 10 on the default chain (a u per slot); four samples compared
    with the oracle."""
    dims, ns, seed = (32, 32, 32), 1024, inputs.unit_seed(3)
    bonds = inputs.ea_bonds(dims, ns, inputs.unit_seed(4))
    betas = inputs.geometric_ladder(0.2, 2.0)
    b = spn.EABatch(dims, bonds, betas, seed, exchange_every=10)
    b.sweep(20)
    words, slots, acc = b.words(), b.slots(), b.exchange_counts()
    subset = [0, 1, 511, 1023]
    w, pi, ac = _oracle_batch(dims, bonds, betas, seed, 20, 10, subset)
    assert np.array_equal(words[subset], w)
    assert np.array_equal(slots[subset], pi)
    assert np.array_equal(acc[subset], ac)
    b.close()


def test_rejections():
    with pytest.raises(spn.SpnError):
        spn.EABatch((36, 36, 36), inputs.ea_bonds((36, 36, 36), 1, 1), inputs.geometric_ladder(0.2, 2.0), 1)
    with pytest.raises(spn.SpnError):
        spn.EABatch((4, 4, 4), inputs.ea_bonds((4, 4, 4), 1, 1), inputs.geometric_ladder(0.2, 2.0)[::-1], 1)
