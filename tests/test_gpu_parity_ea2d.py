"""GPU parity of the 2D +-J EA multi-spin coded batch and of the replica
overlap measurement against the CPU oracle: replica bits, slot maps, exchange
counts and energies bit for bit; every measured q exactly; the device's exact
sums of q^2 and q^4 against sums of the oracle's q; the Binder cumulant from
them."""

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


def _paired_bonds(dims, pairs, seed):
    """Two replicas of each disorder realisation: samples 2p, 2p+1 share couplings."""
    b = inputs.ea_bonds(dims, pairs, seed)
    return np.repeat(b, 2, axis=0)


class _OracleBatch:
    def __init__(self, dims, bonds, betas, seed, X):
        self.dims, self.bonds, self.betas, self.seed, self.X = dims, bonds, betas, seed, X
        ns = bonds.shape[0]
        self.w = np.concatenate([oracle.ea_init_hot(dims, 1, seed, stream0=i) for i in range(ns)])
        self.pi = np.tile(np.arange(32, dtype=np.uint8), (ns, 1))
        self.tau = self.pi.copy()
        self.acc = np.zeros((ns, 32), np.int64)
        self.sweep = 0

    def run(self, n):
        for i in range(self.w.shape[0]):
            w, pi, tau, acc = self.w[i:i + 1].copy(), self.pi[i:i + 1].copy(), self.tau[i:i + 1].copy(), \
                self.acc[i:i + 1].copy()
            oracle.ea_sweeps(self.dims, w, self.bonds[i:i + 1], self.betas, pi, tau, n, self.seed, stream0=i,
                             sweep0=self.sweep, exchange_every=self.X, acc=acc)
            self.w[i], self.pi[i], self.tau[i], self.acc[i] = w[0], pi[0], tau[0], acc[0]
        self.sweep += n

    def overlap(self):
        return oracle.ea_overlap(self.dims, self.w, self.tau)


@pytest.mark.parametrize("dims,pairs,X,sweeps", [((4, 4), 2, 5, 40), ((16, 8), 2, 10, 60), ((2, 6), 1, 3, 30),
                                                ((64, 64), 2, 10, 40), ((200, 200), 1, 10, 20)])
def test_ea2d_batch_matches_oracle(dims, pairs, X, sweeps):
    seed = inputs.unit_seed(400 + pairs)
    bonds = inputs.ea_bonds(dims, 2 * pairs, inputs.unit_seed(401))
    betas = inputs.geometric_ladder(0.3, 3.0)
    b = spn.EABatch(dims, bonds, betas, seed, exchange_every=X)
    b.sweep(sweeps // 2)
    b.sweep(sweeps - sweeps // 2)
    o = _OracleBatch(dims, bonds, betas, seed, X)
    o.run(sweeps)
    assert np.array_equal(b.words(), o.w)
    assert np.array_equal(b.slots(), o.pi)
    assert np.array_equal(b.exchange_counts(), o.acc)
    E, M = b.energies()
    Eo, Mo = oracle.ea_observables(dims, o.w, bonds)
    assert np.array_equal(E, Eo) and np.array_equal(M, Mo)
    b.close()


@pytest.mark.parametrize("dims,pairs", [((8, 6), 3), ((32, 32), 2), ((12, 10, 6), 2), ((30, 30), 1)])
def test_overlap_series_and_sums_match_oracle(dims, pairs):
    """Measurements every 5 sweeps between exchanges every 10: every q exact, and
    the device's sums of q^2 and q^4 equal the sums of the oracle's q."""
    seed = inputs.unit_seed(410 + pairs)
    bonds = _paired_bonds(dims, pairs, inputs.unit_seed(411))
    betas = inputs.geometric_ladder(0.4, 4.0)
    b = spn.EABatch(dims, bonds, betas, seed, exchange_every=10)
    o = _OracleBatch(dims, bonds, betas, seed, 10)
    qs = []
    for _ in range(8):
        b.sweep(5)
        b.measure_overlap()
        o.run(5)
        q = o.overlap()
        qs.append(q)
        assert np.array_equal(b.overlap()["q_last"], q)
    r = b.overlap()
    qs = [[[int(v) for v in row] for row in q] for q in qs]
    assert r["nmeas"] == 8
    for p in range(pairs):
        for t in range(32):
            assert r["q2_sum"][p][t] == sum(q[p][t] ** 2 for q in qs)
            assert r["q4_sum"][p][t] == sum(q[p][t] ** 4 for q in qs)
    m2 = np.array([[sum(q[p][t] ** 2 for q in qs) / 8 for t in range(32)] for p in range(pairs)])
    m4 = np.array([[sum(q[p][t] ** 4 for q in qs) / 8 for t in range(32)] for p in range(pairs)])
    assert np.allclose(r["binder"], oracle.binder(m2, m4), rtol=1e-12, atol=0, equal_nan=True)
    b.overlap_reset()
    assert b.overlap()["nmeas"] == 0 and all(v == 0 for row in b.overlap()["q2_sum"] for v in row)
    b.close()


def test_overlap_of_identical_replicas_is_n():
    dims = (16, 16)
    bonds = _paired_bonds(dims, 1, 3)
    b = spn.EABatch(dims, bonds, inputs.geometric_ladder(0.5, 5.0), 7, exchange_every=0)
    w = b.words()
    w[1] = w[0]
    b.set_words(w)
    b.measure_overlap()
    assert (b.overlap()["q_last"] == 256).all()
    w[1] = ~w[0]
    b.set_words(w)
    b.measure_overlap()
    assert (b.overlap()["q_last"] == -256).all()
    b.close()


def test_overlap_needs_replica_pairs():
    dims = (8, 8)
    betas = inputs.geometric_ladder(0.5, 5.0)
    for bonds in (inputs.ea_bonds(dims, 2, 1), inputs.ea_bonds(dims, 3, 1)):  # different couplings; odd count
        b = spn.EABatch(dims, bonds, betas, 1)
        with pytest.raises(spn.SpnError) as e:
            b.measure_overlap()
        assert e.value.code == spn.SPN_E_STATE
        b.close()


def test_full_size_overlap_batch_sample_subset():
    """512 replica pairs of the 3D L = 32 workload (the 1024-sample batch as
    pairs), 20 sweeps with exchange every 10, one measurement; q of four pairs
    against the oracle."""
    dims, pairs, seed = (32, 32, 32), 512, inputs.unit_seed(5)
    bonds = _paired_bonds(dims, pairs, inputs.unit_seed(6))
    betas = inputs.geometric_ladder(0.2, 2.0)
    b = spn.EABatch(dims, bonds, betas, seed, exchange_every=10)
    b.sweep(20)
    b.measure_overlap()
    q = b.overlap()["q_last"]
    for p in (0, 255, 511):
        sub = [2 * p, 2 * p + 1]
        # the oracle's streams are the sample indices: run each replica with its own stream
        ws, taus = [], []
        for i in sub:
            w = oracle.ea_init_hot(dims, 1, seed, stream0=i)
            pi = np.arange(32, dtype=np.uint8)[None, :].copy()
            tau = pi.copy()
            oracle.ea_sweeps(dims, w, bonds[i:i + 1], betas, pi, tau, 20, seed, stream0=i, exchange_every=10)
            ws.append(w[0])
            taus.append(tau[0])
        qo = oracle.ea_overlap(dims, np.array(ws), np.array(taus))
        assert np.array_equal(q[p], qo[0])
    b.close()
