"""The seeded input generators follow the stated recipe: bond packing round-trips
in the library's bit layout, +-J bonds are iid with the requested balance and
reproducible from their seed, ladders are geometric in T with the stated ends,
and the uneven batch and the served stream draw from the stated ranges."""

from __future__ import annotations

import math

import numpy as np
import pytest

from paper_1006_3865_gb300 import inputs


@pytest.mark.parametrize("dims", [(4, 4), (6, 10), (66, 2), (8, 4, 2), (3 * 64 + 2, 2, 2)])
def test_pack_and_unpack_round_trip(dims):
    rng = np.random.default_rng(5)
    N = inputs.lattice_sites(dims)
    J = np.where(rng.random((3, len(dims), N)) < 0.5, -1, 1).astype(np.int8)
    words = inputs.pack_bonds(J)
    assert words.shape == (3, len(dims), inputs.bond_words(dims)) and words.dtype == np.uint64
    assert np.array_equal(inputs.unpack_bonds(words, N), J)
    n = N - 1  # bit (n % 64) of word n // 64 is set iff J = -1
    assert bool((int(words[0, 0, n // 64]) >> (n % 64)) & 1) == (J[0, 0, n] < 0)
    if N % 64:  # padding bits past the last site stay clear
        assert int(words[0, 0, -1]) >> (N % 64) == 0


def test_uniform_bonds():
    dims = (6, 4, 2)
    N = inputs.lattice_sites(dims)
    assert not inputs.uniform_bonds(dims, 2, +1).any()
    assert np.all(inputs.unpack_bonds(inputs.uniform_bonds(dims, 2, -1), N) == -1)


def test_ea_bonds_are_balanced_and_reproducible():
    dims, ns = (16, 16, 16), 8
    N = inputs.lattice_sites(dims)
    a = inputs.ea_bonds(dims, ns, inputs.unit_seed(1))
    J = inputs.unpack_bonds(a, N)
    n = J.size
    neg = int((J < 0).sum())
    assert abs(neg - n / 2) < 5 * math.sqrt(n / 4)
    assert np.array_equal(a, inputs.ea_bonds(dims, ns, inputs.unit_seed(1)))
    assert not np.array_equal(a, inputs.ea_bonds(dims, ns, inputs.unit_seed(2)))
    assert not np.array_equal(J[0], J[1])  # samples are different realisations
    q = inputs.unpack_bonds(inputs.ea_bonds(dims, ns, inputs.unit_seed(1), p_negative=0.2), N)
    assert abs(int((q < 0).sum()) - 0.2 * n) < 5 * math.sqrt(n * 0.2 * 0.8)


def test_unit_seeds_are_distinct():
    seeds = {inputs.unit_seed(u) for u in range(100000)}
    assert len(seeds) == 100000
    assert inputs.unit_seed(7) != inputs.unit_seed(7, master=inputs.MASTER_SEED + 1)


def test_geometric_ladder():
    betas = inputs.geometric_ladder(0.2, 2.0)
    T = 1.0 / betas
    assert betas.shape == (32,) and np.all(np.diff(betas) < 0)  # ascending temperature
    assert T[0] == pytest.approx(0.2) and T[-1] == pytest.approx(2.0)
    ratio = T[1:] / T[:-1]
    assert np.allclose(ratio, 10.0 ** (1.0 / 31.0))


def test_uneven_batch_ranges():
    batch = inputs.uneven_batch()
    assert len(batch) == 4096
    Ls = np.array([b.dims[0] for b in batch])
    assert all(b.dims[0] == b.dims[1] for b in batch)
    assert set(np.log2(Ls).astype(int)) == set(range(5, 12))
    T = np.array([1.0 / b.beta for b in batch])
    assert T.min() >= 1.5 and T.max() <= 3.5
    s = np.array([b.nsweeps for b in batch])
    assert s.min() >= 100 and s.max() <= 2000
    assert len({b.seed for b in batch}) == 4096


def test_served_stream_ranges():
    reqs = inputs.served_stream()
    assert len(reqs) == 2000
    gaps = np.diff([0.0] + [r.arrival_s for r in reqs])
    assert np.all(gaps > 0) and abs(gaps.mean() - 0.5e-3) < 5 * 0.5e-3 / math.sqrt(2000)
    models = np.array([r.model for r in reqs])
    assert set(models) == {1, 2, 3} and all(abs((models == m).mean() - 1 / 3) < 0.05 for m in (1, 2, 3))
    for r in reqs:
        assert all(e >= 2 and e % 2 == 0 for e in r.dims)
        assert 100 <= r.nsweeps <= 10000
        if r.model == 1:
            assert len(r.dims) == 2 and 64 <= r.dims[0] <= 4096
        elif r.model == 2:
            assert len(r.dims) == 3 and 16 <= r.dims[0] <= 256
        else:
            assert r.dims[0] in (8, 16, 24, 32) and r.betas.shape == (32,)
            assert (1.0 / r.betas[-1]) / (1.0 / r.betas[0]) == pytest.approx(10.0)
            assert 0.5 <= 1.0 / r.betas[0] <= 4.0
            assert r.bonds.shape == (1, 3, inputs.bond_words(r.dims))
