"""GPU parity of the shared-memory-resident path of a single lattice (handle
path 2: every sweep of a call in one launch of the persistent kernel) against
the CPU oracle: bit-exact lattices and per-sweep (E, M) traces in 2D and 3D,
on rows that are not a multiple of 64 sites, on lattices that need a cluster of
CTAs, at beta = 0 and infinity, across calls and temperatures, and mixed with
the other paths on one handle."""

from __future__ import annotations

import numpy as np
import pytest

import oracle
from gpu_util import gpu_run, lib, oracle_run
from paper_1006_3865_gb300 import inputs, spn

pytestmark = pytest.mark.gpu

TC = inputs.TC_2D


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lib()


def _compare(model, dims, seed, sched, **kw):
    s_o, e_o, m_o = oracle_run(dims, seed, sched, stream=kw.get("stream", 0), cold=kw.get("cold", False))
    s_g, e_g, m_g = gpu_run(model, dims, seed, sched, path=spn.PATH_RESIDENT, **kw)
    assert np.array_equal(s_g, s_o), f"lattice differs at {np.count_nonzero(s_g != s_o)} sites"
    assert np.array_equal(e_g, e_o) and np.array_equal(m_g, m_o), "E/M trace differs"
    return s_g


@pytest.mark.parametrize("dims", [(128, 96), (64, 64), (66, 40), (2, 2), (6, 10), (130, 2)])
def test_resident_2d(dims):
    _compare(spn.SPN_ISING2D, dims, inputs.unit_seed(21), [(1.0 / TC, 40)], stream=5)


@pytest.mark.parametrize("dims", [(8, 6, 4), (2, 2, 2), (34, 6, 10), (64, 16, 16)])
def test_resident_3d(dims):
    _compare(spn.SPN_ISING3D, dims, inputs.unit_seed(22), [(inputs.BETA_C_3D, 25)])


@pytest.mark.parametrize("model,dims", [(spn.SPN_ISING2D, (1408, 1400)), (spn.SPN_ISING3D, (160, 128, 128))])
def test_resident_cluster(model, dims):
    """Lattices whose bits exceed one CTA's shared memory run on a cluster."""
    _compare(model, dims, inputs.unit_seed(23), [(0.42 if model == spn.SPN_ISING2D else 0.23, 3)])


def test_resident_schedule_across_calls():
    sched = [(0.5, 3), (0.3, 4), (0.44, 1), (1.0, 2)]
    _compare(spn.SPN_ISING2D, (64, 48), 1234, sched, stream=9)


def test_resident_beta_zero_and_infinity():
    dims = (96, 64)
    s = _compare(spn.SPN_ISING2D, dims, 11, [(0.0, 3)])
    assert np.array_equal(s, -oracle.init_hot(dims, 11))
    s = _compare(spn.SPN_ISING2D, dims, 11, [(float("inf"), 4)], cold=True)
    assert (s == 1).all()


def test_paths_mixed_on_one_handle():
    """Sweeps alternate among the resident, streaming, bit-packed and generic
    paths on one handle; the result is the oracle's for the whole schedule."""
    dims, seed = (256, 96), inputs.unit_seed(24)
    plan = [(spn.PATH_RESIDENT, 0.44, 5), (spn.PATH_STREAM, 0.44, 3), (spn.PATH_RESIDENT, 0.3, 4),
            (spn.PATH_PACKED, 0.5, 2), (spn.PATH_RESIDENT, 0.5, 3), (spn.PATH_GENERIC, 0.41, 2),
            (spn.PATH_RESIDENT, 0.41, 1)]
    s_o, e_o, m_o = oracle_run(dims, seed, [(b, n) for _, b, n in plan])
    lat = spn.Lattice(spn.SPN_ISING2D, dims, seed)
    for path, beta, n in plan:
        lat.path = path
        lat.sweep(beta, n)
    s_g = lat.get_spins()
    e_g, m_g = lat.trace()
    assert lat.observables() == lat.recompute()
    lat.close()
    assert np.array_equal(s_g, s_o)
    assert np.array_equal(e_g, e_o) and np.array_equal(m_g, m_o)


def test_resident_rejects_bonds_and_oversize():
    dims = (16, 16, 16)
    bonds = inputs.ea_bonds(dims, 1, inputs.unit_seed(8))[0]
    lat = spn.Lattice(spn.SPN_EA3D_PMJ, dims, 3, couplings=bonds)
    with pytest.raises(spn.SpnError):
        lat.path = spn.PATH_RESIDENT
    lat.close()
    lat = spn.Lattice(spn.SPN_ISING2D, (4096, 4096), 3)  # 2 MB of bits: more than 8 x 200 KB
    with pytest.raises(spn.SpnError):
        lat.path = spn.PATH_RESIDENT
    lat.close()
