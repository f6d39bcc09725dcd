"""GPU parity of the Heisenberg (continuous-spin) sweep against the CPU oracle.

Spins are binary32 and every step of the update is a correctly rounded
binary32 operation in a fixed order, so lattices must agree bit for bit: the
device exp on a dense grid, hot starts, and the lattice after sweeps at several
temperatures, 2D and 3D, including shapes whose four-site thread groups cross
rows.  Energies and magnetisations differ only by rounding: the oracle sums
the accepted moves' binary32 dE and dS in binary64 in site order, the GPU adds
them as exact fixed-point integers after rounding each to a multiple of
2^-40.  The bound per sweep is n 2^-53 sum|terms| (n <= N terms of magnitude
at most 4 d for dE, 2 for dS; at most d per bond in a recompute) plus
n 2^-41."""

from __future__ import annotations

import numpy as np
import pytest

import oracle
from gpu_util import lib
from paper_1006_3865_gb300 import inputs, spn

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lib()


def test_device_exp_equals_oracle_bitwise():
    xs = np.concatenate([-np.logspace(-9, np.log10(90.0), 6000), np.linspace(-90.0, 0.0, 6001),
                         np.array([0.0, -0.0, -87.0, -86.99999, -1e-30])]).astype(np.float32)
    got = spn.heis_exp_device(xs)
    ref = np.array([oracle.heis_exp(x) for x in xs], dtype=np.float32)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("dims", [(8, 6), (6, 10), (2, 2), (4, 4, 6), (10, 6, 2)])
def test_hot_start_equals_oracle(dims):
    lat = spn.HeisLattice(dims, 77, stream_id=3)
    S = lat.get_spins()
    So = oracle.heis_init_hot(dims, 77, 3)
    assert np.array_equal(S.view(np.uint32), So.view(np.uint32))
    E, M = lat.observables()
    Eo, Mo = oracle.heis_observables(dims, So)
    nd, N = len(dims), int(np.prod(dims))
    assert abs(E - Eo) <= 2 * nd * N * nd * N * EPS
    assert np.abs(M - Mo).max() <= 2 * N * N * EPS
    lat.close()


def _compare(dims, seed, sched, stream=0):
    nd, N = len(dims), int(np.prod(dims))
    lat = spn.HeisLattice(dims, seed, stream_id=stream)
    So = oracle.heis_init_hot(dims, seed, stream)
    E, M = oracle.heis_observables(dims, So)
    tEo, tMo = [], []
    sweep0 = 0
    for beta, n in sched:
        lat.sweep(beta, n)
        E, M, tE, tM = oracle.heis_sweeps(dims, So, beta, n, seed, stream=stream, sweep0=sweep0, E=E, M=M)
        tEo.append(tE)
        tMo.append(tM)
        sweep0 += n
    S = lat.get_spins()
    assert np.array_equal(S.view(np.uint32), So.view(np.uint32)), \
        f"lattice differs at {np.count_nonzero((S != So).any(axis=1))} sites"
    tE, tM = lat.trace()
    tEo, tMo = np.concatenate(tEo), np.concatenate(tMo)
    s = np.arange(1, len(tE) + 1)
    # per sweep at most N accepted moves with |dE| <= 4 nd and |dS_i| <= 2
    q = s * N * 2.0 ** -41  # the GPU's rounding of each term to the 2^-40 grid
    assert (np.abs(tE - tEo) <= 2 * s * N * (N * 4 * nd) * EPS + q).all()
    assert (np.abs(tM - tMo).max(axis=1) <= 2 * s * N * (N * 2) * EPS + q).all()
    Er, Mr = lat.recompute()
    Eor, Mor = oracle.heis_observables(dims, So)
    assert abs(Er - Eor) <= 2 * nd * N * nd * N * EPS
    lat.close()
    return S


@pytest.mark.parametrize("beta", [0.2, 0.7, 1.5, 6.0])
def test_sweeps_2d(beta):
    _compare((32, 24), inputs.unit_seed(500), [(beta, 6)], stream=2)


@pytest.mark.parametrize("dims", [(6, 10), (10, 6), (2, 8), (14, 2), (66, 4)])
def test_sweeps_2d_row_crossing_groups(dims):
    _compare(dims, inputs.unit_seed(501), [(0.9, 5), (0.3, 2)])


@pytest.mark.parametrize("dims", [(8, 8, 8), (6, 4, 10), (2, 2, 2), (10, 6, 4)])
def test_sweeps_3d(dims):
    _compare(dims, inputs.unit_seed(502), [(0.69, 5), (2.0, 2)], stream=1)


def test_beta_zero_takes_every_proposal_and_large_beta_orders():
    dims = (16, 16)
    _compare(dims, 5, [(0.0, 2)])
    S = _compare(dims, 6, [(50.0, 30)])
    E0, _ = oracle.heis_observables(dims, oracle.heis_init_hot(dims, 6))
    E1, _ = oracle.heis_observables(dims, S)
    assert E1 < E0 - 0.5 * 256  # at low temperature the sweeps lower the energy


def test_reinit_set_spins_and_cold_start():
    dims = (12, 8)
    lat = spn.HeisLattice(dims, 1, init=spn.SPN_INIT_COLD)
    S = lat.get_spins()
    assert (S == np.array([0, 0, 1], np.float32)).all()
    E, M = lat.observables()
    assert E == -2 * 96 and np.array_equal(M, [0.0, 0.0, 96.0])
    lat.sweep(0.5, 3)
    lat.reinit(9, 4)
    assert np.array_equal(lat.get_spins().view(np.uint32), oracle.heis_init_hot(dims, 9, 4).view(np.uint32))
    So = oracle.heis_init_hot(dims, 13, 0)
    lat.set_spins(So)
    lat.sweep(0.8, 2)
    oracle.heis_sweeps(dims, So, 0.8, 2, 9, stream=4)
    assert np.array_equal(lat.get_spins().view(np.uint32), So.view(np.uint32))
    lat.close()


def test_int8_calls_are_refused():
    lat = spn.HeisLattice((8, 8), 1)
    with pytest.raises(spn.SpnError) as e:
        lat._lib.spn_observables  # noqa: B018  (the binding exists)
        spn.Lattice.observables(lat)
    assert e.value.code == spn.SPN_E_STATE
    with pytest.raises(spn.SpnError):
        lat._lib.spn_set_path and spn.Lattice.__dict__["path"].fset(lat, spn.PATH_STREAM)
    lat.close()


def test_larger_3d_lattice():
    _compare((64, 64, 64), inputs.unit_seed(503), [(0.69, 3)])


def test_lattice_where_warps_drain_their_queue_midway():
    """2D 3072 x 3072: 36864 groups of 128 sites per colour for about 6000 warps,
    so a warp collects 32 sites whose first proposal call missed several times
    over a launch and finishes them before its last group."""
    _compare((3072, 3072), inputs.unit_seed(504), [(0.9, 2)])

