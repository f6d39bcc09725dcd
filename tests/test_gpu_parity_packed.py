"""GPU parity of the bit-packed streaming sweep (1 bit per spin in HBM between
sweeps) against the CPU oracle: final lattices and per-sweep integer E/M, bit
for bit, for 2D and 3D lattices, row lengths that fill no whole word, tilings
with ragged segment tails, the special temperatures, runs that move between
the packed and the int8 paths, and the full 2D L = 16384 and 3D L = 512
lattices."""

from __future__ import annotations

import numpy as np
import pytest

import oracle
from gpu_util import gpu_run, lib, oracle_run
from paper_1006_3865_gb300 import inputs, spn

pytestmark = pytest.mark.gpu

TC = inputs.TC_2D
PACKED = spn.PATH_PACKED


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lib()


def _compare(model, dims, seed, sched, **kw):
    cold = kw.get("cold", False)
    s_o, e_o, m_o = oracle_run(dims, seed, sched, stream=kw.get("stream", 0), cold=cold)
    s_g, e_g, m_g = gpu_run(model, dims, seed, sched, path=PACKED, **kw)
    assert np.array_equal(s_g, s_o), f"lattice differs at {np.count_nonzero(s_g != s_o)} sites"
    assert np.array_equal(e_g, e_o) and np.array_equal(m_g, m_o), "E/M trace differs"
    return s_g


@pytest.mark.parametrize("T", [2.0, TC, 3.0])
def test_packed_2d(T):
    _compare(spn.SPN_ISING2D, (128, 96), inputs.unit_seed(40), [(1.0 / T, 25)])


@pytest.mark.parametrize("tiling", [(0, 1, 1), (0, 2, 7), (0, 4, 96), (0, 3, 5), (0, 8, 3), (0, 1, 0)])
def test_packed_2d_tilings(tiling):
    _compare(spn.SPN_ISING2D, (256, 96), inputs.unit_seed(41), [(1.0 / TC, 12)], tiling=tiling, stream=5)


@pytest.mark.parametrize("dims,tiling", [((130, 96), None), ((1000, 70), (0, 2, 5)), ((66, 40), (0, 1, 3)),
                                         ((2, 64), None), ((126, 8), (0, 3, 2)), ((64, 32), (0, 2, 4)),
                                         ((192, 20), None), ((4098, 6), (0, 1, 2))])
def test_packed_2d_ragged_rows(dims, tiling):
    """Rows of 1, 3 or 65 words (padding words in the stored row) and rows whose
    last word is partly empty."""
    _compare(spn.SPN_ISING2D, dims, inputs.unit_seed(42), [(1.0 / TC, 9), (0.3, 2)], tiling=tiling, stream=4)


@pytest.mark.parametrize("dims,tiling", [((2048, 64), None), ((4096, 30), (0, 1, 7)), ((16384, 12), (0, 1, 1)),
                                         ((2048, 2), None), ((2048, 4), (0, 1, 3)), ((8192, 40), (0, 0, 13)),
                                         ((2176, 20), None), ((3072, 8), (0, 1, 3)), ((2048, 2048), (0, 1, 1))])
def test_packed_2d_band_parallel(dims, tiling):
    """Bit-packed rows of at least 2048 sites in an even number of 64-site words
    take the band-parallel kernel, each lane copying its two words of a row:
    bands that wrap around the row end, a last band of one to 29 words, segments
    down to one row, two-row lattices, and 2048-row segments whose warps drain
    their queue of tied colour-1 words many times."""
    _compare(spn.SPN_ISING2D, dims, inputs.unit_seed(45), [(1.0 / TC, 7), (0.3, 2)], tiling=tiling, stream=6)


@pytest.mark.parametrize("dims,tiling", [((64, 32, 8), (32, 1, 0)), ((128, 16, 6), (16, 1, 3)),
                                         ((256, 16, 10), (8, 1, 0)), ((256, 16, 10), (16, 0, 10)),
                                         ((512, 32, 4), (32, 1, 0)), ((512, 32, 6), (4, 1, 5)),
                                         ((512, 24, 6), (12, 1, 2)), ((256, 24, 12), (24, 1, 7)),
                                         ((256, 8, 2), (8, 1, 1)), ((512, 8, 4), (8, 1, 4))])
def test_packed_3d_wavefront(dims, tiling):
    """Bit-packed 3D rows of 64 to 512 sites take the wavefront kernel when one
    plane is streamed per step, each lane copying its two words of a row of
    every plane: one to eight compute warps, rows of one word (padded to four in
    the stored row), a band that is the whole lattice, segments down to one
    plane, two-plane lattices, ragged segment splits."""
    _compare(spn.SPN_ISING3D, dims, inputs.unit_seed(46), [(inputs.BETA_C_3D, 6), (0.35, 2)], tiling=tiling, stream=8)


@pytest.mark.parametrize("tiling", [(2, 1, 1), (4, 2, 5), (8, 1, 12), (16, 3, 2), (16, 1, 0)])
def test_packed_3d_tilings(tiling):
    _compare(spn.SPN_ISING3D, (64, 16, 12), inputs.unit_seed(43), [(inputs.BETA_C_3D, 6)], tiling=tiling)


@pytest.mark.parametrize("dims,tiling", [((70, 16, 12), (4, 1, 3)), ((6, 8, 10), (8, 2, 0)), ((202, 4, 6), None),
                                         ((192, 8, 6), (4, 1, 2)), ((128, 32, 8), (32, 1, 2))])
def test_packed_3d_ragged_rows(dims, tiling):
    _compare(spn.SPN_ISING3D, dims, inputs.unit_seed(44), [(inputs.BETA_C_3D, 6), (0.2, 1)], tiling=tiling)


@pytest.mark.parametrize("model,dims", [(spn.SPN_ISING2D, (64, 32)), (spn.SPN_ISING2D, (130, 6)),
                                        (spn.SPN_ISING3D, (64, 8, 6)), (spn.SPN_ISING2D, (2048, 16)),
                                        (spn.SPN_ISING3D, (256, 16, 8))])
def test_packed_beta_zero_and_infinity(model, dims):
    s = _compare(model, dims, 11, [(0.0, 3)])
    assert np.array_equal(s, -oracle.init_hot(dims, 11))
    s = _compare(model, dims, 11, [(float("inf"), 4)], cold=True)
    assert (s == 1).all()


def test_packed_between_other_paths():
    """Packed sweeps interleaved with int8 sweeps, the double checkerboard and
    reads of the lattice: every step continues from the same spins."""
    dims, seed, stream = (256, 64), inputs.unit_seed(45), 6
    lat = spn.Lattice(spn.SPN_ISING2D, dims, seed, stream_id=stream)
    so = oracle.init_hot(dims, seed, stream)
    E, M = oracle.observables(dims, so)
    sweep0 = 0
    plan = [(PACKED, 0.44, 3), (spn.PATH_STREAM, 0.5, 2), (PACKED, 0.3, 1), ("dc", 0.41, 2), (PACKED, 0.6, 2),
            (spn.PATH_GENERIC, 0.2, 1), (PACKED, 0.44, 2)]
    for step in plan:
        if step[0] == "dc":
            _, beta, n = step
            lat.sweep_dc(beta, n, (64, 8), 2)
            E, M, _, _ = oracle.sweeps_dc(dims, so, (64, 8), 2, beta, n, seed, stream=stream, sweep0=sweep0, E=E, M=M)
        else:
            path, beta, n = step
            lat.path = path
            lat.sweep(beta, n)
            E, M, _, _ = oracle.sweeps(dims, so, beta, n, seed, stream=stream, sweep0=sweep0, E=E, M=M)
        sweep0 += n
        assert np.array_equal(lat.get_spins(), so), f"lattice differs after {step}"
        assert lat.observables() == (E, M) == lat.recompute()
    lat.close()


def test_packed_set_spins_and_reinit():
    dims = (192, 40)
    lat = spn.Lattice(spn.SPN_ISING2D, dims, 3)
    lat.path = PACKED
    lat.sweep(0.4, 2)
    s = np.random.default_rng(inputs.unit_seed(46)).choice(np.array([-1, 1], np.int8), size=int(np.prod(dims)))
    lat.set_spins(s)
    assert np.array_equal(lat.get_spins(), s)
    lat.sweep(0.4, 1)
    so = s.copy()
    oracle.sweeps(dims, so, 0.4, 1, 3, sweep0=2)
    assert np.array_equal(lat.get_spins(), so)
    lat.reinit(8, 1)
    lat.sweep(0.35, 3)
    so = oracle.init_hot(dims, 8, 1)
    oracle.sweeps(dims, so, 0.35, 3, 8, stream=1)
    assert np.array_equal(lat.get_spins(), so)
    lat.close()


def test_packed_rejects_bonds():
    dims = (8, 6, 4)
    bonds = inputs.ea_bonds(dims, 1, 1)[0]
    lat = spn.Lattice(spn.SPN_EA3D_PMJ, dims, 1, couplings=bonds)
    with pytest.raises(spn.SpnError):
        lat.path = PACKED
    lat.close()


def test_packed_full_size_2d_L16384():
    dims, seed = (16384, 16384), inputs.unit_seed(47)
    _compare(spn.SPN_ISING2D, dims, seed, [(1.0 / TC, 2)])


def test_packed_full_size_3d_L512():
    dims, seed = (512, 512, 512), inputs.unit_seed(48)
    _compare(spn.SPN_ISING3D, dims, seed, [(inputs.BETA_C_3D, 2)])
