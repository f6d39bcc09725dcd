"""GPU parity of the double-checkerboard sweep with generalised multi-hit
(Sec. 3) against the CPU oracle: final lattices and per-sweep integer E/M,
bit for bit, for 2D and 3D tilings, several hit counts, the special
temperatures, sweeps mixed with the canonical order, and the full 2D L = 16384
lattice."""

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


def _model(dims):
    return spn.SPN_ISING2D if len(dims) == 2 else spn.SPN_ISING3D


def _run(dims, seed, plan, stream=0):
    """plan: list of ("dc", beta, nsweeps, tile, hits) or ("sweep", beta, nsweeps)."""
    lat = spn.Lattice(_model(dims), dims, seed, stream_id=stream)
    so = oracle.init_hot(dims, seed, stream)
    E, M = oracle.observables(dims, so)
    tEo, tMo = [], []
    sweep0 = 0
    for step in plan:
        if step[0] == "dc":
            _, beta, n, tile, hits = step
            lat.sweep_dc(beta, n, tile, hits)
            E, M, tE, tM = oracle.sweeps_dc(dims, so, tile, hits, beta, n, seed, stream=stream, sweep0=sweep0, E=E, M=M)
        else:
            _, beta, n = step
            lat.sweep(beta, n)
            E, M, tE, tM = oracle.sweeps(dims, so, beta, n, seed, stream=stream, sweep0=sweep0, E=E, M=M)
        tEo += list(tE)
        tMo += list(tM)
        sweep0 += n
    s = lat.get_spins()
    tEg, tMg = lat.trace()
    Eg, Mg = lat.observables()
    assert (Eg, Mg) == lat.recompute()
    lat.close()
    assert np.array_equal(s, so), f"lattice differs at {np.count_nonzero(s != so)} sites"
    assert np.array_equal(tEg, tEo) and np.array_equal(tMg, tMo), "E/M trace differs"
    return s


@pytest.mark.parametrize("dims,tile,hits", [((128, 64), (64, 8), 1), ((128, 64), (64, 8), 3), ((256, 96), (64, 12), 2),
                                            ((256, 40), (128, 10), 4), ((128, 6), (64, 3), 2),
                                            ((128, 128), (64, 64), 4), ((128, 128), (64, 16), 2),
                                            ((2048, 40), (128, 2), 2), ((3200, 48), (320, 6), 2),
                                            ((3072, 48), (768, 12), 3), ((4096, 32), (256, 4), 4)])
def test_dc_2d(dims, tile, hits):
    _run(dims, inputs.unit_seed(31), [("dc", 1.0 / inputs.TC_2D, 7, tile, hits)], stream=3)


@pytest.mark.parametrize("dims,tile,hits", [((128, 8, 6), (64, 2, 3), 2), ((128, 16, 16), (64, 4, 4), 1),
                                            ((128, 12, 4), (64, 6, 2), 3)])
def test_dc_3d(dims, tile, hits):
    _run(dims, inputs.unit_seed(32), [("dc", inputs.BETA_C_3D, 5, tile, hits)])


def test_dc_special_temperatures():
    dims, tile = (128, 32), (64, 8)
    s0 = oracle.init_hot(dims, 9)
    s = _run(dims, 9, [("dc", 0.0, 1, tile, 3)])
    assert np.array_equal(s, -s0)  # beta = 0: every site flips three times
    _run(dims, 9, [("dc", float("inf"), 2, tile, 2)])


def test_dc_mixed_with_canonical_sweeps():
    plan = [("sweep", 0.44, 3), ("dc", 0.5, 2, (64, 4), 2), ("sweep", 0.3, 1), ("dc", 0.41, 3, (64, 8), 1)]
    _run((128, 32), inputs.unit_seed(33), plan, stream=7)


def test_dc_rejects_bad_tiles():
    lat = spn.Lattice(spn.SPN_ISING2D, (192, 64), 1)
    for tile in ((32, 8), (64, 8), (64, 5)):  # Tx not a multiple of 64; 3 tiles along x; odd tile count in y
        with pytest.raises(spn.SpnError):
            lat.sweep_dc(0.4, 1, tile, 1)
    lat.close()


# one hit on rows of >= 2048 sites in whole words takes the band-parallel
# wavefront form: one-row and 2-row tiles (every other step straddles a tile
# row), bands of 30 words with a ragged last band (50 words), segments of one
# row (the default for 40 rows: more warps than rows) and of many
@pytest.mark.parametrize("dims,tile,hits", [((2048, 64), (64, 8), 1), ((2048, 40), (64, 2), 1), ((2048, 40), (128, 2), 1),
                                            ((2048, 32), (64, 1), 1), ((3200, 40), (64, 4), 1), ((3200, 48), (320, 6), 1),
                                            ((3072, 48), (768, 12), 1), ((4096, 32), (256, 4), 1),
                                            ((2048, 256), (1024, 32), 1), ((4096, 512), (256, 64), 1)])
def test_dc_wavefront_2d(dims, tile, hits):
    _run(dims, inputs.unit_seed(35), [("dc", 1.0 / inputs.TC_2D, 3, tile, hits)], stream=5)


def test_dc_wavefront_special_temperatures_and_mix():
    dims, tile = (2048, 48), (64, 6)
    s0 = oracle.init_hot(dims, 11)
    s = _run(dims, 11, [("dc", 0.0, 1, tile, 1)])
    assert np.array_equal(s, -s0)  # beta = 0: every site flips once
    _run(dims, 11, [("dc", float("inf"), 2, tile, 1)])
    # the two dc kernels (one hit: wavefront; three: tile) and the canonical sweep in one chain
    plan = [("sweep", 0.44, 2), ("dc", 0.5, 2, (128, 8), 1), ("sweep", 0.3, 1), ("dc", 0.41, 2, (64, 4), 3)]
    _run((2048, 64), inputs.unit_seed(36), plan, stream=2)


def test_dc_full_size_2d_L16384():
    """Full 2D L = 16384 lattice with the benchmark's tiling."""
    _run((16384, 16384), inputs.unit_seed(34), [("dc", 1.0 / inputs.TC_2D, 2, (256, 64), 2)])


def test_dc_full_size_2d_L16384_one_hit():
    """The benchmark's k = 1 case on the wavefront form."""
    _run((16384, 16384), inputs.unit_seed(37), [("dc", 1.0 / inputs.TC_2D, 2, (64, 64), 1)])
