"""GPU parity of the int8 checkerboard sweep against the CPU oracle.

Bit-exact comparison of final lattices and per-sweep integer (E, M) traces for
2D and 3D Ising and the int8 +-J EA lattice, on both kernel paths, across tile
shapes with ragged segment tails, at the special temperatures beta = 0 and
beta = infinity, and on the full 2D L = 16384 and 3D L = 512 lattices with the
launch configuration the benchmark uses."""

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
    bonds = kw.pop("bonds", None)
    cold = kw.get("cold", False)
    s_o, e_o, m_o = oracle_run(dims, seed, sched, stream=kw.get("stream", 0), bonds=bonds, cold=cold)
    s_g, e_g, m_g = gpu_run(model, dims, seed, sched, bonds=bonds, **kw)
    assert np.array_equal(s_g, s_o), f"lattice differs at {np.count_nonzero(s_g != s_o)} sites"
    assert np.array_equal(e_g, e_o) and np.array_equal(m_g, m_o), "E/M trace differs"
    return s_g


def test_ising2d_L64_1000_sweeps_at_tc():
    """The 2D L=64 workload: hot start, T = 2.269185, 1000 sweeps."""
    _compare(spn.SPN_ISING2D, (64, 64), inputs.unit_seed(1), [(1.0 / TC, 1000)])


@pytest.mark.parametrize("path", [spn.PATH_GENERIC, spn.PATH_STREAM])
@pytest.mark.parametrize("T", [2.0, TC, 3.0])
def test_ising2d_paths(path, T):
    _compare(spn.SPN_ISING2D, (128, 96), inputs.unit_seed(2), [(1.0 / T, 25)], path=path)


@pytest.mark.parametrize("tiling", [(0, 1, 1), (0, 2, 7), (0, 4, 96), (0, 3, 5), (0, 8, 3), (0, 1, 0)])
def test_ising2d_stream_tilings(tiling):
    """Rows per step and ragged segment splits give identical bytes."""
    _compare(spn.SPN_ISING2D, (256, 96), inputs.unit_seed(3), [(1.0 / TC, 12)], path=spn.PATH_STREAM,
             tiling=tiling, stream=5)


@pytest.mark.parametrize("dims,tiling", [((130, 96), None), ((1000, 70), (0, 2, 5)), ((66, 40), (0, 1, 3)),
                                         ((2, 64), None), ((126, 8), (0, 3, 2))])
def test_ising2d_stream_padded_rows(dims, tiling):
    """Row lengths that are not multiples of 64 stream from rows padded to 64 bytes."""
    _compare(spn.SPN_ISING2D, dims, inputs.unit_seed(13), [(1.0 / TC, 9), (0.3, 2)], path=spn.PATH_STREAM,
             tiling=tiling, stream=4)


@pytest.mark.parametrize("dims,tiling", [((2048, 64), None), ((4096, 30), (0, 1, 7)), ((6144, 10), (0, 1, 10)),
                                         ((16384, 12), (0, 1, 1)), ((2048, 2), None), ((2048, 4), (0, 1, 3)),
                                         ((8192, 40), (0, 0, 13)), ((4096, 6), (0, 1, 6)), ((2112, 20), None),
                                         ((3008, 8), (0, 1, 3)), ((1920 * 4, 10), (0, 1, 2))])
def test_ising2d_band_parallel(dims, tiling):
    """Rows of at least 2048 sites in whole 64-site words take the band-parallel
    kernel (a warp per band of 30 words and segment of rows, with a recomputed
    halo word on each side): bands that wrap around the row end, a last band of
    one to 29 words, segments down to one row, two-row lattices, ragged
    segment splits."""
    _compare(spn.SPN_ISING2D, dims, inputs.unit_seed(17), [(1.0 / TC, 7), (0.3, 2)], path=spn.PATH_STREAM,
             tiling=tiling, stream=6)


@pytest.mark.parametrize("dims,tiling", [((2048, 2048), (0, 1, 1)), ((4096, 1024), (0, 1, 2))])
def test_ising2d_band_parallel_long_segments(dims, tiling):
    """Segments of 512 to 2048 rows: a warp defers a few hundred colour-1 words
    still tied after 12 planes, so its queue is drained many times in the
    middle of the segment (32 words at a time) as well as at the end."""
    _compare(spn.SPN_ISING2D, dims, inputs.unit_seed(19), [(1.0 / TC, 3), (0.3, 1)], path=spn.PATH_STREAM,
             tiling=tiling, stream=7)


@pytest.mark.parametrize("dims,tiling", [((64, 32, 8), (32, 1, 0)), ((128, 16, 6), (16, 1, 3)),
                                         ((256, 16, 10), (8, 1, 0)), ((256, 16, 10), (16, 0, 10)),
                                         ((512, 32, 4), (32, 1, 0)), ((512, 32, 6), (4, 1, 5)),
                                         ((512, 24, 6), (12, 1, 2)), ((256, 24, 12), (24, 1, 7)),
                                         ((256, 8, 2), (8, 1, 1)), ((512, 8, 4), (8, 1, 4))])
def test_ising3d_wavefront(dims, tiling):
    """3D rows of 64 to 512 sites take the wavefront kernel when one plane is
    streamed per step (a warp per group of rows of a band, a halo warp for the
    rows next to it, neighbours at most one step apart): one to eight compute
    warps, a band that is the whole lattice, segments down to one plane, two-plane
    lattices, ragged segment splits."""
    _compare(spn.SPN_ISING3D, dims, inputs.unit_seed(18), [(inputs.BETA_C_3D, 6), (0.35, 2)], path=spn.PATH_STREAM,
             tiling=tiling, stream=8)


@pytest.mark.parametrize("dims,tiling", [((70, 16, 12), (4, 1, 3)), ((6, 8, 10), (8, 2, 0)), ((202, 4, 6), None)])
def test_ising3d_stream_padded_rows(dims, tiling):
    _compare(spn.SPN_ISING3D, dims, inputs.unit_seed(14), [(inputs.BETA_C_3D, 6)], path=spn.PATH_STREAM,
             tiling=tiling)


@pytest.mark.parametrize("dims", [(2, 2), (6, 10), (34, 18), (50, 4), (16, 2)])
def test_ising2d_generic_small_and_ragged(dims):
    _compare(spn.SPN_ISING2D, dims, inputs.unit_seed(4), [(0.41, 30)], path=spn.PATH_GENERIC)


@pytest.mark.parametrize("path", [spn.PATH_GENERIC, spn.PATH_STREAM])
def test_ising3d_paths(path):
    _compare(spn.SPN_ISING3D, (64, 16, 12), inputs.unit_seed(5), [(inputs.BETA_C_3D, 10), (0.3, 5)], path=path)


@pytest.mark.parametrize("tiling", [(2, 1, 1), (4, 2, 5), (8, 1, 12), (16, 3, 2), (16, 1, 0)])
def test_ising3d_stream_tilings(tiling):
    """Band heights, slices per step and segment splits give identical bytes."""
    _compare(spn.SPN_ISING3D, (64, 16, 12), inputs.unit_seed(6), [(inputs.BETA_C_3D, 6)], path=spn.PATH_STREAM,
             tiling=tiling)


@pytest.mark.parametrize("dims", [(1024, 32, 8), (2048, 16, 4)])
def test_ising3d_wide_rows_default_band(dims):
    """Rows of 16 and 32 words: the default band shrinks until the colour-0
    words of a step fit one CTA, and the streaming sweep still runs."""
    lat = spn.Lattice(spn.SPN_ISING3D, dims, 3)
    assert lat.path == spn.PATH_STREAM
    lat.close()
    _compare(spn.SPN_ISING3D, dims, inputs.unit_seed(15), [(inputs.BETA_C_3D, 3)])
    _compare(spn.SPN_ISING3D, dims, inputs.unit_seed(15), [(inputs.BETA_C_3D, 3)], path=spn.PATH_PACKED)


def test_ising3d_stream_wide_rows():
    _compare(spn.SPN_ISING3D, (192, 8, 6), inputs.unit_seed(12), [(0.25, 4)], path=spn.PATH_STREAM,
             tiling=(4, 1, 2))


@pytest.mark.parametrize("dims", [(2, 2, 2), (6, 4, 10), (4, 4, 2), (18, 6, 8)])
def test_ising3d_generic_small(dims):
    _compare(spn.SPN_ISING3D, dims, inputs.unit_seed(7), [(0.25, 15)], path=spn.PATH_GENERIC)


@pytest.mark.parametrize("dims", [(2, 2, 2), (8, 6, 4), (16, 16, 16)])
def test_ea3d_int8(dims):
    bonds = inputs.ea_bonds(dims, 1, inputs.unit_seed(8))[0]
    _compare(spn.SPN_EA3D_PMJ, dims, inputs.unit_seed(9), [(0.9, 20)], bonds=bonds)


@pytest.mark.parametrize("model,dims,path", [(spn.SPN_ISING2D, (64, 32), spn.PATH_STREAM),
                                             (spn.SPN_ISING2D, (2048, 16), spn.PATH_STREAM),
                                             (spn.SPN_ISING3D, (256, 16, 8), spn.PATH_STREAM),
                                             (spn.SPN_ISING2D, (10, 6), spn.PATH_GENERIC),
                                             (spn.SPN_ISING3D, (64, 8, 6), spn.PATH_STREAM)])
def test_beta_zero_and_infinity(model, dims, path):
    s = _compare(model, dims, 11, [(0.0, 3)], path=path)
    s0 = oracle.init_hot(dims, 11)
    assert np.array_equal(s, -s0)
    s = _compare(model, dims, 11, [(float("inf"), 4)], path=path, cold=True)
    assert (s == 1).all()


def test_schedule_across_calls_and_temperatures():
    sched = [(0.5, 3), (0.3, 4), (0.44, 1), (1.0, 2)]
    _compare(spn.SPN_ISING2D, (64, 48), 1234, sched, path=spn.PATH_STREAM, stream=9)


def _sampled_full_size(model, dims, beta, nsweeps):
    seed = inputs.unit_seed(100 + model)
    sched = [(beta, nsweeps)]
    s_o, e_o, m_o = oracle_run(dims, seed, sched)
    s_g, e_g, m_g = gpu_run(model, dims, seed, sched)
    assert np.array_equal(e_g, e_o) and np.array_equal(m_g, m_o)
    assert np.array_equal(s_g, s_o)


def test_full_size_2d_L16384():
    """Full C2 lattice (2^28 sites) with the default (benchmark) launch configuration."""
    _sampled_full_size(spn.SPN_ISING2D, (16384, 16384), 1.0 / TC, 2)


def test_full_size_3d_L512():
    _sampled_full_size(spn.SPN_ISING3D, (512, 512, 512), inputs.BETA_C_3D, 2)


@pytest.mark.parametrize("model,dims,path", [(spn.SPN_ISING2D, (256, 96), spn.PATH_STREAM),
                                             (spn.SPN_ISING2D, (130, 64), spn.PATH_STREAM),
                                             (spn.SPN_ISING3D, (64, 16, 12), spn.PATH_STREAM),
                                             (spn.SPN_ISING3D, (64, 16, 12), spn.PATH_PACKED)])
def test_autotune_keeps_state_and_results(model, dims, path):
    """The streaming autotuner times tilings on a scratch copy: the handle's
    spins and counters are unchanged, and later sweeps still match the oracle."""
    seed, beta = inputs.unit_seed(16), 0.41
    lat = spn.Lattice(model, dims, seed)
    lat.path = path
    lat.sweep(beta, 3)
    before = lat.get_spins()
    tiling = lat.autotune(beta, 2)
    assert len(tiling) == 3
    assert np.array_equal(lat.get_spins(), before) and lat.sweep_count() == 3
    lat.sweep(beta, 4)
    s = oracle.init_hot(dims, seed)
    _, _, tE, tM = oracle.sweeps(dims, s, beta, 7, seed)
    gE, gM = lat.trace()
    assert np.array_equal(lat.get_spins(), s) and np.array_equal(gE, tE) and np.array_equal(gM, tM)
    lat.close()


@pytest.mark.parametrize("model,dims", [(spn.SPN_ISING2D, (64, 32)), (spn.SPN_ISING2D, (66, 40)),
                                        (spn.SPN_ISING2D, (16, 2)), (spn.SPN_ISING3D, (32, 8, 6)),
                                        (spn.SPN_ISING3D, (10, 6, 4)), (spn.SPN_ISING3D, (16, 2, 2))])
def test_set_spins_observables_and_invalid_values(model, dims):
    """E and M of arbitrary states (the full recompute after set_spins, on rows of
    whole 16-byte chunks and on ragged rows) equal the oracle's; a lattice with a
    value other than +-1 anywhere in a chunk is refused."""
    N = int(np.prod(dims))
    rng = np.random.Generator(np.random.PCG64(inputs.unit_seed(70)))
    lat = spn.Lattice(model, dims, 5)
    for frac in (0.5, 0.0, 1.0, 0.1):
        s = np.where(rng.random(N) < frac, -1, 1).astype(np.int8)
        lat.set_spins(s)
        assert lat.observables() == tuple(oracle.observables(dims, s.copy()))
        assert np.array_equal(lat.get_spins(), s)
    for pos in (0, 1, 15, 16, N // 2, N - 1):
        for bad in (0, 2, -3):
            t = s.copy()
            t[pos] = bad
            with pytest.raises(spn.SpnError):
                lat.set_spins(t)
    lat.close()
