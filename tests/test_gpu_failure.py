"""Failure detection without a device fault: a streaming launch (int8, bit-packed,
the 2D and 3D wavefront kernels, or the wavefront double checkerboard) whose first slice is never copied gives up its
bounded wait, records the failure and returns; the host reports SPN_E_TIMEOUT,
and the context keeps working."""

from __future__ import annotations

import numpy as np
import pytest

from gpu_util import gpu_run, lib, oracle_run
from paper_1006_3865_gb300 import inputs, spn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lib()


@pytest.mark.parametrize("path", [spn.PATH_STREAM, spn.PATH_PACKED])
@pytest.mark.parametrize("model,dims", [(spn.SPN_ISING2D, (256, 256)), (spn.SPN_ISING3D, (64, 16, 12)),
                                        (spn.SPN_ISING2D, (4096, 32)), (spn.SPN_ISING3D, (256, 32, 12))])
def test_bounded_wait_runs_out_and_reports_timeout(model, dims, path):
    lat = spn.Lattice(model, dims, 5)
    lat.path = path
    spn.load().spn_test_expire_next_waits(lat._h, 256)
    lat.sweep(0.44, 1)
    with pytest.raises(spn.SpnError) as e:
        lat.observables()
    assert e.value.code == spn.SPN_E_TIMEOUT
    lat.close()
    # the context is still healthy: a fresh lattice matches the oracle bit for bit
    seed = inputs.unit_seed(61)
    s_o, e_o, m_o = oracle_run(dims, seed, [(0.3, 3)])
    s_g, e_g, m_g = gpu_run(model, dims, seed, [(0.3, 3)], path=path)
    assert np.array_equal(s_g, s_o) and np.array_equal(e_g, e_o) and np.array_equal(m_g, m_o)


def test_bounded_wait_runs_out_in_the_double_checkerboard_wavefront():
    dims = (2048, 64)
    lat = spn.Lattice(spn.SPN_ISING2D, dims, 5)
    spn.load().spn_test_expire_next_waits(lat._h, 256)
    lat.sweep_dc(0.44, 1, (64, 8), 1)
    with pytest.raises(spn.SpnError) as e:
        lat.observables()
    assert e.value.code == spn.SPN_E_TIMEOUT
    lat.close()
    seed = inputs.unit_seed(62)
    s_o, e_o, m_o = oracle_run(dims, seed, [(0.3, 2)])
    s_g, e_g, m_g = gpu_run(spn.SPN_ISING2D, dims, seed, [(0.3, 2)])
    assert np.array_equal(s_g, s_o) and np.array_equal(e_g, e_o) and np.array_equal(m_g, m_o)
