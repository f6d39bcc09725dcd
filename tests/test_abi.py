"""The C-ABI library builds, loads and exports every function of include/spn.h;
host-side argument checks reject bad input before any device work (no GPU
needed)."""

from __future__ import annotations

import ctypes
import subprocess

import numpy as np
import pytest

from paper_1006_3865_gb300 import build as spn_build
from paper_1006_3865_gb300 import spn


@pytest.fixture(scope="module")
def lib():
    spn_build.build()
    return spn.load()


def test_every_header_function_is_exported_and_bound(lib):
    declared = spn.header_functions()
    assert len(declared) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", spn.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    for name in declared:
        assert name in exported, f"{name} declared in spn.h but not exported"
        assert name in spn._SIGNATURES, f"{name} has no binding"
        getattr(lib, name)
    assert set(spn._SIGNATURES) <= set(declared)


def _create(lib, model, dims, couplings=None, init=0):
    h = ctypes.c_void_p()
    d = np.asarray(dims, dtype=np.int32)
    c = None if couplings is None else couplings.ctypes.data_as(ctypes.c_void_p)
    rc = lib.spn_create_ex(ctypes.byref(h), model, d.ctypes.data_as(ctypes.c_void_p), c, 1, 0, init)
    return rc, lib.spn_last_error().decode()


@pytest.mark.parametrize("model,dims", [(1, (3, 4)), (1, (4, 0)), (2, (4, 4, 5)), (2, (4, 2, -2)), (1, (1, 2))])
def test_odd_or_empty_extents_are_rejected(lib, model, dims):
    rc, msg = _create(lib, model, dims)
    assert rc == spn.SPN_E_ARG and "even" in msg


def test_bad_model_and_couplings_are_rejected(lib):
    assert _create(lib, 7, (4, 4))[0] == spn.SPN_E_ARG
    assert _create(lib, spn.SPN_EA3D_PMJ, (4, 4, 4))[0] == spn.SPN_E_ARG
    w = np.zeros(3, np.uint64)
    assert _create(lib, spn.SPN_ISING2D, (8, 8), couplings=w)[0] == spn.SPN_E_ARG
    assert _create(lib, spn.SPN_ISING2D, (8, 8), init=9)[0] == spn.SPN_E_ARG
    assert lib.spn_create_ex(None, 1, None, None, 0, 0, 0) == spn.SPN_E_ARG
    assert lib.spn_sweep(None, 0.3, 1) == spn.SPN_E_ARG
    assert lib.spn_destroy(None) == spn.SPN_E_ARG


def test_version_string(lib):
    assert b"sm_103a" in lib.spn_version()


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without libspn.so the binding raises; nothing falls back to a CPU path."""
    monkeypatch.setattr(spn, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        spn.load(str(tmp_path / "libspn.so"))
    monkeypatch.setattr(spn, "LIB_PATH", str(tmp_path / "libspn.so"))
    with pytest.raises(RuntimeError, match="not found"):
        spn.load()


@pytest.mark.parametrize("model,dims", [(spn.SPN_ISING3D, (2, 32768, 16386)), (spn.SPN_ISING2D, (66, (1 << 28) + 2))])
def test_lattices_beyond_the_counter_range_are_rejected(lib, model, dims):
    """A site's Philox counter word is 8 g + call with g its 64-site row word;
    past 2^29 row words it would wrap, so such lattices are refused (here with
    fewer than 2^35 sites) by every entry point that takes a lattice, before any
    device work."""
    rc, msg = _create(lib, model, dims)
    assert rc == spn.SPN_E_ARG and "counter" in msg
    job = spn.Job(model=model, beta=0.4, nsweeps=1, seed=1)
    for i, e in enumerate(dims):
        job.dims[i] = e
    arr = (spn.Job * 1)(job)
    m = ctypes.c_void_p()
    assert lib.spn_multi_create(ctypes.byref(m), ctypes.cast(arr, ctypes.c_void_p), 1) == spn.SPN_E_ARG
    assert "counter" in lib.spn_last_error().decode()
