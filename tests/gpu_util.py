"""Helpers for the GPU parity tests: build/load libspn and run both sides."""

from __future__ import annotations

import numpy as np

import oracle
from paper_1006_3865_gb300 import build as spn_build
from paper_1006_3865_gb300 import spn


def lib():
    spn_build.build()
    return spn.load()


def oracle_run(dims, seed, beta_schedule, stream=0, bonds=None, cold=False):
    """Oracle lattice after the (beta, nsweeps) schedule; returns spins, traceE, traceM."""
    N = int(np.prod(dims))
    s = np.ones(N, np.int8) if cold else oracle.init_hot(dims, seed, stream)
    E, M = oracle.observables(dims, s, bonds)
    tE, tM = [], []
    sweep0 = 0
    for beta, n in beta_schedule:
        E, M, e, m = oracle.sweeps(dims, s, beta, n, seed, stream=stream, sweep0=sweep0, bonds=bonds, E=E, M=M)
        tE.append(e)
        tM.append(m)
        sweep0 += n
    return s, np.concatenate(tE) if tE else np.zeros(0, np.int64), np.concatenate(tM) if tM else np.zeros(0, np.int64)


def gpu_run(model, dims, seed, beta_schedule, stream=0, bonds=None, cold=False, path=None, tiling=None):
    lat = spn.Lattice(model, dims, seed, couplings=bonds, stream_id=stream,
                      init=spn.SPN_INIT_COLD if cold else spn.SPN_INIT_HOT)
    if path is not None:
        lat.path = path
    if tiling is not None:
        lat.set_tiling(*tiling)
    for beta, n in beta_schedule:
        lat.sweep(beta, n)
    s = lat.get_spins()
    tE, tM = lat.trace()
    E, M = lat.observables()
    Er, Mr = lat.recompute()
    lat.close()
    assert (E, M) == (Er, Mr), "incremental E/M differ from the full recompute"
    return s, tE, tM
