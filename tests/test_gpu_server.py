"""The request server with continuous batching: a job's result does not depend
on what runs beside it or when it arrives (bit for bit against the CPU oracle
and against the job run alone), EA jobs match the EA batch entry points,
admission respects the HBM budget, and polling never blocks."""

from __future__ import annotations

import time

import numpy as np
import pytest

import oracle
from gpu_util import lib
from paper_1006_3865_gb300 import inputs, spn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lib()


def _wait(srv, tickets, limit_s=120.0):
    t0 = time.monotonic()
    pending = set(tickets)
    while pending:
        for t in list(pending):
            done, res = srv.poll(t)
            if done:
                pending.discard(t)
        assert time.monotonic() - t0 < limit_s, "server did not finish in time"
        time.sleep(0.002)


_MIX = [((32, 32), 2.2, 37), ((64, 64), 2.4, 50), ((128, 64), 1.9, 20), ((16, 8), 3.0, 90),
        ((1024, 256), 2.27, 12), ((16, 16, 16), 1 / 4.5, 25), ((64, 16, 8), 1 / 4.4, 9), ((256, 64), 2.1, 700),
        ((8192, 64), 2.3, 3), ((192, 128), 2.0, 6), ((6, 4), 2.5, 41), ((6, 4, 2), 1 / 4.0, 33),
        ((4096, 4096), 2.27, 3), ((256, 256, 256), 1 / 4.51, 2), ((1030, 1026), 2.27, 4),
        ((102, 104, 100), 1 / 4.51, 3), ((1998, 3000), 3.0, 2), ((3650, 3650), 2.27, 2),
        ((6002, 5000), 2.27, 2)]  # 3.8 MB of bits: more than 16 CTAs hold, so it streams


def _submit_ising(srv, k, dims, T, ns):
    model = spn.SPN_ISING2D if len(dims) == 2 else spn.SPN_ISING3D
    return srv.submit(model, dims, ns, inputs.unit_seed(700 + k), beta=1.0 / T if T > 1 else T, stream=k)


def _beta(T):
    return 1.0 / T if T > 1 else T


def test_mix_matches_oracle_and_alone():
    srv = spn.Server(1 << 30)
    tickets = [_submit_ising(srv, k, d, T, ns) for k, (d, T, ns) in enumerate(_MIX)]
    _wait(srv, tickets)
    for k, (d, T, ns) in enumerate(_MIX):
        done, res = srv.poll(tickets[k])
        assert done and res.state == 2 and res.status == 0 and res.sweeps == ns
        s = srv.fetch(tickets[k])
        seed = inputs.unit_seed(700 + k)
        so = oracle.init_hot(d, seed, k)
        oracle.sweeps(d, so, _beta(T), ns, seed, stream=k)
        assert np.array_equal(s, so), (k, d)
        E, M = oracle.observables(d, so)
        assert (res.E, res.M) == (E, M)
    # the same jobs alone, one at a time
    for k in (0, 4, 7, 10, 12, 13, 14, 15, 17, 18):
        d, T, ns = _MIX[k]
        alone = spn.Server(1 << 30)
        t = _submit_ising(alone, k, d, T, ns)
        _wait(alone, [t])
        assert np.array_equal(alone.fetch(t), srv.fetch(tickets[k])), k
        alone.close()
    st = srv.stats()
    expect = sum(int(np.prod(d)) * ns for d, T, ns in _MIX)
    assert st["attempts"] == expect and st["used_bytes"] == 0 and st["rounds"] >= 1
    srv.close()


def test_late_arrivals_join_running_batch():
    srv = spn.Server(1 << 30)
    first = [_submit_ising(srv, 7, *_MIX[7])]
    time.sleep(0.01)
    late = [_submit_ising(srv, k, *_MIX[k]) for k in (0, 1, 5)]
    _wait(srv, first + late)
    for t, k in zip(first + late, (7, 0, 1, 5)):
        d, T, ns = _MIX[k]
        seed = inputs.unit_seed(700 + k)
        so = oracle.init_hot(d, seed, k)
        oracle.sweeps(d, so, _beta(T), ns, seed, stream=k)
        assert np.array_equal(srv.fetch(t), so), k
        done, res = srv.poll(t)
        assert res.t_submit <= res.t_admit <= res.t_done
    srv.close()


@pytest.mark.parametrize("X", [10, 0])
def test_ea_job_matches_batch_and_oracle(X):
    """A served EA job with exchange (default: a u per slot) and one without
    (shared u) against a batch handle and the oracle, bit for bit."""
    dims, ns = (8, 8, 8), 65
    bonds = inputs.ea_bonds(dims, 1, inputs.unit_seed(41))
    betas = inputs.geometric_ladder(0.2, 2.0)
    seed = inputs.unit_seed(42)
    srv = spn.Server(1 << 28)
    t = srv.submit(spn.SPN_EA3D_PMJ, dims, ns, seed, betas=betas, couplings=bonds[0], exchange_every=X)
    t2 = _submit_ising(srv, 1, *_MIX[1])
    _wait(srv, [t, t2])
    words, slots = srv.fetch(t)
    w = oracle.ea_init_hot(dims, 1, seed)
    pi = np.arange(32, dtype=np.uint8)[None, :].copy()
    tau = pi.copy()
    oracle.ea_sweeps(dims, w, bonds, betas, pi, tau, ns, seed, exchange_every=X)
    assert np.array_equal(words, w[0]) and np.array_equal(slots, pi[0])
    b = spn.EABatch(dims, bonds, betas, seed, exchange_every=X)
    b.sweep(ns)
    assert np.array_equal(words, b.words()[0]) and np.array_equal(slots, b.slots()[0])
    E, M = b.energies()
    s0 = int(np.nonzero(slots == 0)[0][0])
    done, res = srv.poll(t)
    assert (res.E, res.M) == (int(E[0, s0]), int(M[0, s0]))
    b.close()
    srv.close()


def test_budget_admission_and_rejection():
    d = (256, 256)
    per_job = 256 * 256 + 4096
    srv = spn.Server(2 * per_job + 100)  # two such jobs fit at a time
    with pytest.raises(spn.SpnError) as e:
        srv.submit(spn.SPN_ISING2D, (1024, 1024), 5, 1, beta=0.4)
    assert e.value.code == spn.SPN_E_BUDGET
    tickets = [srv.submit(spn.SPN_ISING2D, d, 30, inputs.unit_seed(800 + k), beta=0.42, stream=k) for k in range(6)]
    seen_max = 0
    t0 = time.monotonic()
    while True:
        st = srv.stats()
        seen_max = max(seen_max, st["used_bytes"])
        if all(srv.poll(t)[0] for t in tickets):
            break
        assert time.monotonic() - t0 < 120
    assert seen_max <= 2 * per_job + 100
    for k, t in enumerate(tickets):
        so = oracle.init_hot(d, inputs.unit_seed(800 + k), k)
        oracle.sweeps(d, so, 0.42, 30, inputs.unit_seed(800 + k), stream=k)
        assert np.array_equal(srv.fetch(t), so)
    srv.close()


def test_poll_unknown_and_early_fetch():
    srv = spn.Server(1 << 30)
    with pytest.raises(spn.SpnError) as e:
        srv.poll(12345)
    assert e.value.code == spn.SPN_E_NOTFOUND
    t = srv.submit(spn.SPN_ISING2D, (4096, 4096), 40, 3, beta=0.44)
    t0 = time.perf_counter()
    done, res = srv.poll(t)
    assert time.perf_counter() - t0 < 0.05  # polling does not wait for the GPU
    if not done:
        with pytest.raises(spn.SpnError) as e:
            srv.fetch(t)
        assert e.value.code == spn.SPN_E_STATE
    _wait(srv, [t])
    with pytest.raises(spn.SpnError):
        srv.submit(spn.SPN_ISING2D, (5, 4), 3, 1, beta=0.4)
    with pytest.raises(spn.SpnError) as e:  # 2^28 + 2 rows of two 64-site words: past the counter range
        srv.submit(spn.SPN_ISING2D, (66, (1 << 28) + 2), 3, 1, beta=0.4)
    assert e.value.code == spn.SPN_E_ARG and "counter" in str(e.value)
    srv.close()
