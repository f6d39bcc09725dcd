"""Batched runs of many uneven lattices: the persistent resident kernel (one
CTA, or a cluster of CTAs sharing rows through distributed shared memory)
against the CPU oracle and against the per-instance launch loop, bit for bit."""

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


def _jobs_small():
    rng = np.random.default_rng(11)
    jobs = []
    shapes = [(2, (32, 32)), (2, (64, 64)), (2, (128, 64)), (2, (256, 256)), (2, (16, 8)), (2, (2, 2)),
              (3, (16, 16, 16)), (3, (64, 8, 4)), (2, (64, 64)), (2, (1024, 1024)),
              (2, (34, 18)), (2, (130, 6)), (2, (202, 100)), (3, (6, 4, 10)), (3, (70, 6, 4)), (2, (1000, 998))]
    for k, (nd, dims) in enumerate(shapes):
        model = spn.SPN_ISING2D if nd == 2 else spn.SPN_ISING3D
        T = float(rng.uniform(1.5, 3.5)) if nd == 2 else float(rng.uniform(3.5, 5.5))
        jobs.append((model, dims, 1.0 / T, int(rng.integers(3, 40)), inputs.unit_seed(900 + k), k))
    return jobs


def test_batched_matches_oracle():
    jobs = _jobs_small()
    m = spn.Multi(jobs)
    m.run(spn.SPN_RUN_BATCHED)
    for k, (model, dims, beta, ns, seed, stream) in enumerate(jobs):
        s, E, M = m.result(k)
        so = oracle.init_hot(dims, seed, stream)
        _, _, tE, tM = oracle.sweeps(dims, so, beta, ns, seed, stream=stream)
        assert np.array_equal(s, so), (k, dims)
        assert np.array_equal(E, tE) and np.array_equal(M, tM), (k, dims)
    m.close()


def test_batched_equals_loop_and_replays():
    jobs = _jobs_small()
    m = spn.Multi(jobs)
    m.run(spn.SPN_RUN_LOOP)
    loop = [m.result(k) for k in range(len(jobs))]
    for _ in range(2):  # the second batched run replays the captured graph
        m.run(spn.SPN_RUN_BATCHED)
        for k in range(len(jobs)):
            s, E, M = m.result(k)
            assert np.array_equal(s, loop[k][0]) and np.array_equal(E, loop[k][1]) and np.array_equal(M, loop[k][2])
    m.close()


def test_cluster_resident_2048():
    """L = 2048 needs a 4-CTA cluster (512 KB of bits); compare with the loop."""
    jobs = [(spn.SPN_ISING2D, (2048, 2048), 1.0 / 2.3, 6, inputs.unit_seed(1), 0),
            (spn.SPN_ISING2D, (2048, 2048), 1.0 / 1.7, 5, inputs.unit_seed(2), 1)]
    m = spn.Multi(jobs)
    m.run(spn.SPN_RUN_LOOP)
    loop = [m.result(k) for k in range(2)]
    m.run(spn.SPN_RUN_BATCHED)
    for k in range(2):
        s, E, M = m.result(k)
        assert np.array_equal(s, loop[k][0]) and np.array_equal(E, loop[k][1])
    s, E, M = m.result(1)
    so = oracle.init_hot((2048, 2048), jobs[1][4], 1)
    _, _, tE, tM = oracle.sweeps((2048, 2048), so, jobs[1][2], 5, jobs[1][4], stream=1)
    assert np.array_equal(s, so) and np.array_equal(E, tE)
    m.close()


def test_uneven_batch_subset_against_loop():
    """A 64-instance slice of the uneven workload (L = 2^k, k in 5..11)."""
    inst = inputs.uneven_batch(64)
    jobs = [(spn.SPN_ISING2D, i.dims, i.beta, min(i.nsweeps, 60), i.seed, i.stream) for i in inst]
    m = spn.Multi(jobs)
    m.run(spn.SPN_RUN_BATCHED)
    bat = [m.result(k) for k in range(len(jobs))]
    m.run(spn.SPN_RUN_LOOP)
    for k in range(len(jobs)):
        s, E, M = m.result(k)
        assert np.array_equal(s, bat[k][0]) and np.array_equal(E, bat[k][1]) and np.array_equal(M, bat[k][2]), k
    m.close()


def test_rejects_unsupported_shapes():
    with pytest.raises(spn.SpnError):  # 4 MB of bits: more than a cluster of 8 CTAs holds
        spn.Multi([(spn.SPN_ISING2D, (8192, 4096), 0.4, 3, 1, 0)])
    with pytest.raises(spn.SpnError):  # odd extent
        spn.Multi([(spn.SPN_ISING2D, (48, 47), 0.4, 3, 1, 0)])


def test_autotuner_candidates_give_identical_results():
    """Every launch shape the autotuner may pick (cluster size, threads per
    CTA) gives the same lattices and traces, and so does its choice."""
    jobs = [(spn.SPN_ISING2D, (64, 64), 0.44, 30, inputs.unit_seed(600 + k), k) for k in range(6)]
    jobs += [(spn.SPN_ISING2D, (512, 256), 0.4, 12, inputs.unit_seed(610 + k), 10 + k) for k in range(3)]
    jobs += [(spn.SPN_ISING3D, (32, 16, 16), 0.22, 10, inputs.unit_seed(620 + k), 20 + k) for k in range(2)]
    m = spn.Multi(jobs)
    m.run(spn.SPN_RUN_BATCHED)
    ref = [m.result(k) for k in range(len(jobs))]
    groups = m.groups()
    assert len(groups) == 3
    for gi, g in enumerate(groups):
        for cs in (1, 2, 4, 8):
            for threads in (64, 128, 256):
                try:
                    m.set_launch(gi, cs, threads)
                except spn.SpnError:
                    continue  # that cluster size does not fit the shape
                m.run(spn.SPN_RUN_BATCHED)
                for k in range(len(jobs)):
                    got = m.result(k)
                    assert all(np.array_equal(x, y) for x, y in zip(got, ref[k])), (gi, cs, threads, k)
    tuned = m.autotune(5)
    assert all(t["trial_attempts_per_ns"] > 0 for t in tuned)
    m.run(spn.SPN_RUN_BATCHED)
    for k in range(len(jobs)):
        assert all(np.array_equal(x, y) for x, y in zip(m.result(k), ref[k]))
    m.close()
    # a new batch with the same shapes starts from the tuned launch shapes
    m2 = spn.Multi(jobs)
    assert [(g["cs"], g["threads"]) for g in m2.groups()] == [(t["cs"], t["threads"]) for t in tuned]
    m2.close()
