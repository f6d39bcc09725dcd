"""Pins of the oracle's Heisenberg (continuous-spin) sweep, the generalisation
Sec. 4 names for single-precision GPU arithmetic.

* The binary32 exp of the acceptance against the binary64 library exp: within
  4 ulp on [-87, 0], and 0 below -87.
* Marsaglia proposals: unit length, mean 0, <z^2> = 1/3, z and the azimuth
  uniform (Kolmogorov-Smirnov), as a uniform point on the sphere has.
* beta = 0 accepts every proposal: the lattice after a sweep is the sweep's
  proposals.
* The 2 x 2 torus is a ring of four spins with doubled bonds; its exact
  <E>(beta) follows from the ring partition function Z = sum_l (2l+1) i_l(K)^4
  (K = 2 beta, i_l the modified spherical Bessel functions; the transfer
  operator of a classical Heisenberg bond).  Long runs match it at three beta.
* 3D at small beta: each bond's <S.S'> = beta/3 + O(beta^3) (the leading
  high-temperature term), which fails if the sweep's field misses a direction.
* The incrementally tracked energy stays within binary32 rounding of a fresh
  recompute."""

from __future__ import annotations

import math

import numpy as np
import pytest
import scipy.special as sp
import scipy.stats as st

import oracle
from exact_ising import binned_mean_err, binned_variance_err


def test_exp_within_four_ulp():
    xs = np.concatenate([-np.logspace(-9, math.log10(87.0), 4000), np.linspace(-87.0, 0.0, 4001)]).astype(np.float32)
    for x in xs:
        got = float(oracle.heis_exp(x))
        ref = math.exp(float(x))
        assert abs(got - ref) <= 4 * np.spacing(np.float32(ref)), (x, got, ref)
    assert float(oracle.heis_exp(-87.01)) == 0.0 and float(oracle.heis_exp(-200.0)) == 0.0
    assert float(oracle.heis_exp(0.0)) == 1.0


def test_proposals_are_uniform_on_the_sphere():
    n = 60000
    P = np.array([oracle.heis_proposal(11, 3, 5, m & 1, 5, m) for m in range(n)])
    norm = np.linalg.norm(P.astype(np.float64), axis=1)
    assert np.abs(norm - 1).max() < 4e-7
    assert np.abs(P.mean(axis=0)).max() < 4 * math.sqrt(1 / 3 / n)
    assert abs((P[:, 2].astype(np.float64) ** 2).mean() - 1 / 3) < 4 * math.sqrt(4 / 45 / n)
    assert st.kstest(P[:, 2], "uniform", args=(-1, 2)).pvalue > 1e-3
    phi = np.arctan2(P[:, 1], P[:, 0])
    assert st.kstest(phi, "uniform", args=(-math.pi, 2 * math.pi)).pvalue > 1e-3


def test_beta_zero_takes_every_proposal():
    dims, seed = (6, 4, 4), 21
    S = oracle.heis_init_hot(dims, seed)
    oracle.heis_sweeps(dims, S, 0.0, 1, seed, sweep0=7)
    for n in range(S.shape[0]):
        x, y, z = n % 6, (n // 6) % 4, n // 24
        p = oracle.heis_proposal(seed, 0, 7, (x + y + z) & 1, 5, n >> 1)
        assert np.array_equal(S[n], p)


def _ring_energy(beta, N=4, J=2.0, lmax=60):
    K = J * beta
    l = np.arange(lmax)
    i = sp.spherical_in(l, K)
    di = sp.spherical_in(l, K, derivative=True)
    Z = ((2 * l + 1) * i ** N).sum()
    dZ = ((2 * l + 1) * N * i ** (N - 1) * di).sum() * J
    return -dZ / Z


@pytest.mark.parametrize("beta", [0.3, 1.0, 2.5])
def test_two_by_two_torus_matches_exact_ring(beta):
    dims, seed = (2, 2), 1000 + int(10 * beta)
    S = oracle.heis_init_hot(dims, seed)
    _, _, tE, _ = oracle.heis_sweeps(dims, S, beta, 200000, seed)
    m, e = binned_mean_err(tE[2000:], nbins=50)
    exact = _ring_energy(beta)
    assert abs(m - exact) < 4 * e, (beta, m, exact, e)


def test_ring_formula_limits():
    # beta -> 0: <E> -> 0; small K: each of 4 doubled bonds has <S.S'> = K/3
    assert abs(_ring_energy(1e-4) - (-4 * 2 * (2e-4) / 3)) < 1e-9
    # large beta: the ring orders; 4 spins x 2 angles less the 2 of the common
    # direction leave 6 quadratic modes of 1 / (2 beta) each: E -> -8 + 3 / beta
    assert _ring_energy(50.0) == pytest.approx(-8 + 3 / 50.0, abs=1e-3)
    assert _ring_energy(20.0) == pytest.approx(-8 + 3 / 20.0, abs=1e-3)


def _ring_energy_variance(beta, N=4, J=2.0, lmax=60):
    """Var(E) = d^2 ln Z / d beta^2 of the same ring; i_l'' from the modified
    spherical Bessel equation x^2 i'' + 2 x i' - l (l + 1) i = x^2 i."""
    K = J * beta
    l = np.arange(lmax)
    i = sp.spherical_in(l, K)
    d1 = sp.spherical_in(l, K, derivative=True)
    d2 = i * (1 + l * (l + 1) / K ** 2) - 2 * d1 / K
    w = 2 * l + 1
    Z = (w * i ** N).sum()
    Z1 = (w * N * i ** (N - 1) * d1).sum() * J
    Z2 = (w * (N * (N - 1) * i ** (N - 2) * d1 ** 2 + N * i ** (N - 1) * d2)).sum() * J ** 2
    return Z2 / Z - (Z1 / Z) ** 2


def test_ring_variance_limits():
    # beta -> 0: four uncorrelated doubled bonds, -2 S.S' with S.S' uniform on [-1, 1]
    assert _ring_energy_variance(1e-3) == pytest.approx(16 / 3, rel=1e-5)
    # large beta: six quadratic modes, Var(E) = -d<E>/d beta -> 3 / beta^2
    assert _ring_energy_variance(50.0) == pytest.approx(3 / 50.0 ** 2, rel=0.02)


@pytest.mark.parametrize("beta", [0.3, 1.0, 2.5])
def test_two_by_two_torus_specific_heat_matches_exact_ring(beta):
    """The energy fluctuations of the same runs (c = beta^2 Var(E) / N)
    against the exact ring, within 4 jackknife sigma."""
    dims, seed = (2, 2), 1000 + int(10 * beta)
    S = oracle.heis_init_hot(dims, seed)
    _, _, tE, _ = oracle.heis_sweeps(dims, S, beta, 200000, seed)
    v, ev = binned_variance_err(tE[2000:], nbins=50)
    exact = _ring_energy_variance(beta)
    assert abs(v - exact) < 4 * ev, (beta, v, exact, ev)


def test_3d_high_temperature_bond_correlation():
    dims, seed, beta = (8, 8, 8), 5, 0.05
    S = oracle.heis_init_hot(dims, seed)
    _, _, tE, _ = oracle.heis_sweeps(dims, S, beta, 3000, seed)
    bonds = 3 * 512
    m, e = binned_mean_err(tE[200:] / bonds)
    assert abs(m + beta / 3) < 4 * e + beta ** 3, (m, -beta / 3, e)


def test_incremental_energy_tracks_recompute():
    dims, seed = (16, 12), 8
    S = oracle.heis_init_hot(dims, seed)
    E, M, tE, tM = oracle.heis_sweeps(dims, S, 0.7, 50, seed)
    Er, Mr = oracle.heis_observables(dims, S)
    # each accepted move adds its binary32 dE (relative rounding <= 2^-23 of |dS| |h| <= 8)
    moves = 50 * 192
    assert abs(E - Er) < moves * 8 * 2.0 ** -22
    assert np.abs(M - Mr).max() < moves * 2 * 2.0 ** -23
