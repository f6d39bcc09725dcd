"""The autocorrelation-time estimator used to weigh the multi-hit order of
Sec. 3 against its autocorrelation cost, pinned to closed forms:

* an AR(1) process x_t = r x_{t-1} + sqrt(1 - r^2) e_t has rho(t) = r^t, so
  tau_int = 1/2 + r / (1 - r) = (1 + r) / (2 (1 - r));
* independent samples have tau_int = 1/2;
* the variance of the mean of n correlated samples is 2 tau_int sigma^2 / n
  (to O(tau / n)), an independent check of the factor 2 and of the sum;
* rho(t) of a short series equals the pair average written out by hand.
"""

from __future__ import annotations

import numpy as np
import pytest

from paper_1006_3865_gb300 import autocorr

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _ar1(r: float, n: int, runs: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    e = rng.standard_normal((runs, n))
    x = np.empty((runs, n))
    x[:, 0] = e[:, 0]
    s = np.sqrt(1.0 - r * r)
    for t in range(1, n):
        x[:, t] = r * x[:, t - 1] + s * e[:, t]
    return x


@pytest.mark.parametrize("r", [0.5, 0.8, 0.95])
def test_ar1_closed_form(r):
    x = _ar1(r, 20000, 8, seed=int(r * 1000))
    tau, err, w = autocorr.tau_int(x)
    exact = (1 + r) / (2 * (1 - r))
    tail = r ** (w + 1) / (1 - r)  # part of the sum beyond the window
    assert w >= 6 * tau
    assert abs(tau - exact) < 4 * err + tail, (tau, err, exact)


def test_independent_samples():
    rng = np.random.Generator(np.random.PCG64(5))
    tau, err, _ = autocorr.tau_int(rng.standard_normal((4, 50000)))
    assert abs(tau - 0.5) < 4 * err


def test_variance_of_the_mean():
    r, n, runs = 0.9, 4000, 400
    x = _ar1(r, n, runs, seed=11)
    tau, err, _ = autocorr.tau_int(x)
    # 2 tau sigma^2 / n with the finite-n sum written out
    t = np.arange(1, n)
    tau_n = 0.5 + np.sum((1 - t / n) * r ** t)
    v = x.mean(axis=1).var(ddof=1) * n / x.var()
    assert abs(v / 2 - tau_n) < 4 * tau_n * np.sqrt(2.0 / runs)
    assert abs(tau - tau_n) < 4 * err + 0.05 * tau_n


def test_rho_by_hand():
    x = np.array([1.0, 3.0, -2.0, 0.5, 4.0, -1.0, 2.0])
    d = x - x.mean()
    n = x.size
    gamma = [np.mean([d[i] * d[i + t] for i in range(n - t)]) for t in range(n)]
    np.testing.assert_allclose(autocorr.autocorrelation(x), np.array(gamma) / gamma[0], rtol=1e-12, atol=1e-12)


def test_runs_share_one_mean():
    a = np.array([[1.0, 2.0, 0.0, 1.5], [3.0, -1.0, 2.0, 0.5]])
    d = a - a.mean()
    g = [np.mean([d[k, i] * d[k, i + t] for k in range(2) for i in range(4 - t)]) for t in range(4)]
    np.testing.assert_allclose(autocorr.autocorrelation(a), np.array(g) / g[0], rtol=1e-12, atol=1e-12)


def test_rejects_constant_and_short():
    with pytest.raises(ValueError):
        autocorr.tau_int(np.ones(100))
    with pytest.raises(ValueError):
        autocorr.tau_int(np.ones(1))
