"""Integrated autocorrelation time of a per-sweep observable series.

Sec. 3 notes that the k-fold multi-hit of the double-checkerboard order lengthens
autocorrelation times near the critical point, so its throughput gain is worth
only as much as it is not eaten by slower decorrelation.  This module measures
that cost from the per-sweep energy / magnetisation traces the library records.

Estimator (Madras and Sokal, J. Stat. Phys. 50 (1988) 109):

    rho(t)     = Gamma(t) / Gamma(0),  Gamma(t) = mean over pairs (x_i - xbar)(x_{i+t} - xbar)
    tau_int(W) = 1/2 + sum_{t=1}^{W} rho(t)

with the window W the smallest one for which W >= c tau_int(W) (c = 6), and the
statistical error tau sqrt(2 (2 W + 1) / n) for n samples in all.  Several
independent runs of equal length (replicas) share one mean and one Gamma(t),
averaged over all pairs of all runs.  Host-side analysis only: it reads traces
that the GPU path wrote and computes nothing of the sweep itself.
"""

from __future__ import annotations

import numpy as np


def autocorrelation(series) -> np.ndarray:
    """rho(t), t = 0 .. n-1, of one series or of a 2D array of equal-length runs
    (one run per row), about the mean of all runs."""
    x = np.atleast_2d(np.asarray(series, dtype=np.float64))
    runs, n = x.shape
    if n < 2:
        raise ValueError("need at least two samples per run")
    d = x - x.mean()
    m = 1 << int(np.ceil(np.log2(2 * n)))  # zero padding: linear, not circular, correlation
    f = np.fft.rfft(d, m, axis=1)
    acf = np.fft.irfft(f * np.conj(f), m, axis=1)[:, :n].sum(axis=0)
    gamma = acf / (runs * (n - np.arange(n)))
    if gamma[0] <= 0.0:
        raise ValueError("the series is constant")
    return gamma / gamma[0]


def tau_int(series, c: float = 6.0) -> tuple[float, float, int]:
    """(tau_int, its error, window W) of one series or of equal-length runs.

    tau_int is in units of the sampling interval (one sweep of the trace).  If
    no window up to n - 1 satisfies W >= c tau, the last one is used and the
    estimate is a lower bound."""
    x = np.atleast_2d(np.asarray(series, dtype=np.float64))
    rho = autocorrelation(x)
    n = rho.size
    taus = 0.5 + np.cumsum(rho[1:])  # taus[W - 1] = tau_int(W)
    W = np.arange(1, n)
    ok = np.nonzero(W >= c * taus)[0]
    w = int(W[ok[0]]) if ok.size else n - 1
    tau = float(taus[w - 1])
    err = tau * np.sqrt(2.0 * (2 * w + 1) / x.size)
    return tau, float(err), w
