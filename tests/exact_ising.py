"""Exact results for the 2D Ising model used to pin the CPU oracle.

* Brute-force enumeration of small periodic lattices (energies written from the
  Hamiltonian of Eq. 1 with numpy bit operations, independent of the oracle).
* Kaufman's partition function of the finite m x n torus, in the form used by
  Ferdinand and Fisher (Phys. Rev. 185, 832 (1969)) -- the exact finite-size
  reference the paper itself compares its 2D data with (Sec. 4).
  Its first and second beta-derivatives give the exact energy and energy
  variance (specific heat c = beta^2 Var(E) / N) the paper checks against.
* Onsager's internal energy per spin of the infinite lattice.
"""

from __future__ import annotations

import math

import mpmath as mp
import numpy as np


def enumerate_2d(Lx: int, Ly: int):
    """All 2^(Lx*Ly) states of the periodic Lx x Ly lattice: (E, M) arrays.

    Site n = x + Lx*y holds bit n of the state index; bit 1 means spin -1."""
    N = Lx * Ly
    idx = np.arange(1 << N, dtype=np.uint64)
    s = 1 - 2 * ((idx[:, None] >> np.arange(N, dtype=np.uint64)) & np.uint64(1)).astype(np.int8)
    s = s.reshape(-1, Ly, Lx).astype(np.int32)
    E = -(s * np.roll(s, -1, axis=2)).sum(axis=(1, 2)) - (s * np.roll(s, -1, axis=1)).sum(axis=(1, 2))
    M = s.sum(axis=(1, 2))
    return E.astype(np.int64), M.astype(np.int64)


def exact_averages(E: np.ndarray, M: np.ndarray, beta: float):
    """Canonical <E>, <|M|>, <E^2> from an enumerated spectrum."""
    w = np.exp(-beta * (E - E.min()).astype(np.float64))
    Z = w.sum()
    e = (w * E).sum() / Z
    am = (w * np.abs(M)).sum() / Z
    e2 = (w * E.astype(np.float64) ** 2).sum() / Z
    return e, am, e2


def log_z_enumerated(E: np.ndarray, beta: float) -> float:
    Emin = E.min()
    return float(-beta * Emin + np.log(np.exp(-beta * (E - Emin).astype(np.float64)).sum()))


def kaufman_log_z(m: int, n: int, K, dps: int = 40):
    """ln Z of the periodic m x n Ising torus at coupling K = beta J (mpmath).

    Z = 1/2 (2 sinh 2K)^(mn/2) [Z1 + Z2 + Z3 + Z4], with
    Z1,2 = prod_{r<n} 2 cosh|sinh (m/2 gamma_{2r+1}),
    Z3,4 = prod_{r<n} 2 cosh|sinh (m/2 gamma_{2r}),
    cosh gamma_l = cosh 2K coth 2K - cos(pi l / n), and the signed
    gamma_0 = 2K + ln tanh K."""
    with mp.workdps(dps):
        K = mp.mpf(K)
        c = mp.cosh(2 * K) / mp.tanh(2 * K)

        def gamma(l):
            if l % (2 * n) == 0:
                return 2 * K + mp.log(mp.tanh(K))
            return mp.acosh(c - mp.cos(mp.pi * l / n))

        half = mp.mpf(m) / 2
        z1 = z2 = z3 = z4 = mp.mpf(1)
        for r in range(n):
            go = gamma(2 * r + 1)
            ge = gamma(2 * r)
            z1 *= 2 * mp.cosh(half * go)
            z2 *= 2 * mp.sinh(half * go)
            z3 *= 2 * mp.cosh(half * ge)
            z4 *= 2 * mp.sinh(half * ge)
        pre = (mp.mpf(m * n) / 2) * mp.log(2 * mp.sinh(2 * K))
        return pre + mp.log((z1 + z2 + z3 + z4) / 2)


def kaufman_energy(m: int, n: int, beta: float) -> float:
    """Exact <E> = -d ln Z / d beta for the m x n torus (J = 1)."""
    with mp.workdps(60):
        b = mp.mpf(beta)
        h = mp.mpf("1e-15")
        d = (kaufman_log_z(m, n, b + h, dps=60) - kaufman_log_z(m, n, b - h, dps=60)) / (2 * h)
        return float(-d)


def kaufman_energy_variance(m: int, n: int, beta: float) -> float:
    """Exact Var(E) = d^2 ln Z / d beta^2 for the m x n torus (J = 1), by a
    central second difference at 80 digits (step 1e-12, truncation ~1e-24)."""
    with mp.workdps(80):
        b = mp.mpf(beta)
        h = mp.mpf("1e-12")

        def f(x):
            return kaufman_log_z(m, n, x, dps=80)

        return float((f(b + h) - 2 * f(b) + f(b - h)) / h ** 2)


def onsager_energy_per_spin(T: float) -> float:
    """Onsager's u(T) = -coth 2K [1 + (2/pi)(2 tanh^2 2K - 1) K(k)],
    k = 2 sinh 2K / cosh^2 2K, K(k) the complete elliptic integral of the first kind."""
    K = 1.0 / T
    k = 2.0 * math.sinh(2 * K) / math.cosh(2 * K) ** 2
    k2 = min(k * k, 1.0)
    if k2 == 1.0:  # T = T_c: the prefactor vanishes and the elliptic integral diverges logarithmically
        return -1.0 / math.tanh(2 * K)
    Kk = float(mp.ellipk(k2))
    return -1.0 / math.tanh(2 * K) * (1.0 + (2.0 / math.pi) * (2.0 * math.tanh(2 * K) ** 2 - 1.0) * Kk)


def binned_mean_err(x: np.ndarray, nbins: int = 32):
    """Mean and its error from nbins equal blocks (blocking removes autocorrelation)."""
    x = np.asarray(x, dtype=np.float64)
    n = len(x) // nbins * nbins
    b = x[:n].reshape(nbins, -1).mean(axis=1)
    return float(b.mean()), float(b.std(ddof=1) / math.sqrt(nbins))


def binned_variance_err(x: np.ndarray, nbins: int = 32):
    """Variance of a time series and its jackknife error over nbins equal blocks."""
    x = np.asarray(x, dtype=np.float64)
    n = len(x) // nbins * nbins
    b1 = x[:n].reshape(nbins, -1).mean(axis=1)
    b2 = (x[:n] ** 2).reshape(nbins, -1).mean(axis=1)
    full = float(b2.mean() - b1.mean() ** 2)
    loo1 = (b1.sum() - b1) / (nbins - 1)
    loo2 = (b2.sum() - b2) / (nbins - 1)
    jk = loo2 - loo1 ** 2
    return full, float(math.sqrt((nbins - 1) / nbins * ((jk - jk.mean()) ** 2).sum()))


def energy_histogram_pvalue(levels: np.ndarray, probs: np.ndarray, samples: np.ndarray, min_expected: float = 10.0):
    """Pearson chi-square p-value of sampled energies against exact level
    probabilities (levels ascending); adjacent levels are merged, in energy
    order, until each merged bin expects at least min_expected samples."""
    from scipy import stats

    n = len(samples)
    obs = np.array([(samples == e).sum() for e in levels], dtype=np.float64)
    assert obs.sum() == n, "a sampled energy is not an exact level"
    merged_o, merged_e, co, ce = [], [], 0.0, 0.0
    for o, e in zip(obs, n * probs):
        co, ce = co + o, ce + e
        if ce >= min_expected:
            merged_o.append(co)
            merged_e.append(ce)
            co = ce = 0.0
    merged_o[-1] += co
    merged_e[-1] += ce
    o, e = np.array(merged_o), np.array(merged_e)
    return float(stats.chisquare(o, e * o.sum() / e.sum()).pvalue)
