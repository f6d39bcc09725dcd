"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds no arithmetic of the method: it only draws seeds, couplings,
temperature ladders and workload descriptions, and packs couplings into the
library's bit layout.  The CUDA path and the CPU oracle each consume these
inputs independently.

Workloads (all synthetic; the paper measures on no public data set):
  * ``ising2d_small``   2D L=64, T = 2.269185 (Onsager T_c), 1000 sweeps.
  * ``plain_large``     2D L=16384 at T in {2.0, 2.269185, 3.0}, 200 sweeps each,
                        plus 3D L=512 at beta = 0.221654, 100 sweeps.
  * ``ea_batched``      3D +-J EA, L=32, 1024 samples, bonds iid +-1 (p = 1/2),
                        32 temperatures geometric on [0.2, 2.0], exchange every
                        10 sweeps, 10^4 sweeps.
  * ``uneven_batch``    4096 2D instances, L = 2^k with k uniform on {5..11},
                        T uniform on [1.5, 3.5], sweeps uniform on [100, 2000].
  * ``served_stream``   Poisson arrivals (mean gap 0.5 ms) of 2D / 3D / EA jobs.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

MASTER_SEED = 0x5EED5EED
_MASK64 = (1 << 64) - 1

TC_2D = 2.269185
BETA_C_3D = 0.221654


def splitmix64(x: int) -> int:
    """SplitMix64 finaliser (Steele, Lea, Flood 2014), used only to derive seeds."""
    z = (x + 0x9E3779B97F4A7C15) & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def unit_seed(unit: int, master: int = MASTER_SEED) -> int:
    """Per-unit seed: splitmix64(master xor unit id)."""
    return splitmix64((master ^ unit) & _MASK64)


def lattice_sites(dims) -> int:
    return int(np.prod(np.asarray(dims, dtype=np.int64)))


def bond_words(dims) -> int:
    return (lattice_sites(dims) + 63) // 64


def pack_bonds(J: np.ndarray) -> np.ndarray:
    """Pack couplings J[..., dir, n] in {+1, -1} into uint64 words [..., dir, nw].

    Bit (n % 64) of word n // 64 is set iff J = -1."""
    J = np.asarray(J)
    N = J.shape[-1]
    nw = (N + 63) // 64
    bits = np.zeros(J.shape[:-1] + (nw * 64,), dtype=np.uint8)
    bits[..., :N] = (J < 0).astype(np.uint8)
    b = bits.reshape(J.shape[:-1] + (nw, 64)).astype(np.uint64)
    weights = (np.uint64(1) << np.arange(64, dtype=np.uint64))
    return (b * weights).sum(axis=-1, dtype=np.uint64)


def unpack_bonds(words: np.ndarray, N: int) -> np.ndarray:
    """Inverse of pack_bonds: int8 couplings [..., dir, N] in {+1, -1}."""
    w = np.asarray(words, dtype=np.uint64)
    bits = (w[..., :, None] >> np.arange(64, dtype=np.uint64)) & np.uint64(1)
    bits = bits.reshape(w.shape[:-1] + (-1,))[..., :N]
    return (1 - 2 * bits.astype(np.int8)).astype(np.int8)


def ea_bonds(dims, nsamples: int, seed: int, p_negative: float = 0.5) -> np.ndarray:
    """iid +-J couplings, J = -1 with probability p_negative, packed [sample][dir][nw]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    N = lattice_sites(dims)
    nd = len(dims)
    J = np.where(rng.random((nsamples, nd, N)) < p_negative, -1, 1).astype(np.int8)
    return pack_bonds(J)


def uniform_bonds(dims, nsamples: int, value: int) -> np.ndarray:
    """All couplings equal to ``value`` (+1 or -1), packed [sample][dir][nw]."""
    N = lattice_sites(dims)
    J = np.full((nsamples, len(dims), N), value, dtype=np.int8)
    return pack_bonds(J)


def geometric_ladder(t_min: float, t_max: float, n: int = 32) -> np.ndarray:
    """n temperatures geometric on [t_min, t_max], as betas in ascending-T order."""
    k = np.arange(n, dtype=np.float64)
    T = t_min * (t_max / t_min) ** (k / (n - 1))
    return 1.0 / T


@dataclasses.dataclass
class Instance:
    dims: tuple
    beta: float
    nsweeps: int
    seed: int
    stream: int = 0


def uneven_batch(n_instances: int = 4096, master: int = MASTER_SEED, k_lo: int = 5, k_hi: int = 11,
                 t_lo: float = 1.5, t_hi: float = 3.5, s_lo: int = 100, s_hi: int = 2000) -> list[Instance]:
    """2D instances with L = 2^k (k uniform), T uniform, sweeps uniform."""
    rng = np.random.Generator(np.random.PCG64(splitmix64(master ^ 0xC4)))
    ks = rng.integers(k_lo, k_hi + 1, size=n_instances)
    Ts = rng.uniform(t_lo, t_hi, size=n_instances)
    ss = rng.integers(s_lo, s_hi + 1, size=n_instances)
    return [Instance((1 << int(k), 1 << int(k)), 1.0 / float(T), int(s), unit_seed(i, master), 0)
            for i, (k, T, s) in enumerate(zip(ks, Ts, ss))]


@dataclasses.dataclass
class Request:
    arrival_s: float
    model: int            # 1 = 2D Ising, 2 = 3D Ising, 3 = 3D EA (32-temperature ladder)
    dims: tuple
    beta: float           # Ising models
    betas: np.ndarray | None  # EA ladder (ascending T)
    nsweeps: int
    seed: int
    bonds: np.ndarray | None


def _even_round(x: float) -> int:
    return max(2, 2 * int(round(x / 2.0)))


def served_stream(n_requests: int = 2000, mean_gap_s: float = 0.5e-3, master: int = MASTER_SEED,
                  sweeps_lo: float = 1e2, sweeps_hi: float = 1e4) -> list[Request]:
    """Poisson arrivals of mixed jobs.

    2D L log-uniform on [64, 4096] (rounded to even), 3D L log-uniform on [16, 256]
    (even), EA L in {8, 16, 24, 32} with a 32-temperature geometric ladder on
    [T, 10 T]; T uniform on [0.5, 4.0]; sweeps log-uniform on [1e2, 1e4]."""
    rng = np.random.Generator(np.random.PCG64(splitmix64(master ^ 0xC5)))
    t = 0.0
    out = []
    for i in range(n_requests):
        t += float(rng.exponential(mean_gap_s))
        model = int(rng.integers(1, 4))
        T = float(rng.uniform(0.5, 4.0))
        ns = int(round(math.exp(rng.uniform(math.log(sweeps_lo), math.log(sweeps_hi)))))
        seed = unit_seed(0x50000 + i, master)
        if model == 1:
            L = _even_round(math.exp(rng.uniform(math.log(64), math.log(4096))))
            out.append(Request(t, 1, (L, L), 1.0 / T, None, ns, seed, None))
        elif model == 2:
            L = _even_round(math.exp(rng.uniform(math.log(16), math.log(256))))
            out.append(Request(t, 2, (L, L, L), 1.0 / T, None, ns, seed, None))
        else:
            L = int(rng.choice([8, 16, 24, 32]))
            dims = (L, L, L)
            out.append(Request(t, 3, dims, 0.0, geometric_ladder(T, 10.0 * T), ns, seed,
                               ea_bonds(dims, 1, splitmix64(seed))))
    return out
