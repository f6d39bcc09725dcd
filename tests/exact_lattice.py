"""Exact enumeration helpers for tiny periodic lattices in 2D and 3D, written
from Eq. 1 and the sub-lattice procedure of Sec. 3 in numpy, independent of the
oracle: forward and backward neighbours, the energy of every state, and the
set of states the checkerboard sweep can reach from a start."""

from __future__ import annotations

import numpy as np


def neighbours(dims, step=-1):
    """Forward (step -1 of the roll) or backward (+1) neighbour of every site along each axis."""
    idx = np.arange(int(np.prod(dims))).reshape(dims[::-1])  # [z][y][x] or [y][x], x fastest
    nd = len(dims)
    return np.stack([np.roll(idx, step, axis=nd - 1 - d).reshape(-1) for d in range(nd)])


def energy(spins, J, nb):
    """E = -sum_n sum_d J[d][n] s_n s_{n + e_d} for spins [..., N] in {+1, -1}."""
    s = spins.astype(np.int64)
    return -sum((J[d] * s * s[..., nb[d]]).sum(axis=-1) for d in range(len(nb)))


def reachable(dims, J, start):
    """States the checkerboard sweep (colour 0, then colour 1, a move with
    dE <= 0 always taken, one with dE > 0 taken with probability in (0, 1))
    can reach from `start`, as a boolean mask over all 2^N states."""
    n_sites, nd = int(np.prod(dims)), len(dims)
    nb, bk = neighbours(dims), neighbours(dims, +1)
    colour = np.stack(np.unravel_index(np.arange(n_sites), dims[::-1])).sum(axis=0) & 1
    S = 1 - 2 * ((np.arange(1 << n_sites)[:, None] >> np.arange(n_sites)) & 1)
    dE = 2 * S * sum(J[d] * S[:, nb[d]] + J[d][bk[d]] * S[:, bk[d]] for d in range(nd))
    bits = np.int64(1) << np.arange(n_sites, dtype=np.int64)
    forced = [((dE <= 0) & (colour == c)) @ bits for c in (0, 1)]
    optional = [((dE > 0) & (colour == c)) @ bits for c in (0, 1)]

    def half(front, c):
        s = np.nonzero(front)[0]
        sites = np.nonzero(colour == c)[0]
        out = np.zeros(1 << n_sites, bool)
        for F in range(1 << len(sites)):
            m = int(sum(bits[sites[j]] for j in range(len(sites)) if (F >> j) & 1))
            out[s ^ forced[c][s] ^ (m & optional[c][s])] = True
        return out

    R = np.zeros(1 << n_sites, bool)
    R[start] = True
    front = R.copy()
    while front.any():
        nxt = half(half(front, 0), 1)
        front = nxt & ~R
        R |= nxt
    return R
