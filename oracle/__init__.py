"""CPU oracle for the checkerboard Metropolis sweep (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import this package.  The product path (the CUDA library in
``paper_1006_3865_gb300``) never does, and the two share no code: the oracle is
plain C (``spn_oracle.c``) written from the paper's Eq. 1-2 and the sub-lattice
procedure of Sec. 3, loaded here through ctypes.

Every wrapper takes and returns numpy arrays; see ``spn_oracle.c`` for the exact
definitions (site order, colours, Philox counters, thresholds, exchange rule).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spn_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``spn_oracle.c`` with gcc (OpenMP if available) and return the path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp", "-o", tmp, _SRC, "-lm"], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp, _SRC, "-lm"], check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            u32, u64, i64, dbl, cint, vp = (ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64,
                                           ctypes.c_double, ctypes.c_int, ctypes.c_void_p)
            L.orc_philox4x32_10.argtypes = [vp, vp, vp]
            L.orc_philox4x32_10.restype = None
            L.orc_site_word.argtypes = [u64, u32, u32, cint, cint, u64]
            L.orc_site_word.restype = u32
            L.orc_metropolis_u.argtypes = [u64, u32, u32, cint, u64]
            L.orc_metropolis_u.restype = u32
            L.orc_hot_word.argtypes = [u64, u32, cint, u64]
            L.orc_hot_word.restype = u32
            L.orc_threshold.argtypes = [dbl, cint]
            L.orc_threshold.restype = u64
            L.orc_accept.argtypes = [dbl, cint, u32]
            L.orc_accept.restype = cint
            L.orc_delta_e.argtypes = [cint, vp, vp, vp, i64]
            L.orc_delta_e.restype = cint
            L.orc_observables.argtypes = [cint, vp, vp, vp, vp, vp]
            L.orc_observables.restype = cint
            L.orc_init_hot.argtypes = [cint, vp, u64, u32, vp]
            L.orc_init_hot.restype = cint
            L.orc_sweeps.argtypes = [cint, vp, vp, vp, dbl, u64, u32, u32, i64, vp, vp, vp, vp]
            L.orc_sweeps.restype = cint
            L.orc_sweeps_ex.argtypes = [cint, vp, vp, vp, dbl, u64, u32, u32, i64, cint, vp, vp, vp, vp]
            L.orc_sweeps_ex.restype = cint
            L.orc_sweeps_dc.argtypes = [cint, vp, vp, vp, cint, dbl, u64, u32, u32, i64, vp, vp, vp, vp]
            L.orc_sweeps_dc.restype = cint
            L.orc_msc_u.argtypes = [u64, u32, u32, cint, u64]
            L.orc_msc_u.restype = u32
            L.orc_ea_init_hot.argtypes = [cint, vp, cint, u64, u32, vp]
            L.orc_ea_init_hot.restype = cint
            L.orc_ea_observables.argtypes = [cint, vp, cint, vp, vp, vp, vp]
            L.orc_ea_observables.restype = cint
            L.orc_ea_sweeps.argtypes = [cint, vp, cint, vp, vp, vp, vp, vp, u64, u32, u32, i64, cint, vp]
            L.orc_ea_sweeps.restype = cint
            L.orc_ea_sweeps_ex.argtypes = [cint, vp, cint, vp, vp, vp, vp, vp, u64, u32, u32, i64, cint, vp, cint]
            L.orc_ea_sweeps_ex.restype = cint
            L.orc_ea_dp_group.argtypes = [cint]
            L.orc_ea_dp_group.restype = cint
            L.orc_ea_dp_sweeps.argtypes = [cint, vp, cint, vp, vp, vp, u64, u32, i64, cint, vp, cint]
            L.orc_ea_dp_sweeps.restype = cint
            L.orc_ea_overlap.argtypes = [cint, vp, cint, vp, vp, vp]
            L.orc_ea_overlap.restype = cint
            flt = ctypes.c_float
            L.orc_heis_exp.argtypes = [flt]
            L.orc_heis_exp.restype = flt
            L.orc_heis_proposal.argtypes = [u64, u32, u32, cint, cint, u64, vp]
            L.orc_heis_proposal.restype = cint
            L.orc_heis_init_hot.argtypes = [cint, vp, u64, u32, vp]
            L.orc_heis_init_hot.restype = cint
            L.orc_heis_observables.argtypes = [cint, vp, vp, vp, vp]
            L.orc_heis_observables.restype = cint
            L.orc_heis_sweeps.argtypes = [cint, vp, vp, dbl, u64, u32, u32, i64, vp, vp, vp, vp]
            L.orc_heis_sweeps.restype = cint
            L.orc_num_threads.argtypes = []
            L.orc_num_threads.restype = cint
            L.orc_set_num_threads.argtypes = [cint]
            L.orc_set_num_threads.restype = None
            _lib = L
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _dims(dims) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(dims, dtype=np.int64))


def _bonds(bonds):
    return None if bonds is None else np.ascontiguousarray(bonds, dtype=np.uint64)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle: {what} rejected its arguments (rc={rc})")


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(n: int):
    """Threads of the oracle's OpenMP loops (1: serial)."""
    lib().orc_set_num_threads(int(n))


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def site_word(seed: int, stream: int, t: int, colour: int, purpose: int, m: int) -> int:
    """Plane word of site key m (the within-colour index when Lx % 64 == 0)."""
    return int(lib().orc_site_word(seed, stream, t, colour, purpose, m))


def metropolis_u(seed: int, stream: int, sweep: int, colour: int, m: int) -> int:
    return int(lib().orc_metropolis_u(seed, stream, sweep, colour, m))


def hot_word(seed: int, stream: int, colour: int, m: int) -> int:
    return int(lib().orc_hot_word(seed, stream, colour, m))


def threshold(beta: float, dE: int) -> int:
    return int(lib().orc_threshold(float(beta), int(dE)))


def accept(beta: float, dE: int, u: int) -> bool:
    return bool(lib().orc_accept(float(beta), int(dE), int(u)))


def delta_e(dims, spins: np.ndarray, n: int, bonds=None) -> int:
    d = _dims(dims)
    s = np.ascontiguousarray(spins, dtype=np.int8).reshape(-1)
    return int(lib().orc_delta_e(len(d), _p(d), _p(s), _p(_bonds(bonds)), int(n)))


def observables(dims, spins: np.ndarray, bonds=None) -> tuple[int, int]:
    d = _dims(dims)
    s = np.ascontiguousarray(spins, dtype=np.int8).reshape(-1)
    E = np.zeros(1, np.int64)
    M = np.zeros(1, np.int64)
    _check(lib().orc_observables(len(d), _p(d), _p(s), _p(_bonds(bonds)), _p(E), _p(M)), "observables")
    return int(E[0]), int(M[0])


def init_hot(dims, seed: int, stream: int = 0) -> np.ndarray:
    d = _dims(dims)
    s = np.zeros(int(np.prod(d)), dtype=np.int8)
    _check(lib().orc_init_hot(len(d), _p(d), seed, stream, _p(s)), "init_hot")
    return s


def msc_u(seed: int, stream: int, sweep: int, colour: int, m: int) -> int:
    return int(lib().orc_msc_u(seed, stream, sweep, colour, m))


def sweeps(dims, spins: np.ndarray, beta: float, nsweeps: int, seed: int, stream: int = 0,
           sweep0: int = 0, bonds=None, E: int | None = None, M: int | None = None, msc_u_words: bool = False):
    """Run ``nsweeps`` sweeps in place on ``spins`` (flat int8, site order n).

    Returns (E, M, traceE, traceM) with the per-sweep integer trace.  With
    ``msc_u_words`` the sites draw u as the multi-spin coded path does."""
    d = _dims(dims)
    if spins.dtype != np.int8 or not spins.flags.c_contiguous:
        raise TypeError("spins must be a contiguous int8 array")
    b = _bonds(bonds)
    if E is None or M is None:
        E, M = observables(d, spins, b)
    Ea = np.array([E], np.int64)
    Ma = np.array([M], np.int64)
    tE = np.zeros(max(nsweeps, 1), np.int64)
    tM = np.zeros(max(nsweeps, 1), np.int64)
    _check(lib().orc_sweeps_ex(len(d), _p(d), _p(spins), _p(b), float(beta), seed, stream, sweep0, int(nsweeps),
                               1 if msc_u_words else 0, _p(Ea), _p(Ma), _p(tE), _p(tM)), "sweeps")
    return int(Ea[0]), int(Ma[0]), tE[:nsweeps], tM[:nsweeps]


def sweeps_dc(dims, spins: np.ndarray, tile, hits: int, beta: float, nsweeps: int, seed: int, stream: int = 0,
              sweep0: int = 0, E: int | None = None, M: int | None = None):
    """Double-checkerboard sweeps with `hits`-fold multi-hit on tiles of extent
    `tile` (Sec. 3), in place.  Returns (E, M, traceE, traceM)."""
    d = _dims(dims)
    T = _dims(tile)
    if spins.dtype != np.int8 or not spins.flags.c_contiguous:
        raise TypeError("spins must be a contiguous int8 array")
    if E is None or M is None:
        E, M = observables(d, spins)
    Ea = np.array([E], np.int64)
    Ma = np.array([M], np.int64)
    tE = np.zeros(max(nsweeps, 1), np.int64)
    tM = np.zeros(max(nsweeps, 1), np.int64)
    _check(lib().orc_sweeps_dc(len(d), _p(d), _p(spins), _p(T), int(hits), float(beta), seed, stream, sweep0,
                               int(nsweeps), _p(Ea), _p(Ma), _p(tE), _p(tM)), "sweeps_dc")
    return int(Ea[0]), int(Ma[0]), tE[:nsweeps], tM[:nsweeps]


def ea_init_hot(dims, nsamples: int, seed: int, stream0: int = 0) -> np.ndarray:
    d = _dims(dims)
    N = int(np.prod(d))
    sp = np.zeros((nsamples, N), dtype=np.uint32)
    _check(lib().orc_ea_init_hot(len(d), _p(d), nsamples, seed, stream0, _p(sp)), "ea_init_hot")
    return sp


def ea_observables(dims, words: np.ndarray, bonds: np.ndarray):
    """Per-replica (E, M), each of shape [nsamples, 32], indexed by slot."""
    d = _dims(dims)
    w = np.ascontiguousarray(words, dtype=np.uint32)
    ns = w.shape[0]
    E = np.zeros((ns, 32), np.int64)
    M = np.zeros((ns, 32), np.int64)
    _check(lib().orc_ea_observables(len(d), _p(d), ns, _p(w), _p(_bonds(bonds)), _p(E), _p(M)), "ea_observables")
    return E, M


def ea_sweeps(dims, words: np.ndarray, bonds: np.ndarray, betas, temp_of_slot: np.ndarray,
              slot_of_temp: np.ndarray, nsweeps: int, seed: int, stream0: int = 0, sweep0: int = 0,
              exchange_every: int = 0, acc: np.ndarray | None = None, u_per_slot: bool | None = None):
    """Multi-spin coded sweeps, in place on ``words`` [nsamples, N] and the slot maps.
    u_per_slot: every temperature slot draws its own u (32 bit planes, eight
    Philox calls per site) instead of sharing the site's one u; None takes the
    per-slot u with replica exchange (exchange_every > 0) and the shared u
    without, as a batch does by default."""
    if u_per_slot is None:
        u_per_slot = exchange_every > 0
    d = _dims(dims)
    for a, dt in ((words, np.uint32), (temp_of_slot, np.uint8), (slot_of_temp, np.uint8)):
        if a.dtype != dt or not a.flags.c_contiguous:
            raise TypeError("ea_sweeps: in/out arrays must be contiguous with the documented dtypes")
    be = np.ascontiguousarray(np.asarray(betas, dtype=np.float64))
    if be.shape != (32,):
        raise ValueError("ea_sweeps: 32 betas required")
    if acc is not None and (acc.dtype != np.int64 or not acc.flags.c_contiguous):
        raise TypeError("acc must be contiguous int64")
    _check(lib().orc_ea_sweeps_ex(len(d), _p(d), words.shape[0], _p(words), _p(_bonds(bonds)), _p(be),
                                  _p(temp_of_slot), _p(slot_of_temp), seed, stream0, sweep0, int(nsweeps),
                                  int(exchange_every), _p(acc), 1 if u_per_slot else 0), "ea_sweeps")


def ea_dp_group(sample: int) -> int:
    """Group of a sample in the disorder-parallel layout (its 32 samples share u)."""
    return int(lib().orc_ea_dp_group(sample))


def ea_dp_sweeps(dims, words: np.ndarray, bonds: np.ndarray, betas, nsweeps: int, seed: int, sweep0: int = 0,
                 exchange_every: int = 0, acc: np.ndarray | None = None, sample0: int = 0):
    """Disorder-parallel multi-spin coded sweeps, in place on ``words`` [nsamples, N]
    (bit t = the configuration at temperature t): the samples of a group share
    the site's u at each temperature, replica exchange swaps configurations.
    acc: [nsamples, 32] int64 exchange counters (optional).  Row i is sample
    sample0 + i of the batch."""
    d = _dims(dims)
    if words.dtype != np.uint32 or not words.flags.c_contiguous:
        raise TypeError("ea_dp_sweeps: words must be contiguous uint32")
    be = np.ascontiguousarray(np.asarray(betas, dtype=np.float64))
    if be.shape != (32,):
        raise ValueError("ea_dp_sweeps: 32 betas required")
    if acc is not None and (acc.dtype != np.int64 or not acc.flags.c_contiguous):
        raise TypeError("acc must be contiguous int64")
    _check(lib().orc_ea_dp_sweeps(len(d), _p(d), words.shape[0], _p(words), _p(_bonds(bonds)), _p(be), seed,
                                  sweep0, int(nsweeps), int(exchange_every), _p(acc), int(sample0)), "ea_dp_sweeps")


def ea_overlap(dims, words: np.ndarray, slot_of_temp: np.ndarray) -> np.ndarray:
    """Overlaps q[p, t] = sum_n s_n^(2p)(t) s_n^(2p+1)(t) of the replica pairs
    (samples 2p, 2p+1) at every temperature index t; shape [nsamples // 2, 32]."""
    d = _dims(dims)
    w = np.ascontiguousarray(words, dtype=np.uint32)
    sot = np.ascontiguousarray(slot_of_temp, dtype=np.uint8)
    if w.shape[0] % 2 or sot.shape != (w.shape[0], 32):
        raise ValueError("ea_overlap: an even number of samples and [nsamples, 32] slot maps")
    q = np.zeros((w.shape[0] // 2, 32), np.int64)
    _check(lib().orc_ea_overlap(len(d), _p(d), w.shape[0] // 2, _p(w), _p(sot), _p(q)), "ea_overlap")
    return q


def binder(q2: np.ndarray, q4: np.ndarray) -> np.ndarray:
    """Binder cumulant of the overlap per temperature, g = (3 - [<q^4>] / [<q^2>]^2) / 2,
    from per-pair thermal moments <q^2>, <q^4> (shape [pairs, T]); [.] is the
    average over pairs (disorder realisations)."""
    m2 = np.mean(np.asarray(q2, dtype=np.float64), axis=0)
    m4 = np.mean(np.asarray(q4, dtype=np.float64), axis=0)
    return 0.5 * (3.0 - m4 / (m2 * m2))


# ---- Heisenberg spins (binary32 vectors, [N, 3])

def heis_exp(x: float) -> np.float32:
    """The deterministic binary32 exp of the Heisenberg acceptance (x <= 0)."""
    return np.float32(lib().orc_heis_exp(float(np.float32(x))))


def heis_proposal(seed: int, stream: int, t: int, colour: int, purpose: int, m: int):
    """Marsaglia proposal of site key m (purpose 5: Metropolis, 7: hot start), or None."""
    out = np.zeros(3, np.float32)
    ok = lib().orc_heis_proposal(seed, stream, t, colour, purpose, m, _p(out))
    return out if ok else None


def heis_init_hot(dims, seed: int, stream: int = 0) -> np.ndarray:
    d = _dims(dims)
    S = np.zeros((int(np.prod(d)), 3), np.float32)
    _check(lib().orc_heis_init_hot(len(d), _p(d), seed, stream, _p(S)), "heis_init_hot")
    return S


def heis_observables(dims, S: np.ndarray):
    """(E, M[3]) in binary64, summed in site order."""
    d = _dims(dims)
    s = np.ascontiguousarray(S, dtype=np.float32)
    E = np.zeros(1, np.float64)
    M = np.zeros(3, np.float64)
    _check(lib().orc_heis_observables(len(d), _p(d), _p(s), _p(E), _p(M)), "heis_observables")
    return float(E[0]), M


def heis_sweeps(dims, S: np.ndarray, beta: float, nsweeps: int, seed: int, stream: int = 0, sweep0: int = 0,
                E: float | None = None, M=None):
    """Heisenberg sweeps in place on S (binary32 [N, 3]).  Returns (E, M, traceE, traceM[n, 3])."""
    d = _dims(dims)
    if S.dtype != np.float32 or not S.flags.c_contiguous or S.shape != (int(np.prod(d)), 3):
        raise TypeError("S must be a contiguous float32 [N, 3] array")
    if E is None or M is None:
        E, M = heis_observables(d, S)
    Ea = np.array([E], np.float64)
    Ma = np.array(M, np.float64).copy()
    tE = np.zeros(max(nsweeps, 1), np.float64)
    tM = np.zeros((max(nsweeps, 1), 3), np.float64)
    _check(lib().orc_heis_sweeps(len(d), _p(d), _p(S), float(beta), seed, stream, sweep0, int(nsweeps), _p(Ea),
                                 _p(Ma), _p(tE), _p(tM)), "heis_sweeps")
    return float(Ea[0]), Ma, tE[:nsweeps], tM[:nsweeps]
