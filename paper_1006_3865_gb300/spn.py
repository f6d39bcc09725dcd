"""Thin ctypes binding of libspn (the C ABI in ``include/spn.h``).

Argument marshalling only: every step of a sweep runs in the CUDA kernels of
``libspn.so``.  ``load()`` fails loudly when the library has not been built or
cannot be loaded; there is no CPU fallback.
"""

from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libspn.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
HEADER = os.path.join(INCLUDE, "spn.h")
HEADERS = (HEADER, os.path.join(INCLUDE, "spn_testing.h"))

SPN_OK = 0
SPN_E_ARG = -1
SPN_E_NOMEM = -2
SPN_E_BUDGET = -3
SPN_E_CUDA = -4
SPN_E_TIMEOUT = -5
SPN_E_STATE = -6
SPN_E_NOTFOUND = -7

SPN_ISING2D = 1
SPN_ISING3D = 2
SPN_EA3D_PMJ = 3
SPN_EA2D_PMJ = 4
SPN_HEIS2D = 5
SPN_HEIS3D = 6

SPN_INIT_HOT = 0
SPN_INIT_COLD = 1

SPN_RUN_BATCHED = 0
SPN_RUN_LOOP = 1

PATH_GENERIC = 0
PATH_STREAM = 1
PATH_RESIDENT = 2
PATH_PACKED = 3

_lock = threading.Lock()
_lib = None

_c = ctypes
_vp, _i32, _i64, _u32, _u64, _dbl, _sz = (_c.c_void_p, _c.c_int32, _c.c_int64, _c.c_uint32, _c.c_uint64,
                                          _c.c_double, _c.c_size_t)
_P = _c.POINTER

# name -> (restype, argtypes); every entry is an extern "C" function of spn.h
_SIGNATURES = {
    "spn_last_error": (_c.c_char_p, []),
    "spn_version": (_c.c_char_p, []),
    "spn_create": (_c.c_int, [_P(_vp), _c.c_int, _vp, _vp, _u64]),
    "spn_create_ex": (_c.c_int, [_P(_vp), _c.c_int, _vp, _vp, _u64, _u32, _c.c_int]),
    "spn_sweep": (_c.c_int, [_vp, _dbl, _i64]),
    "spn_sweep_dc": (_c.c_int, [_vp, _dbl, _i64, _P(_i32), _i32]),
    "spn_test_expire_next_waits": (_c.c_int, [_vp, _u32]),
    "spn_observables": (_c.c_int, [_vp, _P(_i64), _P(_i64)]),
    "spn_recompute": (_c.c_int, [_vp, _P(_i64), _P(_i64)]),
    "spn_trace": (_c.c_int, [_vp, _vp, _vp, _i64, _P(_i64)]),
    "spn_get_spins": (_c.c_int, [_vp, _vp, _sz]),
    "spn_set_spins": (_c.c_int, [_vp, _vp, _sz]),
    "spn_sweep_count": (_c.c_int, [_vp, _P(_u64)]),
    "spn_set_stream": (_c.c_int, [_vp, _vp]),
    "spn_sync": (_c.c_int, [_vp]),
    "spn_destroy": (_c.c_int, [_vp]),
    "spn_set_tiling": (_c.c_int, [_vp, _i32, _i32, _i32]),
    "spn_get_path": (_c.c_int, [_vp, _P(_i32)]),
    "spn_set_path": (_c.c_int, [_vp, _i32]),
    "spn_reinit": (_c.c_int, [_vp, _u64, _u32, _c.c_int]),
    "spn_launch_count": (_c.c_int, [_P(_u64)]),
    "spn_sweep_noalloc": (_c.c_int, [_c.c_int, _vp, _vp, _dbl, _u64, _u32, _u32, _i64, _vp, _vp]),
    "spn_multi_create": (_c.c_int, [_P(_vp), _vp, _c.c_int]),
    "spn_multi_run": (_c.c_int, [_vp, _c.c_int]),
    "spn_multi_sync": (_c.c_int, [_vp]),
    "spn_multi_result": (_c.c_int, [_vp, _c.c_int, _vp, _sz, _vp, _vp, _i64]),
    "spn_multi_set_stream": (_c.c_int, [_vp, _vp]),
    "spn_multi_destroy": (_c.c_int, [_vp]),
    "spn_server_create": (_c.c_int, [_P(_vp), _sz]),
    "spn_submit": (_c.c_int, [_vp, _vp, _P(_u64)]),
    "spn_poll": (_c.c_int, [_vp, _u64, _P(_c.c_int), _vp]),
    "spn_server_fetch": (_c.c_int, [_vp, _u64, _vp, _sz]),
    "spn_server_stats": (_c.c_int, [_vp, _P(_u64), _P(_dbl), _P(_u64), _P(_sz)]),
    "spn_server_destroy": (_c.c_int, [_vp]),
    "spn_create_batch": (_c.c_int, [_P(_vp), _c.c_int, _vp, _c.c_int, _vp, _vp, _c.c_int, _u64, _c.c_int]),
    "spn_batch_set_u_per_slot": (_c.c_int, [_vp, _c.c_int32]),
    "spn_create_batch_dp": (_c.c_int, [_P(_vp), _c.c_int, _vp, _c.c_int, _vp, _vp, _c.c_int, _u64, _c.c_int]),
    "spn_batch_sweep": (_c.c_int, [_vp, _i64]),
    "spn_batch_get_words": (_c.c_int, [_vp, _vp, _sz]),
    "spn_batch_set_words": (_c.c_int, [_vp, _vp, _sz]),
    "spn_batch_get_slots": (_c.c_int, [_vp, _vp, _sz]),
    "spn_batch_set_slots": (_c.c_int, [_vp, _vp, _sz]),
    "spn_batch_energies": (_c.c_int, [_vp, _vp, _vp, _sz]),
    "spn_batch_exchange_counts": (_c.c_int, [_vp, _vp, _sz]),
    "spn_batch_measure_overlap": (_c.c_int, [_vp]),
    "spn_multi_autotune": (_c.c_int, [_vp, _i32, _vp, _sz]),
    "spn_autotune": (_c.c_int, [_vp, _dbl, _i32, _vp]),
    "spn_multi_groups": (_c.c_int, [_vp, _vp, _sz]),
    "spn_multi_set_launch": (_c.c_int, [_vp, _i32, _i32, _i32]),
    "spn_heis_get_spins": (_c.c_int, [_vp, _vp, _sz]),
    "spn_heis_set_spins": (_c.c_int, [_vp, _vp, _sz]),
    "spn_heis_observables": (_c.c_int, [_vp, _vp, _vp]),
    "spn_heis_recompute": (_c.c_int, [_vp, _vp, _vp]),
    "spn_heis_trace": (_c.c_int, [_vp, _vp, _vp, _c.c_int64, _vp]),
    "spn_test_heis_exp": (_c.c_int, [_vp, _vp, _sz]),
    "spn_batch_overlap": (_c.c_int, [_vp, _vp, _vp, _vp, _vp, _sz]),
    "spn_batch_overlap_reset": (_c.c_int, [_vp]),
}


class Job(ctypes.Structure):
    """spn_job: one lattice of a batched run."""

    _fields_ = [("model", ctypes.c_int32), ("dims", ctypes.c_int32 * 3), ("beta", ctypes.c_double),
                ("nsweeps", ctypes.c_int64), ("seed", ctypes.c_uint64), ("stream", ctypes.c_uint32),
                ("reserved", ctypes.c_int32)]


class Request(ctypes.Structure):
    """spn_request."""

    _fields_ = [("model", ctypes.c_int32), ("dims", ctypes.c_int32 * 3), ("beta", ctypes.c_double),
                ("betas", ctypes.c_void_p), ("nsweeps", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("stream", ctypes.c_uint32), ("exchange_every", ctypes.c_int32), ("couplings", ctypes.c_void_p)]


class Result(ctypes.Structure):
    """spn_result."""

    _fields_ = [("status", ctypes.c_int32), ("state", ctypes.c_int32), ("sweeps", ctypes.c_int64),
                ("E", ctypes.c_int64), ("M", ctypes.c_int64), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


class SpnError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libspn error {code}: {msg}")
        self.code = code


def header_functions() -> list[str]:
    """Names of the functions declared in include/spn.h and include/spn_testing.h."""
    text = "".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(spn_[a-z0-9_]+)\s*\(", text)))


# A server round runs more concurrent launches than CUDA's default 8 hardware
# work queues; this takes effect only if no CUDA context exists yet.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")


def load(path: str | None = None):
    """Load libspn.so (build it first with paper_1006_3865_gb300.build.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libspn.so not found at {p}: run __graft_entry__.build() "
                               "(or paper_1006_3865_gb300.build.build()) first; there is no CPU fallback")
        lib = ctypes.CDLL(p)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _check(rc: int):
    if rc != SPN_OK:
        raise SpnError(rc, load().spn_last_error().decode(errors="replace"))


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(_vp)


def _dims(dims) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(dims, dtype=np.int32))


def _stream_ptr(stream) -> int | None:
    """cudaStream_t of a torch.cuda.Stream (or an int / None)."""
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def launch_count() -> int:
    """Kernels launched by libspn in this process so far."""
    c = _u64()
    _check(load().spn_launch_count(_c.byref(c)))
    return c.value


def sweep_noalloc(model: int, dims, d_spins: int, beta: float, seed: int, stream_id: int, sweep0: int,
                  nsweeps: int, d_trace: int, cuda_stream=None):
    """spn_sweep_noalloc on caller-owned device buffers (raw device pointers as ints)."""
    d = _dims(dims)
    _check(load().spn_sweep_noalloc(model, _ptr(d), d_spins, float(beta), seed, stream_id, sweep0, int(nsweeps),
                                    d_trace, _stream_ptr(cuda_stream)))


class Lattice:
    """One lattice handle (spn_create ... spn_destroy)."""

    def __init__(self, model: int, dims, seed: int, couplings: np.ndarray | None = None, stream_id: int = 0,
                 init: int = SPN_INIT_HOT):
        self._lib = load()
        self.model = model
        self.dims = tuple(int(d) for d in dims)
        self.N = int(np.prod(self.dims))
        d = _dims(dims)
        b = None if couplings is None else np.ascontiguousarray(couplings, dtype=np.uint64)
        h = _vp()
        _check(self._lib.spn_create_ex(_c.byref(h), model, _ptr(d), _ptr(b), seed, stream_id, init))
        self._h = h

    @property
    def handle(self):
        return self._h

    def sweep(self, beta: float, nsweeps: int):
        _check(self._lib.spn_sweep(self._h, float(beta), int(nsweeps)))

    def sweep_dc(self, beta: float, nsweeps: int, tile, hits: int = 1):
        """Double-checkerboard sweeps with `hits`-fold multi-hit (spn_sweep_dc)."""
        t = (_c.c_int32 * 3)(*(list(tile) + [1] * (3 - len(tile))))
        _check(self._lib.spn_sweep_dc(self._h, float(beta), int(nsweeps), t, int(hits)))

    def observables(self) -> tuple[int, int]:
        E, M = _i64(), _i64()
        _check(self._lib.spn_observables(self._h, _c.byref(E), _c.byref(M)))
        return E.value, M.value

    def recompute(self) -> tuple[int, int]:
        E, M = _i64(), _i64()
        _check(self._lib.spn_recompute(self._h, _c.byref(E), _c.byref(M)))
        return E.value, M.value

    def trace(self) -> tuple[np.ndarray, np.ndarray]:
        n = _i64()
        _check(self._lib.spn_trace(self._h, None, None, 0, _c.byref(n)))
        E = np.zeros(n.value, np.int64)
        M = np.zeros(n.value, np.int64)
        _check(self._lib.spn_trace(self._h, _ptr(E), _ptr(M), n.value, _c.byref(n)))
        return E, M

    def get_spins(self, out: np.ndarray | None = None) -> np.ndarray:
        if out is None:
            out = np.empty(self.N, dtype=np.int8)
        if out.dtype != np.int8 or out.size != self.N or not out.flags.c_contiguous:
            raise ValueError("out must be a contiguous int8 array of N elements")
        _check(self._lib.spn_get_spins(self._h, _ptr(out), self.N))
        return out

    def set_spins(self, spins: np.ndarray):
        s = np.ascontiguousarray(spins, dtype=np.int8).reshape(-1)
        _check(self._lib.spn_set_spins(self._h, _ptr(s), s.size))

    def reinit(self, seed: int, stream_id: int = 0, init: int = SPN_INIT_HOT):
        _check(self._lib.spn_reinit(self._h, seed, stream_id, init))

    def sweep_count(self) -> int:
        c = _u64()
        _check(self._lib.spn_sweep_count(self._h, _c.byref(c)))
        return c.value

    def set_stream(self, stream):
        _check(self._lib.spn_set_stream(self._h, _stream_ptr(stream)))

    def sync(self):
        _check(self._lib.spn_sync(self._h))

    def set_tiling(self, tile_y: int, step_slices: int = 0, seg: int = 0):
        _check(self._lib.spn_set_tiling(self._h, tile_y, step_slices, seg))

    def autotune(self, beta: float, trial_sweeps: int = 5) -> tuple[int, int, int]:
        """Time the streaming tilings on a scratch copy and keep the fastest (tile_y, step_slices, seg)."""
        out = np.zeros(3, np.int32)
        _check(self._lib.spn_autotune(self._h, float(beta), int(trial_sweeps), _ptr(out)))
        return tuple(int(x) for x in out)

    @property
    def path(self) -> int:
        p = _i32()
        _check(self._lib.spn_get_path(self._h, _c.byref(p)))
        return p.value

    @path.setter
    def path(self, value: int):
        _check(self._lib.spn_set_path(self._h, int(value)))

    def close(self):
        if getattr(self, "_h", None):
            _check(self._lib.spn_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class HeisLattice:
    """Classical Heisenberg lattice (spn_create_ex with SPN_HEIS2D / SPN_HEIS3D)."""

    def __init__(self, dims, seed: int, stream_id: int = 0, init: int = SPN_INIT_HOT):
        self._lib = load()
        self.dims = tuple(int(d) for d in dims)
        self.N = int(np.prod(self.dims))
        model = SPN_HEIS3D if len(self.dims) == 3 else SPN_HEIS2D
        d = _dims(dims)
        h = _vp()
        _check(self._lib.spn_create_ex(_c.byref(h), model, _ptr(d), None, seed, stream_id, init))
        self._h = h

    def sweep(self, beta: float, nsweeps: int):
        _check(self._lib.spn_sweep(self._h, float(beta), int(nsweeps)))

    def reinit(self, seed: int, stream_id: int = 0, init: int = SPN_INIT_HOT):
        _check(self._lib.spn_reinit(self._h, seed, stream_id, init))

    def get_spins(self) -> np.ndarray:
        out = np.empty((self.N, 3), np.float32)
        _check(self._lib.spn_heis_get_spins(self._h, _ptr(out), out.size))
        return out

    def set_spins(self, S: np.ndarray):
        s = np.ascontiguousarray(S, dtype=np.float32).reshape(-1)
        _check(self._lib.spn_heis_set_spins(self._h, _ptr(s), s.size))

    def observables(self):
        E = _c.c_double()
        M = np.empty(3, np.float64)
        _check(self._lib.spn_heis_observables(self._h, _c.byref(E), _ptr(M)))
        return E.value, M

    def recompute(self):
        E = _c.c_double()
        M = np.empty(3, np.float64)
        _check(self._lib.spn_heis_recompute(self._h, _c.byref(E), _ptr(M)))
        return E.value, M

    def trace(self):
        n = _i64()
        _check(self._lib.spn_heis_trace(self._h, None, None, 0, _c.byref(n)))
        E = np.empty(n.value, np.float64)
        M = np.empty((n.value, 3), np.float64)
        _check(self._lib.spn_heis_trace(self._h, _ptr(E), _ptr(M), n.value, _c.byref(n)))
        return E, M

    def set_stream(self, stream):
        _check(self._lib.spn_set_stream(self._h, _stream_ptr(stream)))

    def sync(self):
        _check(self._lib.spn_sync(self._h))

    def close(self):
        if getattr(self, "_h", None):
            _check(self._lib.spn_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def heis_exp_device(x: np.ndarray) -> np.ndarray:
    """The device binary32 exp of the Heisenberg acceptance (test support)."""
    xs = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty_like(xs)
    _check(load().spn_test_heis_exp(_ptr(xs), _ptr(y), xs.size))
    return y


class EABatch:
    """Multi-spin coded +-J EA samples with replica exchange (spn_create_batch)."""

    def __init__(self, dims, couplings: np.ndarray, betas, seed: int, exchange_every: int = 10,
                 u_per_slot: bool | None = None, disorder_parallel: bool = False):
        """u_per_slot: every temperature slot draws its own u (spn_batch_set_u_per_slot).  None keeps the
        library's default: a u per slot with replica exchange (exchange_every > 0), a shared u without.
        disorder_parallel: the layout of spn_create_batch_dp (samples in the bits of a word)."""
        self._lib = load()
        self.dims = tuple(int(d) for d in dims)
        self.N = int(np.prod(self.dims))
        J = np.ascontiguousarray(couplings, dtype=np.uint64)
        self.nsamples = int(J.shape[0])
        b = np.ascontiguousarray(np.asarray(betas, dtype=np.float64))
        d = _dims(dims)
        h = _vp()
        model = SPN_EA2D_PMJ if len(self.dims) == 2 else SPN_EA3D_PMJ
        create = self._lib.spn_create_batch_dp if disorder_parallel else self._lib.spn_create_batch
        _check(create(_c.byref(h), model, _ptr(d), self.nsamples, _ptr(J), _ptr(b), int(b.size), seed,
                      int(exchange_every)))
        self._h = h
        if u_per_slot is not None:
            _check(self._lib.spn_batch_set_u_per_slot(self._h, 1 if u_per_slot else 0))

    def sweep(self, nsweeps: int):
        _check(self._lib.spn_batch_sweep(self._h, int(nsweeps)))

    def words(self) -> np.ndarray:
        out = np.empty((self.nsamples, self.N), dtype=np.uint32)
        _check(self._lib.spn_batch_get_words(self._h, _ptr(out), out.size))
        return out

    def set_words(self, words: np.ndarray):
        w = np.ascontiguousarray(words, dtype=np.uint32)
        _check(self._lib.spn_batch_set_words(self._h, _ptr(w), w.size))

    def slots(self) -> np.ndarray:
        out = np.empty((self.nsamples, 32), dtype=np.uint8)
        _check(self._lib.spn_batch_get_slots(self._h, _ptr(out), out.size))
        return out

    def set_slots(self, temp_of_slot: np.ndarray):
        t = np.ascontiguousarray(temp_of_slot, dtype=np.uint8)
        _check(self._lib.spn_batch_set_slots(self._h, _ptr(t), t.size))

    def energies(self) -> tuple[np.ndarray, np.ndarray]:
        E = np.empty((self.nsamples, 32), np.int64)
        M = np.empty((self.nsamples, 32), np.int64)
        _check(self._lib.spn_batch_energies(self._h, _ptr(E), _ptr(M), E.size))
        return E, M

    def exchange_counts(self) -> np.ndarray:
        out = np.empty((self.nsamples, 32), np.int64)
        _check(self._lib.spn_batch_exchange_counts(self._h, _ptr(out), out.size))
        return out

    def measure_overlap(self):
        """Enqueue one overlap measurement of the replica pairs (samples 2p, 2p+1)."""
        _check(self._lib.spn_batch_measure_overlap(self._h))

    def overlap(self) -> dict:
        """The overlap measurements so far: nmeas, the last q [pairs, 32], the
        exact integer sums of q^2 and q^4 (Python ints, [pairs][32]), the
        moments <q^2>, <q^4> per pair and temperature, and the Binder cumulant
        per temperature g = (3 - [<q^4>] / [<q^2>]^2) / 2 over the pairs (NaN
        where [<q^2>] = 0: every pair kept q = 0, so g is undefined)."""
        P = self.nsamples // 2
        n = _c.c_int64()
        q = np.empty((P, 32), np.int64)
        q2 = np.empty((P, 32), np.uint64)
        q4 = np.empty((P, 32, 2), np.uint64)
        _check(self._lib.spn_batch_overlap(self._h, _c.byref(n), _ptr(q), _ptr(q2), _ptr(q4), P * 32))
        s2 = [[int(q2[p, t]) for t in range(32)] for p in range(P)]
        s4 = [[int(q4[p, t, 0]) | (int(q4[p, t, 1]) << 64) for t in range(32)] for p in range(P)]
        out = {"nmeas": int(n.value), "q_last": q, "q2_sum": s2, "q4_sum": s4}
        if n.value > 0:
            m2 = np.array([[x / n.value for x in row] for row in s2])
            m4 = np.array([[x / n.value for x in row] for row in s4])
            out["q2"], out["q4"] = m2, m4
            a2, a4 = m2.mean(axis=0), m4.mean(axis=0)
            ratio = np.full_like(a2, np.nan)
            np.divide(a4, a2 ** 2, out=ratio, where=a2 > 0)
            out["binder"] = 0.5 * (3.0 - ratio)
        return out

    def overlap_reset(self):
        _check(self._lib.spn_batch_overlap_reset(self._h))

    def set_stream(self, stream):
        _check(self._lib.spn_set_stream(self._h, _stream_ptr(stream)))

    def sync(self):
        _check(self._lib.spn_sync(self._h))

    def close(self):
        if getattr(self, "_h", None):
            _check(self._lib.spn_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Multi:
    """Batched run of many independent lattices (spn_multi_*)."""

    def __init__(self, jobs):
        """jobs: iterable of (model, dims, beta, nsweeps, seed, stream)."""
        self._lib = load()
        arr = (Job * len(jobs))()
        self.shapes = []
        for k, (model, dims, beta, nsweeps, seed, stream) in enumerate(jobs):
            d = list(dims) + [1] * (3 - len(dims))
            arr[k] = Job(model, (ctypes.c_int32 * 3)(*d), float(beta), int(nsweeps), int(seed), int(stream), 0)
            self.shapes.append((tuple(int(x) for x in dims), int(nsweeps)))
        h = _vp()
        _check(self._lib.spn_multi_create(_c.byref(h), ctypes.cast(arr, _vp), len(jobs)))
        self._h = h

    def run(self, mode: int = SPN_RUN_BATCHED):
        _check(self._lib.spn_multi_run(self._h, mode))

    def sync(self):
        _check(self._lib.spn_multi_sync(self._h))

    def set_stream(self, stream):
        _check(self._lib.spn_multi_set_stream(self._h, _stream_ptr(stream)))

    def result(self, job: int, spins: bool = True, trace: bool = True):
        dims, ns = self.shapes[job]
        N = int(np.prod(dims))
        s = np.empty(N, np.int8) if spins else None
        E = np.empty(ns, np.int64) if trace else None
        M = np.empty(ns, np.int64) if trace else None
        _check(self._lib.spn_multi_result(self._h, job, _ptr(s), N if spins else 0, _ptr(E), _ptr(M),
                                          ns if trace else 0))
        return s, E, M

    def groups(self) -> list[dict]:
        """Launch shape per lattice shape: nd, dims, cluster size, threads, ctas."""
        n = len({(len(d), d) for d, _ in self.shapes})  # the library groups jobs by (dimension, extents)
        out = np.empty(7 * n, np.int32)
        _check(self._lib.spn_multi_groups(self._h, _ptr(out), out.size))
        rows = out.reshape(-1, 7)
        return [{"nd": int(r[0]), "dims": tuple(int(x) for x in r[1:4]), "cs": int(r[4]), "threads": int(r[5]),
                 "ctas": int(r[6])} for r in rows]

    def autotune(self, trial_sweeps: int = 20) -> list[dict]:
        """Time the launch shapes of every lattice shape and keep the fastest."""
        g = self.groups()
        rates = np.zeros(len(g), np.float64)
        _check(self._lib.spn_multi_autotune(self._h, int(trial_sweeps), _ptr(rates), rates.size))
        out = self.groups()
        for d, r in zip(out, rates):
            d["trial_attempts_per_ns"] = float(r)
        return out

    def set_launch(self, group: int, cs: int, threads: int):
        _check(self._lib.spn_multi_set_launch(self._h, int(group), int(cs), int(threads)))

    def close(self):
        if getattr(self, "_h", None):
            _check(self._lib.spn_multi_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request server (spn_server_*)."""

    def __init__(self, hbm_budget_bytes: int):
        self._lib = load()
        h = _vp()
        _check(self._lib.spn_server_create(_c.byref(h), int(hbm_budget_bytes)))
        self._h = h
        self._keep = {}

    def submit(self, model: int, dims, nsweeps: int, seed: int, beta: float = 0.0, stream: int = 0,
               betas=None, couplings=None, exchange_every: int = 10) -> int:
        d = list(dims) + [1] * (3 - len(dims))
        b = None if betas is None else np.ascontiguousarray(np.asarray(betas, dtype=np.float64))
        c = None if couplings is None else np.ascontiguousarray(couplings, dtype=np.uint64)
        r = Request(model, (ctypes.c_int32 * 3)(*d), float(beta), None if b is None else b.ctypes.data,
                    int(nsweeps), int(seed), int(stream), int(exchange_every), None if c is None else c.ctypes.data)
        t = _u64()
        _check(self._lib.spn_submit(self._h, _c.byref(r), _c.byref(t)))
        self._keep[t.value] = (model, tuple(int(x) for x in dims))
        return t.value

    def poll(self, ticket: int):
        done = _c.c_int()
        res = Result()
        _check(self._lib.spn_poll(self._h, ticket, _c.byref(done), _c.byref(res)))
        return bool(done.value), res

    def fetch(self, ticket: int):
        model, dims = self._keep[ticket]
        N = int(np.prod(dims))
        if model == SPN_EA3D_PMJ:
            buf = np.empty(N * 4 + 32, np.uint8)
            _check(self._lib.spn_server_fetch(self._h, ticket, _ptr(buf), buf.size))
            return buf[:N * 4].view(np.uint32).copy(), buf[N * 4:].copy()
        out = np.empty(N, np.int8)
        _check(self._lib.spn_server_fetch(self._h, ticket, _ptr(out), N))
        return out

    def stats(self):
        a, b, r, u = _u64(), _dbl(), _u64(), _sz()
        _check(self._lib.spn_server_stats(self._h, _c.byref(a), _c.byref(b), _c.byref(r), _c.byref(u)))
        return {"attempts": a.value, "busy_s": b.value, "rounds": r.value, "used_bytes": u.value}

    def close(self):
        if getattr(self, "_h", None):
            _check(self._lib.spn_server_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
