"""spn_sweep_noalloc against the oracle and the handle path.

Callers that may not let a library allocate device memory (a framework's
caching allocator owns the device memory, a plugin host only hands out buffers,
a latency-critical loop cannot afford cudaMalloc / cudaFree) use
spn_sweep_noalloc on their own device lattice.  Its only scratch is a static
device array.  These tests check, on two calls in a row, that the lattice and
per-sweep energies equal bit for bit those of the CPU oracle and of a
library-owned handle with the same seed, stream and sweep counters -- on the
streaming path, on shapes the streaming path refuses (2D and 3D), and on a
lattice that starts one byte into a caller's buffer -- and that oversized
lattices are refused.  The file is collected last so that a failure here
leaves every other test already run."""

from __future__ import annotations

import numpy as np
import pytest

from gpu_util import lib, oracle_run
from paper_1006_3865_gb300 import inputs, spn

pytestmark = pytest.mark.gpu


def _two_calls(model, dims, start, beta, seed, sid, offset):
    """Two spn_sweep_noalloc calls (5 then 4 sweeps) on a device copy of `start`
    placed `offset` bytes into a larger caller buffer; returns spins and the
    per-sweep (dE, dM) rows."""
    torch = pytest.importorskip("torch")
    N = start.size
    buf = torch.zeros(N + 64, dtype=torch.int8, device="cuda")
    d_s = buf[offset:offset + N]
    d_s.copy_(torch.from_numpy(start).cuda())
    d_t1 = torch.zeros(2 * 5, dtype=torch.int64, device="cuda")
    d_t2 = torch.zeros(2 * 4, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    assert d_s.data_ptr() % 16 == offset % 16
    spn.sweep_noalloc(model, dims, d_s.data_ptr(), beta, seed, sid, 0, 5, d_t1.data_ptr())
    spn.sweep_noalloc(model, dims, d_s.data_ptr(), beta, seed, sid, 5, 4, d_t2.data_ptr())
    torch.cuda.synchronize()
    out = buf.cpu().numpy()
    # the bytes around the lattice are untouched
    assert not out[:offset].any() and not out[offset + N:].any()
    deltas = np.concatenate([d_t1.cpu().numpy(), d_t2.cpu().numpy()]).reshape(-1, 2)
    return out[offset:offset + N].copy(), deltas


@pytest.mark.parametrize("offset", [0, 1])
@pytest.mark.parametrize("model,dims", [(spn.SPN_ISING2D, (256, 128)), (spn.SPN_ISING3D, (64, 32, 16)),
                                        (spn.SPN_ISING2D, (34, 18)), (spn.SPN_ISING3D, (34, 18, 10))])
def test_noalloc_matches_oracle_and_handle_path_on_two_calls(model, dims, offset):
    lib()
    seed, sid, beta = inputs.unit_seed(77), 3, 0.4
    lat = spn.Lattice(model, dims, seed, stream_id=sid)
    start = lat.get_spins().copy()
    E0, M0 = lat.observables()
    lat.sweep(beta, 5)
    lat.sweep(beta, 4)
    ref_s = lat.get_spins().copy()
    ref_E, ref_M = lat.trace()
    lat.close()
    orc_s, orc_E, orc_M = oracle_run(dims, seed, [(beta, 5), (beta, 4)], stream=sid)

    s, deltas = _two_calls(model, dims, start, beta, seed, sid, offset)
    E = E0 + np.cumsum(deltas[:, 0])
    M = M0 + np.cumsum(deltas[:, 1])
    assert np.array_equal(s, orc_s) and np.array_equal(E, orc_E) and np.array_equal(M, orc_M)
    assert np.array_equal(s, ref_s) and np.array_equal(E, ref_E) and np.array_equal(M, ref_M)


def test_noalloc_refuses_lattices_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    lib()
    d_s = torch.ones(8, dtype=torch.int8, device="cuda")
    d_t = torch.zeros(2, dtype=torch.int64, device="cuda")
    with pytest.raises(spn.SpnError) as e:
        spn.sweep_noalloc(spn.SPN_ISING2D, (8192, 4096), d_s.data_ptr(), 0.4, 1, 0, 0, 1, d_t.data_ptr())
    assert e.value.code == spn.SPN_E_ARG and "static scratch" in str(e.value)
