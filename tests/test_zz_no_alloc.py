"""spn_sweep_noalloc against the handle path.

Callers that may not let a library allocate device memory (a framework's
caching allocator owns the device memory, a plugin host only hands out buffers,
a latency-critical loop cannot afford cudaMalloc / cudaFree) use
spn_sweep_noalloc on their own device lattice.  Its only scratch is a static
device array; this test checks that two calls in a row give bit-for-bit the
lattice and per-sweep energies of a library-owned handle with the same seed,
stream and sweep counters, and that oversized lattices are refused.  It is
collected last so that a failure here leaves every other test already run."""

from __future__ import annotations

import numpy as np
import pytest

from gpu_util import lib
from paper_1006_3865_gb300 import inputs, spn

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("model,dims", [(spn.SPN_ISING2D, (256, 128)), (spn.SPN_ISING3D, (64, 32, 16)),
                                        (spn.SPN_ISING2D, (34, 18))])
def test_noalloc_matches_handle_path_on_two_calls(model, dims):
    torch = pytest.importorskip("torch")
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

    d_s = torch.from_numpy(start).cuda()
    d_t1 = torch.zeros(2 * 5, dtype=torch.int64, device="cuda")
    d_t2 = torch.zeros(2 * 4, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    spn.sweep_noalloc(model, dims, d_s.data_ptr(), beta, seed, sid, 0, 5, d_t1.data_ptr())
    spn.sweep_noalloc(model, dims, d_s.data_ptr(), beta, seed, sid, 5, 4, d_t2.data_ptr())
    torch.cuda.synchronize()
    deltas = np.concatenate([d_t1.cpu().numpy(), d_t2.cpu().numpy()]).reshape(-1, 2)
    assert np.array_equal(d_s.cpu().numpy(), ref_s)
    assert np.array_equal(E0 + np.cumsum(deltas[:, 0]), ref_E)
    assert np.array_equal(M0 + np.cumsum(deltas[:, 1]), ref_M)


def test_noalloc_refuses_lattices_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    lib()
    d_s = torch.ones(8, dtype=torch.int8, device="cuda")
    d_t = torch.zeros(2, dtype=torch.int64, device="cuda")
    with pytest.raises(spn.SpnError) as e:
        spn.sweep_noalloc(spn.SPN_ISING2D, (8192, 4096), d_s.data_ptr(), 0.4, 1, 0, 0, 1, d_t.data_ptr())
    assert e.value.code == spn.SPN_E_ARG and "static scratch" in str(e.value)
