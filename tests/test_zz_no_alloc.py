"""vlbm_invariants_noalloc: the invariant reduction for callers that cannot allocate.

Some callers may not call cudaMalloc -- code living inside a memory pool that
owns all device memory, or a real-time loop that must not take the allocator's
locks or its implicit synchronisation.  They hold the population lattice in
their own device memory and call this entry point, which keeps its partial
sums in a static device array instead of allocating.  This test hands it a
lattice taken from a handle's checkpoint and compares its result with the
handle's own vlbm_invariants, on two calls in a row (device result, then host
result), so that the second call must not be disturbed by what the first left
in the shared static array.  Collected last, so that a run stopping at the
first failure has already run every other test; it also passes on its own.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2607_24059_b300 as v  # noqa: E402
import synthetic  # noqa: E402

TOL = {"fp64": 1e-12, "fp32": 1e-6}     # the tolerances of the other invariant tests


def caller_owned_lattice(lat):
    """Copy of the handle's population lattice in caller-owned device memory."""
    blob = torch.empty(v.vlbm_state_bytes(lat.handle), dtype=torch.uint8, device="cuda")
    v.vlbm_get_state(lat.handle, blob)
    header = blob.numel() - lat.derived.lattice_bytes
    return blob[header:].clone()


def close(a, b, tol):
    scale = np.max(np.abs(b))
    return np.allclose(a, b, rtol=tol, atol=tol * scale)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_invariants_match_vlbm_invariants(precision):
    u, phi, dx = synthetic.taylor_green_2d(96)
    u = u + 0.05
    lat = v.Lattice((96, 96), dx, nu=0.01, precision=precision)
    lat.init(torch.from_numpy(u).cuda(), torch.from_numpy(phi).cuda())
    lat.step(25)

    # call 1: result in device memory
    lattice = caller_owned_lattice(lat)
    out_dev = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
    v.vlbm_invariants_noalloc(lat.params, lattice, out_dev)
    ref1 = lat.invariants()
    got1 = out_dev.cpu().numpy()
    assert close(got1, ref1, TOL[precision]), (got1, ref1)

    # call 2, right after, on a later state: result in host memory
    lat.step(40)
    lattice = caller_owned_lattice(lat)
    out_host = np.full(8, np.nan)
    v.vlbm_invariants_noalloc(lat.params, lattice, out_host)
    ref2 = lat.invariants()
    assert close(out_host, ref2, TOL[precision]), (out_host, ref2)
    assert not np.allclose(out_host[4], got1[4], rtol=1e-9)     # the state did change
    lat.close()


def test_noalloc_rejects_oversized_lattice_and_host_lattice():
    p = v.vlbm_params_default(2, (8192, 8193), 1e-3, 1e-4, v.VLBM_FP32)
    small = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = np.zeros(8)
    with pytest.raises(v.VlbmError) as e:
        v.vlbm_invariants_noalloc(p, small, out)       # 8192 x 8193 nodes: above the limit
    assert e.value.code == v.VLBM_EINVAL
    p = v.vlbm_params_default(2, (4, 4), 0.1, 1e-2, v.VLBM_FP32)
    host = np.zeros(4 * 4 * 15, dtype=np.float32)
    with pytest.raises(v.VlbmError):
        v.vlbm_invariants_noalloc(p, host.ctypes.data, out)   # lattice must be device memory
