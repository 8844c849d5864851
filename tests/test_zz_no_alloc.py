"""vlbm_invariants_noalloc: the invariant reduction for callers that cannot allocate.

Some callers may not call cudaMalloc -- code living inside a memory pool that
owns all device memory, or a real-time loop that must not take the allocator's
locks or its implicit synchronisation.  They hold the population lattice in
their own device memory and call this entry point, which keeps its partial
sums in a static device array instead of allocating.  These tests hand it a
lattice taken from a handle's checkpoint and compare its result with the
handle's own vlbm_invariants, slot by slot, on two calls in a row (device
result, then host result), so that the second call must not be disturbed by
what the first left in the shared static array.  Every storage format is
covered (the 16-bit ones depend on the entry point reproducing the handle's
storage scales), in 2D and 3D, and one lattice large enough for the two-stage
fold of the partial rows.  Collected last, so that a run stopping at the first
failure has already run every other test; it also passes on its own.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2607_24059_b300 as v  # noqa: E402
import synthetic  # noqa: E402

# Both sides reduce the same stored values with the same per-node arithmetic; only the
# grouping of the partial sums differs (float-pair and FP64 sums), so every slot agrees to
# far below these bounds.  A wrong storage scale would be off by orders of magnitude.
TOL = {"fp64": 1e-12, "fp32": 1e-9, "fp16": 1e-9, "bf16": 1e-9, "fp16split": 1e-9, "bf16split": 1e-9}


def caller_owned_lattice(lat):
    """Copy of the handle's population lattice in caller-owned device memory."""
    blob = torch.empty(v.vlbm_state_bytes(lat.handle), dtype=torch.uint8, device="cuda")
    v.vlbm_get_state(lat.handle, blob)
    header = blob.numel() - lat.derived.lattice_bytes
    return blob[header:].clone()


def assert_slots_match(got, ref, tol, nodes, dx, dim, umax, phimax):
    """Slot-wise comparison, each slot against its own scale:
    0 N rho_bar + sum(rho - rho_bar), 1..3 momentum totals, 4 kinetic energy, 5 max|u|,
    6 non-finite nodes, 7 sum(rho - rho_bar)."""
    scale = [
        abs(ref[0]),
        nodes * umax, nodes * umax, nodes * umax,          # sums of |q| bound the totals
        abs(ref[4]),
        abs(ref[5]),
        0.0,
        nodes * dx * dx * phimax,                           # sum of |rho - rho_bar| ~ N dx^2 |phi|
    ]
    for i in range(8):
        if i == 3 and dim == 2:
            assert got[3] == 0.0 and ref[3] == 0.0
            continue
        if i == 6:
            assert got[6] == ref[6] == 0.0
            continue
        assert abs(got[i] - ref[i]) <= tol * scale[i], (i, got[i], ref[i])


def state_2d(n):
    u, phi, dx = synthetic.taylor_green_2d(n)
    return u + 0.05, phi, dx                        # nonzero net momentum


def state_3d(n):
    u, phi, dx = synthetic.taylor_green_3d(n)
    u = u.copy()
    u[2] += 0.03
    return u, phi, dx


def check_two_calls(lat, u, phi, dx, tol):
    nodes = int(np.prod(lat.n))
    umax = float(np.max(np.abs(u))) * 1.1
    phimax = float(np.max(np.abs(phi))) + 1.0
    lat.init(torch.from_numpy(u).cuda(), torch.from_numpy(phi).cuda())
    lat.step(25)

    # call 1: result in device memory
    lattice = caller_owned_lattice(lat)
    out_dev = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
    v.vlbm_invariants_noalloc(lat.params, lattice, out_dev)
    ref1 = lat.invariants()
    got1 = out_dev.cpu().numpy()
    assert_slots_match(got1, ref1, tol, nodes, dx, lat.dim, umax, phimax)

    # call 2, right after, on a later state: result in host memory
    lat.step(40)
    lattice = caller_owned_lattice(lat)
    out_host = np.full(8, np.nan)
    v.vlbm_invariants_noalloc(lat.params, lattice, out_host)
    ref2 = lat.invariants()
    assert_slots_match(out_host, ref2, tol, nodes, dx, lat.dim, umax, phimax)
    assert not np.allclose(out_host[4], got1[4], rtol=1e-9)     # the state did change


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16", "bf16", "fp16split", "bf16split"])
def test_noalloc_invariants_match_vlbm_invariants(precision):
    u, phi, dx = state_2d(96)
    lat = v.Lattice((96, 96), dx, nu=0.01, precision=precision)
    check_two_calls(lat, u, phi, dx, TOL[precision])
    lat.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16split"])
def test_noalloc_invariants_3d(precision):
    u, phi, dx = state_3d(16)
    lat = v.Lattice((16, 16, 16), dx, nu=0.01, precision=precision)
    check_two_calls(lat, u, phi, dx, TOL[precision])
    lat.close()


def test_noalloc_invariants_two_stage_fold():
    """2048^2 nodes = 512 partial rows: folded by the first stage before the final pass."""
    u, phi, dx = state_2d(2048)
    lat = v.Lattice((2048, 2048), dx, nu=1e-3, precision="fp32")
    check_two_calls(lat, u, phi, dx, TOL["fp32"])
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
