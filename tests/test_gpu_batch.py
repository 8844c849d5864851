"""Batched problems against the oracle and against single handles (needs a B300)."""
import math

import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2607_24059_b300 as v  # noqa: E402

# uneven sizes (n_x a multiple of 4), viscosities and resolutions
PROBLEMS = [
    dict(n=(64, 64), nu=0.01, seed=1),
    dict(n=(32, 48), nu=0.003, seed=2),
    dict(n=(128, 16), nu=0.0005, seed=3),
    dict(n=(8, 40), nu=0.02, seed=4),
    dict(n=(96, 96), nu=0.001, seed=5),
]
# fp64/fp32: max-abs error relative to max|u|; 16-bit storage: the L2 velocity gate of the
# reduced-precision and batched forms (relative L2 error <= 1e-3 against the oracle)
# (the shifted 16-bit forms do not hold the L2 gate on slowly evolving flows; they are tied to
# the single-handle kernels below, which are checked node by node against the oracle)
TOL = {"fp64": 1e-12, "fp32": 1e-5, "fp16split": 1e-3, "bf16split": 1e-3}


def l2_rel(a, b):
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))


def problem_inputs(q):
    """Seeded smooth field on a (nx, ny) lattice with dx = 2 pi / nx."""
    nx, ny = q["n"]
    dx = 2 * math.pi / nx
    rng = np.random.default_rng(q["seed"])
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dx
    X, Y = np.meshgrid(x, y, indexing="xy")
    ky = 2 * math.pi / (ny * dx)
    u = np.stack([0.3 * np.sin(X + rng.uniform()) * np.cos(ky * Y), -0.2 * np.cos(X) * np.sin(ky * Y + rng.uniform())])
    phi = 0.3 * np.cos(X + ky * Y)
    return u, phi, dx


def batch_and_oracle(precision, steps):
    qs = [dict(n=q["n"], dx=problem_inputs(q)[2], nu=q["nu"]) for q in PROBLEMS]
    b = v.Batch(qs, precision=precision)
    orc = oracle.default()
    refs = []
    for i, q in enumerate(PROBLEMS):
        u, phi, dx = problem_inputs(q)
        b.init(i, torch.from_numpy(u).cuda(), torch.from_numpy(phi).cuda())
        op = oracle.make_params(q["n"], dx, nu=q["nu"])
        _, uo, _ = orc.macros(op, orc.run(op, orc.init(op, u, phi), steps))
        refs.append(uo)
    return b, refs


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16split", "bf16split"])
def test_batch_matches_oracle_per_problem(precision):
    steps = 70          # crosses a graph replay (32 steps) and single launches
    b, refs = batch_and_oracle(precision, steps)
    b.step(steps)
    for i, uo in enumerate(refs):
        ug = b.velocity(i).cpu().numpy()
        if precision in ("fp64", "fp32"):
            err = np.max(np.abs(ug - uo)) / np.max(np.abs(uo))
        else:
            err = l2_rel(ug, uo)
        assert err <= TOL[precision], (i, err)
    n_total, s, launches = b.info()
    assert s == steps and n_total == sum(q["n"][0] * q["n"][1] for q in PROBLEMS)
    b.close()


@pytest.mark.parametrize("precision,lanes", [("fp32", 4), ("fp16split", 4), ("fp16", 4), ("bf16", 4),
                                           ("fp16", 2), ("bf16", 2)])
def test_batch_equals_single_handles(precision, lanes):
    """lanes: nodes per lane of the batched kernel (the single-lattice 16-bit kernels take 4)."""
    qs = [dict(n=q["n"], dx=problem_inputs(q)[2], nu=q["nu"]) for q in PROBLEMS]
    b = v.Batch(qs, precision=precision)
    b.set_config(256, 2, lanes)
    singles = []
    for i, q in enumerate(PROBLEMS):
        u, phi, dx = problem_inputs(q)
        b.init(i, torch.from_numpy(u).cuda(), torch.from_numpy(phi).cuda())
        lat = v.Lattice(q["n"], dx, nu=q["nu"], precision=precision)
        lat.init(torch.from_numpy(u).cuda(), torch.from_numpy(phi).cuda())
        lat.step(40)
        singles.append(lat.macros()[1].cpu().numpy())
        lat.close()
    b.step(40)
    # same arithmetic and the same stochastic-rounding words (nodes are numbered within
    # their problem, one step counter), inlined into a different kernel: FMA contraction may
    # differ, and for 16-bit storage a flipped rounding then moves a stored value by one
    # quantum (2^-11 FP16, 2^-8 BF16)
    tol = {"fp32": 1e-6, "fp16split": 1e-4, "fp16": 2e-3, "bf16": 1.6e-2}[precision]
    for i, us in enumerate(singles):
        ub = b.velocity(i).cpu().numpy()
        assert np.max(np.abs(ub - us)) <= tol * np.max(np.abs(us)), i
    b.close()


@pytest.mark.parametrize("precision", ["fp32", "fp16split"])
def test_autotune_keeps_state_and_results(precision):
    qs = [dict(n=q["n"], dx=problem_inputs(q)[2], nu=q["nu"]) for q in PROBLEMS]
    out = []
    for tune in (False, True):
        b = v.Batch(qs, precision=precision)
        for i, q in enumerate(PROBLEMS):
            u, phi, _ = problem_inputs(q)
            b.init(i, torch.from_numpy(u).cuda(), torch.from_numpy(phi).cuda())
        b.step(5)
        if tune:
            cfg, ms = b.autotune(repeats=2)
            assert cfg[0] in (128, 256) and 1 <= cfg[1] <= 16 and ms > 0
        b.step(45)
        out.append([b.velocity(i).cpu().numpy() for i in range(len(PROBLEMS))])
        assert b.info()[1] == 50
        b.close()
    for a, c in zip(*out):
        assert np.max(np.abs(a - c)) <= 1e-5 * np.max(np.abs(c))


def test_batch_graph_replay_equals_launches():
    qs = [dict(n=q["n"], dx=problem_inputs(q)[2], nu=q["nu"]) for q in PROBLEMS]
    out = []
    for graph in (True, False):
        b = v.Batch(qs, precision="fp32")
        for i, q in enumerate(PROBLEMS):
            u, phi, _ = problem_inputs(q)
            b.init(i, torch.from_numpy(u).cuda(), torch.from_numpy(phi).cuda())
        b.step(67, graph=graph)
        out.append([b.velocity(i).cpu().numpy() for i in range(len(PROBLEMS))])
        b.close()
    for a, c in zip(*out):
        assert np.array_equal(a, c)


def test_batch_invariants_match_oracle():
    b, _ = batch_and_oracle("fp64", 0)
    orc = oracle.default()
    b.step(20)
    for i, q in enumerate(PROBLEMS):
        u, phi, dx = problem_inputs(q)
        op = oracle.make_params(q["n"], dx, nu=q["nu"])
        inv_o = orc.invariants(op, orc.run(op, orc.init(op, u, phi), 20))
        inv_g = b.invariants(i)
        assert abs(inv_g[4] - inv_o[4]) <= 1e-12 * inv_o[4]
        assert np.allclose(inv_g[1:3], inv_o[1:3], rtol=1e-10, atol=1e-10)
    b.close()


def test_batch_rejects_bad_problems():
    with pytest.raises(v.VlbmError):
        v.Batch([dict(n=(32, 16), dx=0.1, nu=0.01), dict(n=(0, 16), dx=0.1, nu=0.01)])   # empty lattice
    with pytest.raises(v.VlbmError):
        v.Batch([dict(n=(32, 16), dx=0.1, nu=0.01, omega_q=2.5)])                         # omega outside (0, 2)


_MEMBER_REFS = {}


@pytest.mark.parametrize("precision", ["fp16split", "bf16split", "fp32"])
def test_batched_problem_set_members_match_oracle(orc, precision):
    """Problems drawn from the batched workload's own set (sides 512 and 1024, seeded random
    Fourier fields, their own viscosities), advanced together 200 steps in the batched 16-bit
    split storage the benchmark uses (and FP32), each against the oracle at the L2 gate of 1e-3.
    (The shifted 16-bit forms miss that gate on these flows: 4e-3 to 1.3e-2 after 200 steps.)"""
    chosen = [q for q in synthetic.batched_problem_set(512) if q.side >= 512][:8]
    assert len(chosen) == 8
    specs, inputs = [], []
    for q in chosen:
        u, phi, dx = synthetic.random_fourier_field(q.side, q.seed)
        specs.append(dict(n=(q.side, q.side), dx=dx, nu=q.nu))
        inputs.append((u, phi, dx))
    b = v.Batch(specs, precision=precision)
    for i, (u, phi, _) in enumerate(inputs):
        b.init(i, torch.from_numpy(u).cuda(), torch.from_numpy(phi).cuda())
    steps = 200
    b.step(steps)
    for i, (q, (u, phi, dx)) in enumerate(zip(chosen, inputs)):
        key = (q.index, steps)
        if key not in _MEMBER_REFS:     # the oracle's velocity, shared by the storage forms
            op = oracle.make_params((q.side, q.side), dx, nu=q.nu)
            _MEMBER_REFS[key] = orc.macros(op, orc.run(op, orc.init(op, u, phi), steps))[1]
        uo = _MEMBER_REFS[key]
        assert np.isfinite(uo).all(), q
        ug = b.velocity(i).cpu().numpy()
        err = l2_rel(ug, uo)
        print(f"{precision} problem {q.index}: side {q.side}, nu {q.nu:.2e}: L2 {err:.2e}")
        assert err <= 1e-3, (q, err)
        if precision == "fp32":     # the FP32 gate: max-abs error <= 1e-5 of max|u|
            assert np.max(np.abs(ug - uo)) <= 1e-5 * np.max(np.abs(uo)), q
    b.close()


def batch_of_problems(precision):
    qs = [dict(n=q["n"], dx=problem_inputs(q)[2], nu=q["nu"]) for q in PROBLEMS]
    b = v.Batch(qs, precision=precision)
    for i, q in enumerate(PROBLEMS):
        u, phi, _ = problem_inputs(q)
        b.init(i, torch.from_numpy(u).cuda(), torch.from_numpy(phi).cuda())
    return b


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16", "bf16", "fp16split", "bf16split"])
def test_persistent_launch_matches_per_step_launches(precision):
    """VLBM_STEP_PERSISTENT runs the steps in one cooperative launch whose blocks wait for each
    other at step boundaries; it advances every problem as per-step launches do (odd and even
    step counts, so the levels end on either parity, and a per-step launch after it)."""
    out = []
    for persistent in (False, True):
        b = batch_of_problems(precision)
        b.set_config(128, 4, 4)
        b.step(7, graph=False, persistent=persistent)
        b.step(10, graph=False, persistent=persistent)
        b.step(1, graph=False)
        out.append([b.velocity(i).cpu().numpy() for i in range(len(PROBLEMS))])
        assert b.info()[1] == 18
        b.close()
    # the two launch forms instantiate the same per-node arithmetic with different loads; the
    # compiler may still contract a multiply-add pair differently in the two kernels
    rel = {"fp64": 1e-13, "fp32": 1e-6}.get(precision, 2e-3 if "fp16" in precision else 1.6e-2)
    for a, c in zip(*out):
        assert np.max(np.abs(a - c)) <= rel * np.max(np.abs(c)), np.max(np.abs(a - c)) / np.max(np.abs(c))


def test_persistent_launch_timeout_path_reports_and_recovers():
    """The test flag makes the first step boundary wait for a block that does not exist: every
    block gives up after its bounded wait (about one second), the call reports VLBM_ETIMEOUT,
    and the batch steps normally afterwards."""
    b = batch_of_problems("fp32")
    with pytest.raises(v.VlbmError) as e:
        v.vlbm_batch_step(b.handle, 2, v.VLBM_STEP_PERSISTENT | v.VLBM_STEP_TEST_TIMEOUT)
    assert e.value.code == v.VLBM_ETIMEOUT
    b.step(3, graph=False)
    b.step(2, graph=False, persistent=True)
    for i in range(len(PROBLEMS)):
        assert np.all(np.isfinite(b.velocity(i).cpu().numpy()))
    b.close()


# widths that are not multiples of the nodes per lane (4 for FP32, 2 for FP64, 4 or 2 for the
# split and shifted 16-bit formats): those problems run the per-node body, one node per lane
RAGGED = [
    dict(n=(37, 23), nu=0.01, seed=11),
    dict(n=(50, 30), nu=0.004, seed=12),
    dict(n=(36, 20), nu=0.002, seed=13),
    dict(n=(64, 16), nu=0.006, seed=14),
    dict(n=(13, 11), nu=0.01, seed=15),
]


@pytest.mark.parametrize("persistent", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16split", "bf16split"])
def test_ragged_widths_match_oracle_per_problem(precision, persistent):
    qs = [dict(n=q["n"], dx=problem_inputs(q)[2], nu=q["nu"]) for q in RAGGED]
    b = v.Batch(qs, precision=precision)
    orc = oracle.default()
    steps = 37
    refs = []
    for i, q in enumerate(RAGGED):
        u, phi, dx = problem_inputs(q)
        b.init(i, torch.from_numpy(u).cuda(), torch.from_numpy(phi).cuda())
        op = oracle.make_params(q["n"], dx, nu=q["nu"])
        refs.append(orc.macros(op, orc.run(op, orc.init(op, u, phi), steps))[1])
    b.step(steps, graph=False, persistent=persistent)
    for i, uo in enumerate(refs):
        ug = b.velocity(i).cpu().numpy()
        err = np.max(np.abs(ug - uo)) / np.max(np.abs(uo)) if precision in ("fp64", "fp32") else l2_rel(ug, uo)
        assert err <= TOL[precision], (RAGGED[i]["n"], err)
    b.close()


@pytest.mark.parametrize("lanes", [4, 2])
@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_ragged_widths_shifted_equal_single_handles(precision, lanes):
    qs = [dict(n=q["n"], dx=problem_inputs(q)[2], nu=q["nu"]) for q in RAGGED]
    b = v.Batch(qs, precision=precision)
    b.set_config(256, 2, lanes)
    singles = []
    for i, q in enumerate(RAGGED):
        u, phi, dx = problem_inputs(q)
        b.init(i, torch.from_numpy(u).cuda(), torch.from_numpy(phi).cuda())
        lat = v.Lattice(q["n"], dx, nu=q["nu"], precision=precision)
        lat.init(torch.from_numpy(u).cuda(), torch.from_numpy(phi).cuda())
        lat.step(25)
        singles.append(lat.macros()[1].cpu().numpy())
        lat.close()
    b.step(25)
    tol = {"fp16": 2e-3, "bf16": 1.6e-2}[precision]
    for i, us in enumerate(singles):
        ub = b.velocity(i).cpu().numpy()
        assert np.max(np.abs(ub - us)) <= tol * np.max(np.abs(us)), RAGGED[i]["n"]
    b.close()

