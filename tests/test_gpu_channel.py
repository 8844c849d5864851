"""Channel boundaries (ghost cells of Section 6.2.1) on the GPU against the oracle and Table 2."""
import numpy as np
import pytest

import oracle
from oracle.poiseuille import Poiseuille, exact

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2607_24059_b300 as v  # noqa: E402

TABLE2_75 = {  # Table 2, 75 cells per direction: (omega_q, corrected) -> printed L2 error on u_x
    (1.0, False): 2.938e-05, (1.15, False): 5.661e-04, (1.0, True): 2.943e-05, (1.15, True): 1.485e-05,
}


def channel_lattice(sim: Poiseuille, precision):
    """A GPU lattice with the oracle simulation's parameters, initial state and boundaries."""
    op = sim.p
    lat = v.Lattice(op.n, op.dx, nu=0.0, precision=precision, mu=op.mu, omega_rho=op.omega[0],
                    alpha_rho=op.alpha[0], omega_q=op.omega[1], alpha_q=op.alpha[1])
    u, phi, _, _ = exact(sim.n, nx=sim.nx)
    lat.init(torch.from_numpy(u).cuda(), torch.from_numpy(phi).cuda())
    lat.set_channel(u[0][:, 0], phi_out=0.0, wall_correction=sim.corrected)
    return lat


def l2_error_ux(u, sim):
    return float(np.sqrt(sim.dx ** 2 * np.sum((u[0] - sim.u_ex[0]) ** 2)))


@pytest.mark.parametrize("corrected", [False, True])
@pytest.mark.parametrize("omega_q", [1.0, 1.15])
@pytest.mark.parametrize("shape", [(20, 20), (12, 33)])
def test_channel_fp64_matches_oracle(orc, shape, omega_q, corrected):
    """FP64 storage, every velocity against the oracle's Poiseuille simulation after 300 steps
    (a square and a channel longer than wide, n_x not a multiple of the vector width)."""
    n, nx = shape
    sim = Poiseuille(orc, n, omega_q, corrected=corrected, nx=nx)
    lat = channel_lattice(sim, "fp64")
    lat.step(300)
    sim.step(300)
    _, ug, _ = lat.macros()
    _, uo, _ = orc.macros(sim.p, sim.f)
    lat.close()
    assert np.max(np.abs(ug.cpu().numpy() - uo)) <= 1e-12 * np.max(np.abs(uo))


@pytest.mark.parametrize("corrected", [False, True])
@pytest.mark.parametrize("omega_q", [1.0, 1.15])
def test_channel_reproduces_table2_at_75_cells(orc, omega_q, corrected):
    """The GPU in FP64 reproduces the 75-cell row of Table 2 to within one unit of its fourth
    printed digit (2250 steps to t = 0.05); FP32 storage agrees with FP64 storage to 1e-5 of
    max|u| and gives the same printed digits to within a few units."""
    sim = Poiseuille(orc, 75, omega_q, corrected=corrected)
    ref = TABLE2_75[(omega_q, corrected)]
    unit = 10.0 ** (np.floor(np.log10(ref)) - 3)
    out = {}
    for precision in ("fp64", "fp32"):
        lat = channel_lattice(sim, precision)
        lat.step(2250)
        out[precision] = lat.macros()[1].cpu().numpy()
        lat.close()
    e64 = l2_error_ux(out["fp64"], sim)
    e32 = l2_error_ux(out["fp32"], sim)
    print(f"omega_q {omega_q} corrected {corrected}: FP64 {e64:.5e}, FP32 {e32:.5e}, printed {ref:.3e}")
    assert abs(e64 - ref) <= unit, (e64, ref)
    assert np.max(np.abs(out["fp32"] - out["fp64"])) <= 1e-5 * np.max(np.abs(out["fp64"]))
    assert abs(e32 - ref) <= 5 * unit, (e32, ref)


def test_channel_graph_replay_and_launch_count(orc):
    """Graph replay of channel steps equals step-by-step launches bit for bit; a channel step is
    two launches (ghost populations, stream-collide)."""
    sim = Poiseuille(orc, 24, 1.15, corrected=True, nx=40)
    out = []
    for graph in (True, False):
        lat = channel_lattice(sim, "fp32")
        c0 = lat.launch_count()
        lat.step(130, graph=graph)
        assert lat.launch_count() - c0 == 260
        out.append(lat.populations(deviation=True).cpu().numpy())
        lat.close()
    assert np.array_equal(out[0], out[1])


def test_channel_back_to_periodic_and_rejections(orc):
    """Setting periodic boundaries again gives the periodic step; channels are refused for 3D,
    for 16-bit storage, and by vlbm_step_record."""
    n = 16
    u = np.zeros((2, n, n))
    u[0] = 0.1 * np.sin(2 * np.pi * (np.arange(n) + 0.5) / n)[:, None]
    phi = np.zeros((n, n))
    op = oracle.make_params((n, n), 2 * np.pi / n, nu=0.01)
    lat = v.Lattice(op.n, op.dx, nu=0.0, precision="fp64", mu=op.mu, omega_rho=op.omega[0], alpha_rho=op.alpha[0],
                    omega_q=op.omega[1], alpha_q=op.alpha[1])
    lat.init(torch.from_numpy(u).cuda(), torch.from_numpy(phi).cuda())
    lat.set_channel(np.zeros(n))
    with pytest.raises(v.VlbmError):
        lat.step_record(2, 1)
    lat.set_periodic()
    lat.step(20)
    _, ug, _ = lat.macros()
    lat.close()
    _, uo, _ = orc.macros(op, orc.run(op, orc.init(op, u, phi), 20))
    assert np.max(np.abs(ug.cpu().numpy() - uo)) <= 1e-12 * np.max(np.abs(uo))
    for shape, precision in (((8, 8), "fp16"), ((8, 8), "fp16split"), ((8, 8, 8), "fp64")):
        lat = v.Lattice(shape, 0.1, nu=0.01, precision=precision)
        with pytest.raises(v.VlbmError):
            lat.set_channel(np.zeros(8))
        lat.close()
