"""Planted mistakes in a copy of the oracle must each fail at least one pin.

Each mutation below is a plausible slip (a dropped term, a wrong sign, a wrong
index or operand) applied to a temporary copy of oracle/vlbm_oracle.c; the
committed source is never touched.  The copy is compiled on the CPU and run
through the fast pins of oracle_pins.py.
"""
import os
import shutil
import subprocess

import pytest

import oracle
from oracle import build as obuild
import oracle_pins as P

SRC = os.path.join(os.path.dirname(oracle.__file__), "vlbm_oracle.c")

MUTATIONS = {
    "rest_q_without_dx": ("fx[0] = dx * (1.0 - 4.0 * ax) * qx;", "fx[0] = (1.0 - 4.0 * ax) * qx;"),
    "pressure_sign": ("fx[1] = dx * ax * qx + dx * dx / (2.0 * mu) * qx * qx / rho + P / (2.0 * mu);",
                      "fx[1] = dx * ax * qx + dx * dx / (2.0 * mu) * qx * qx / rho - P / (2.0 * mu);"),
    "advection_dropped": ("fx[1] = dx * ax * qx + dx * dx / (2.0 * mu) * qx * qx / rho + P / (2.0 * mu);",
                          "fx[1] = dx * ax * qx + P / (2.0 * mu);"),
    "advection_operand": ("fy[3] = dx * ay * qy + dx * dx / (2.0 * mu) * qy * qy / rho + P / (2.0 * mu);",
                          "fy[3] = dx * ay * qy + dx * dx / (2.0 * mu) * qx * qy / rho + P / (2.0 * mu);"),
    "mass_flux_sign": ("fr[1] = ar * rho + dx / (2.0 * mu) * qx;", "fr[1] = ar * rho - dx / (2.0 * mu) * qx;"),
    "rest_weight": ("fr[0] = (1.0 - 4.0 * ar) * rho;", "fr[0] = (1.0 - 3.0 * ar) * rho;"),
    "alpha_of_wrong_field": ("fy[0] = dx * (1.0 - 4.0 * ay) * qy;", "fy[0] = dx * (1.0 - 4.0 * ax) * qy;"),
    "stream_direction": ("case 1: sx = (x - 1 + nx) % nx; break;", "case 1: sx = (x + 1) % nx; break;"),
    "stream_missing_axis": ("case 4: sy = (y + 1) % ny; break;", "case 4: sy = y; break;"),
    "omega_of_wrong_field": ("out[k * Q + l] = (1.0 - p->omega[k]) * f[k * Q + l] + p->omega[k] * feq[k * Q + l];",
                             "out[k * Q + l] = (1.0 - p->omega[0]) * f[k * Q + l] + p->omega[0] * feq[k * Q + l];"),
    "moment_not_divided": ("q[d] = t / p->dx;", "q[d] = t;"),
    "init_pressure_scale": ("p->dx * p->dx * p->rho_bar * ph", "p->dx * p->rho_bar * ph"),
    "macro_velocity_sign": ("u_out[d * N + node] = q[d] / rho;", "u_out[d * N + node] = -q[d] / rho;"),
}


@pytest.fixture(scope="module")
def workdir(tmp_path_factory):
    d = tmp_path_factory.mktemp("mutants")
    shutil.copy(os.path.join(os.path.dirname(SRC), "vlbm_oracle.h"), d / "vlbm_oracle.h")
    return d


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(workdir, name):
    old, new = MUTATIONS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    src = workdir / f"{name}.c"
    src.write_text(text.replace(old, new))
    lib = str(workdir / f"lib{name}.so")
    subprocess.run(["gcc", *obuild.CFLAGS, "-I", str(workdir), str(src), "-o", lib, "-lm"], check=True)
    bad = P.failing_pins(oracle.Oracle(lib))
    assert bad, f"mutation {name} passes every pin"


# The Poiseuille driver (oracle/poiseuille.py) uses the oracle's relaxation, equilibria,
# initialisation and read-out but streams with its own ghost cells, so the two transport
# mutations cannot reach it; and its two momentum fields share one alpha, which hides
# alpha_of_wrong_field.  Those three are caught by the other pins (test above).
NOT_REACHED_BY_TABLE2 = {"stream_direction", "stream_missing_axis", "alpha_of_wrong_field"}


@pytest.mark.parametrize("name", sorted(set(MUTATIONS) - NOT_REACHED_BY_TABLE2))
def test_planted_mistake_misses_table2(workdir, name):
    """The same mistakes against the printed values alone: the 75-cell Poiseuille run of Table 2
    (omega_q = 1.15, corrected walls, printed 1.485E-05) moves by more than one printed unit."""
    from oracle.poiseuille import Poiseuille
    lib = workdir / f"lib{name}.so"
    if not lib.exists():
        old, new = MUTATIONS[name]
        src = workdir / f"{name}.c"
        src.write_text(open(SRC).read().replace(old, new))
        subprocess.run(["gcc", *obuild.CFLAGS, "-I", str(workdir), str(src), "-o", str(lib), "-lm"], check=True)
    sim = Poiseuille(oracle.Oracle(str(lib)), 75, 1.15, corrected=True)
    sim.run_to(0.05)
    err = sim.l2_error_ux()
    assert not abs(err - 1.485e-05) <= 1e-08, (name, err)
