"""C-ABI library: loads, exports every declared symbol, host-side parameter logic (CPU)."""
import math
import os
import re

import pytest

import paper_2607_24059_b300 as v
from paper_2607_24059_b300 import _binding as b

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            text = open(os.path.join(inc, fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(vlbm_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    names = declared_functions()
    assert len(names) >= 18
    for name in names:
        assert hasattr(b.lib, name), name
        assert name in b.EXPORTED, f"{name} not bound in python"


def test_defaults_follow_section_6():
    p = v.vlbm_params_default(2, (64, 64), 2 * math.pi / 64, 0.01, v.VLBM_FP32)
    assert p.mu == 8.0 and p.omega[0] == 1.2 and p.alpha[0] == 0.075 and p.omega[1] == 1.15
    rc, d = v.vlbm_params_check(p)
    assert rc == v.VLBM_OK
    # Prop. 1: nu = 2 mu alpha (1/omega - 1/2)
    assert abs(2 * 8.0 * d.alpha[1] * (1 / 1.15 - 0.5) - 0.01) < 1e-15
    assert abs(d.alpha[1] - 1.691176470588235e-3) < 1e-15
    assert abs(d.viscosity[2] - 0.01) < 1e-15
    assert abs(d.dt - (2 * math.pi / 64) ** 2 / 8.0) < 1e-18
    assert d.nodes == 64 * 64 and d.populations_per_node == 15 and d.bytes_per_population == 4
    assert d.lattice_bytes == 64 * 64 * 15 * 4
    p3 = v.vlbm_params_default(3, (8, 8, 8), 0.1, 0.01, v.VLBM_FP64)
    _, d3 = v.vlbm_params_check(p3)
    assert d3.populations_per_node == 28 and d3.lattice_bytes == 512 * 28 * 8


@pytest.mark.parametrize("field,value", [
    ("omega0", 0.0), ("omega0", 2.0), ("omega1", -0.1), ("alpha0", 0.26), ("alpha0", -0.01),
    ("gamma", 0.9), ("dx", 0.0), ("mu", -1.0), ("rho_bar", 0.0), ("n0", 0), ("dim", 4), ("precision", 9),
    ("reserved", 1), ("nu", -1.0),
])
def test_invalid_parameters_are_rejected(field, value):
    p = v.vlbm_params_default(2, (16, 16), 0.1, 0.01, v.VLBM_FP32)
    if field.startswith("omega"):
        p.omega[int(field[-1])] = value
    elif field.startswith("alpha"):
        p.alpha[int(field[-1])] = value
    elif field == "n0":
        p.n[0] = value
    else:
        setattr(p, field, value)
    with pytest.raises(v.VlbmError) as e:
        v.vlbm_params_check(p)
    assert e.value.code == v.VLBM_EINVAL


def test_alpha_from_nu_out_of_range_is_rejected():
    # a huge viscosity asks for alpha_q > 1/4 (Lemma 1)
    p = v.vlbm_params_default(2, (16, 16), 0.1, 10.0, v.VLBM_FP32)
    with pytest.raises(v.VlbmError):
        v.vlbm_params_check(p)


def test_3d_alpha_bound_is_one_sixth():
    p = v.vlbm_params_default(3, (8, 8, 8), 0.1, 0.0, v.VLBM_FP32)
    p.alpha[0] = 0.2
    with pytest.raises(v.VlbmError):
        v.vlbm_params_check(p)
    p.alpha[0] = 1.0 / 6.0
    assert v.vlbm_params_check(p)[0] in (v.VLBM_OK, v.VLBM_WSTABILITY)


def test_mu_bound_warning_and_strict_error():
    p = v.vlbm_params_default(2, (16, 16), 0.1, 0.01, v.VLBM_FP32)
    p.mu = 2.0          # below (alpha_rho + alpha_q)^(-1/2) = 3.6
    with pytest.warns(RuntimeWarning):
        rc, d = v.vlbm_params_check(p)
    assert rc == v.VLBM_WSTABILITY and d.mu_min > 2.0
    p.strict = 1
    with pytest.raises(v.VlbmError) as e:
        v.vlbm_params_check(p)
    assert e.value.code == v.VLBM_ESTABILITY


def test_strerror_covers_codes():
    for code in (0, 1, -1, -2, -3, -4, -5, -6, -7):
        assert v.vlbm_strerror(code) != "unknown status"


def test_null_pointers_are_einval():
    assert b.lib.vlbm_params_check(None, None) == v.VLBM_EINVAL
    assert b.lib.vlbm_step(None, 1, 0) == v.VLBM_EINVAL
    assert b.lib.vlbm_init(None, None, None, 0) == v.VLBM_EINVAL
    assert b.lib.vlbm_invariants(None, None) == v.VLBM_EINVAL
    assert b.lib.vlbm_state_bytes(None) == 0
    b.lib.vlbm_destroy(None)


def test_tensor_core_entry_points_reject_misaligned_arrays():
    """Alignment is checked on the host before any launch, so fake addresses are never dereferenced."""
    a = 0x100000                                   # 16-byte aligned
    # conv: X, W, Y and Z 16-byte aligned
    assert b.lib.vlbm_sur_conv3x3(a + 8, a, a, a, None, 1, 8, 8, 64, 64, 1, a, None) == v.VLBM_EINVAL
    assert b.lib.vlbm_sur_conv3x3(a, a + 8, a, a, None, 1, 8, 8, 64, 64, 1, a, None) == v.VLBM_EINVAL
    assert b.lib.vlbm_sur_conv3x3(a, a, a, a + 8, None, 1, 8, 8, 64, 64, 1, a, None) == v.VLBM_EINVAL
    assert b.lib.vlbm_sur_conv3x3(a, a, a, a, a + 8, 1, 8, 8, 64, 64, 1, a, None) == v.VLBM_EINVAL
    # weight gradient: X and dZ 16-byte aligned
    assert b.lib.vlbm_sur_conv3x3_wgrad(a + 8, a, a, a, 1, 8, 8, 64, 64, a, None) == v.VLBM_EINVAL
    assert b.lib.vlbm_sur_conv3x3_wgrad(a, a + 8, a, a, 1, 8, 8, 64, 64, a, None) == v.VLBM_EINVAL
    # GEMM: A and B 16-byte aligned
    assert b.lib.vlbm_tc_gemm_bf16(a + 8, a, a, 128, 16, 64, a, None) == v.VLBM_EINVAL
    assert b.lib.vlbm_tc_gemm_bf16(a, a + 8, a, 128, 16, 64, a, None) == v.VLBM_EINVAL


def test_binding_constants_match_header():
    """Every VLBM_* integer constant of the binding has the value include/vlbm.h defines."""
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    text = open(os.path.join(root, "include", "vlbm.h")).read()
    defines = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(VLBM_\w+)\s+\(?(-?\d+)\)?", text)}
    assert "VLBM_OPT_ROUNDING_16" in defines
    checked = 0
    for name, value in defines.items():
        if hasattr(v, name):
            assert getattr(v, name) == value, name
            checked += 1
    assert checked >= 10
