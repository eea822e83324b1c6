"""The C-ABI library loads, exports every symbol include/lbm.h declares, and
its structs have the layout the Python binding assumes.  No compute calls: this
file runs without a GPU."""
from __future__ import annotations

import ctypes as ct
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2209_01444_gb300 import build_ext, lbm

    build_ext.build()
    return lbm.load()


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^LBM_API\s+[\w\s\*]+?\b(lbm_\w+)\s*\(", txt, flags=re.M)))


def test_header_declares_the_api():
    names = _declared()
    for required in ("lbm_create", "lbm_init_seeds", "lbm_step", "lbm_get_fields", "lbm_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2209_01444_gb300 import lbm

    out = subprocess.run(["nm", "-D", "--defined-only", lbm.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(lbm_\w+)$", out, flags=re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    for n in _declared():
        assert hasattr(lib, n)
        assert n in lbm.SIGNATURES, f"binding lacks {n}"


def test_struct_layout_matches_the_binding(tmp_path):
    from paper_2209_01444_gb300 import lbm

    src = tmp_path / "probe.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lbm.h"\n'
                   "int main(void){printf(\"%zu %zu %zu %zu %zu\\n\", sizeof(lbm_params), sizeof(lbm_seed),"
                   " sizeof(lbm_metrics), offsetof(lbm_params, storage), offsetof(lbm_params, bc));return 0;}\n")
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    sizes = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert sizes == [ct.sizeof(lbm.lbm_params), ct.sizeof(lbm.lbm_seed), ct.sizeof(lbm.lbm_metrics),
                     lbm.lbm_params.storage.offset, lbm.lbm_params.bc.offset]


def test_version_and_default_params(lib):
    from paper_2209_01444_gb300 import lbm

    assert b"sm_103a" in lib.lbm_version()
    p = lbm.lbm_params()
    assert lib.lbm_params_default(ct.byref(p), 64, 32) == 0
    assert (p.nx, p.ny, p.n_sub, p.storage) == (64, 32, 1, 0)
    assert p.k == pytest.approx(0.15) and p.lambda_ == pytest.approx(3.1913)


@pytest.mark.parametrize("field,value,why", [
    ("nx", 3, "nx and ny"),
    ("ny", 262141, "ny must be <= 262140"),
    ("isothermal", 2, "isothermal"),
    ("k", 1.0, "k must"),
    ("eps_s", 0.4, "eps_s"),
    ("n_sub", 0, "n_sub"),
    ("D", 0.0, "D, alpha, nu"),
    ("storage", 7, "storage"),
    ("lambda_", float("nan"), "finite"),
    ("gbetaT", float("inf"), "finite"),
    ("dir_theta", float("-inf"), "finite"),
])
def test_create_rejects_invalid_parameters_without_touching_the_device(lib, field, value, why):
    from paper_2209_01444_gb300 import lbm

    p = lbm.lbm_params()
    lib.lbm_params_default(ct.byref(p), 64, 64)
    setattr(p, field, value)
    h = ct.c_void_p()
    assert lib.lbm_create(ct.byref(p), ct.byref(h)) == lbm.LBM_EINVAL
    assert not h.value
    assert why in lib.lbm_last_error(None).decode()


def test_create_rejects_unpaired_periodic_walls(lib):
    from paper_2209_01444_gb300 import lbm

    p = lbm.lbm_params()
    lib.lbm_params_default(ct.byref(p), 64, 64)
    p.bc[0] = lbm.BC["inflow"]
    h = ct.c_void_p()
    assert lib.lbm_create(ct.byref(p), ct.byref(h)) == lbm.LBM_EINVAL
    assert "periodicity" in lib.lbm_last_error(None).decode()


def test_null_handle_is_refused_without_touching_the_device(lib):
    """Entry points given no handle return LBM_EINVAL before any CUDA call
    (each checks the handle first), so a caller's mistake costs no device
    state."""
    from paper_2209_01444_gb300 import lbm

    buf = (ct.c_double * 4)()
    fbuf = (ct.c_float * 4)()
    assert lib.lbm_step(None, 1) == lbm.LBM_EINVAL
    assert lib.lbm_synchronize(None) == lbm.LBM_EINVAL
    assert lib.lbm_set_io_chunk(None, 1 << 20) == lbm.LBM_EINVAL
    assert lib.lbm_get_fields(None, 1, ct.cast(buf, ct.POINTER(ct.c_double))) == lbm.LBM_EINVAL
    assert lib.lbm_get_fields_f32(None, 1, ct.cast(fbuf, ct.c_void_p)) == lbm.LBM_EINVAL
    assert lib.lbm_get_state(None, ct.cast(buf, ct.POINTER(ct.c_double))) == lbm.LBM_EINVAL
