"""CPU-side checks of the C ABI: the library builds and loads, exports every
function include/lbm.h declares, and rejects invalid parameters before touching
a device.  No compute call runs here."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1906_11027_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_every_declared_function():
    lib_path = lbm._build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r" T (lbm_[a-z0-9_]+)", out))
    missing = declared_functions() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"
    lib = lbm.load()
    for name in declared_functions():
        assert hasattr(lib, name)


def test_binding_covers_the_header():
    assert declared_functions() <= set(lbm.exported_symbols())


def test_strerror_and_defaults():
    assert lbm.lbm_strerror(lbm.LBM_EINVAL) == "invalid argument"
    p = lbm.lbm_params_default()
    assert (p.nx, p.ny, p.nz, p.lattice, p.G, p.tau) == (64, 64, 1, lbm.LBM_D2Q9, -5.0, 1.0)


@pytest.mark.parametrize("field,value,code", [
    ("nx", 4, lbm.LBM_EINVAL),
    ("tau", 0.5, lbm.LBM_EINVAL),
    ("lattice", 9, lbm.LBM_EINVAL),
    ("stencil", 5, lbm.LBM_EINVAL),
    ("precision", 7, lbm.LBM_EINVAL),
])
def test_create_rejects_invalid_parameters(field, value, code):
    p = lbm.lbm_params_default()
    setattr(p, field, value)
    h = ctypes.c_void_p()
    assert lbm.load().lbm_create(ctypes.byref(p), ctypes.byref(h)) == code
    assert h.value is None


@pytest.mark.parametrize("changes,code", [
    (dict(lattice=lbm.LBM_D2Q13, collision=lbm.LBM_MRT), lbm.LBM_EUNSUPPORTED),
    (dict(lattice=lbm.LBM_D3Q19, nz=16, stencil=lbm.LBM_ISO10), lbm.LBM_EUNSUPPORTED),
    (dict(psi=lbm.LBM_PSI_PENG_ROBINSON, T_over_Tc=0.8, G=-1.0, precision=lbm.LBM_FP32_SHIFTED),
     lbm.LBM_EUNSUPPORTED),
    (dict(psi=lbm.LBM_PSI_PENG_ROBINSON, T_over_Tc=0.8, G=1.0), lbm.LBM_EINVAL),
    (dict(collision=lbm.LBM_MRT, s_q=2.5), lbm.LBM_EINVAL),
    (dict(lattice=lbm.LBM_D3Q19, nz=16, wall_rows=1), lbm.LBM_EUNSUPPORTED),
    (dict(wall_rows=2, path=lbm.LBM_PATH_ONE_PASS), lbm.LBM_EUNSUPPORTED),
    (dict(lattice=lbm.LBM_D2Q25, wall_rows=1), lbm.LBM_EINVAL),   # thinner than the reach of 2
    (dict(stencil=lbm.LBM_ISO8, wall_rows=1), lbm.LBM_EINVAL),    # thinner than the force radius of 2
    (dict(wall_rows=64), lbm.LBM_EINVAL),                          # no fluid left
    (dict(wall_rows=2, rho_w=0.0), lbm.LBM_EINVAL),
])
def test_create_rejects_unsupported_combinations(changes, code):
    p = lbm.lbm_params_default()
    for k, v in changes.items():
        setattr(p, k, v)
    h = ctypes.c_void_p()
    assert lbm.load().lbm_create(ctypes.byref(p), ctypes.byref(h)) == code


def test_null_arguments_rejected():
    lib = lbm.load()
    assert lib.lbm_create(None, None) == lbm.LBM_EINVAL
    assert lib.lbm_step(None, 1) == lbm.LBM_EINVAL
    assert lib.lbm_destroy(None) == lbm.LBM_OK


def test_params_layout_matches_the_header(tmp_path):
    """The ctypes mirror of lbm_params has the C struct's size and field offsets."""
    fields = [f[0] for f in lbm.lbm_params._fields_]
    prog = tmp_path / "layout.c"
    prog.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "lbm.h"\nint main(void) {\n'
                    '  printf("size %zu\\n", sizeof(lbm_params));\n'
                    + "".join(f'  printf("{f} %zu\\n", offsetof(lbm_params, {f}));\n' for f in fields)
                    + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(prog)], check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                        check=True).stdout.splitlines())
    assert int(out["size"]) == ctypes.sizeof(lbm.lbm_params)
    for f in fields:
        assert int(out[f]) == getattr(lbm.lbm_params, f).offset, f
