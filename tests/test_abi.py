"""The C-ABI library builds, loads and exports every entry point of include/gz.h
(no GPU needed: only host-side calls that touch no device are made)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gz.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:gz_status|const char\s*\*)\s*(gz_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    import paper_1712_01294_gb300 as gz
    return gz.load_library()


def test_header_declares_the_hot_path_calls():
    names = declared_functions()
    for n in ("gz_create", "gz_destroy", "gz_density", "gz_gradients", "gz_hydro_fluxes",
              "gz_step", "gz_step_backward", "gz_get_status", "gz_timestep"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\sT\s(gz_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert getattr(lib, n) is not None


def test_param_struct_layout_matches_header(lib, tmp_path):
    import paper_1712_01294_gb300 as gz
    prog = tmp_path / "layout.c"
    fields = [f for f, _ in gz.Params._fields_]
    body = "\n".join(f'printf("%zu\\n", offsetof(gz_params, {f}));' for f in fields)
    prog.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"gz.h\"\nint main(void){\n"
                    + body + '\nprintf("%zu\\n", sizeof(gz_params));\n'
                    + 'printf("%zu\\n", sizeof(gz_particles));\nreturn 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    offs = [getattr(gz.Params, f).offset for f in fields]
    assert vals[:-2] == offs
    assert vals[-2] == C.sizeof(gz.Params)
    assert vals[-1] == C.sizeof(gz._Particles)


def test_default_params_and_argument_validation_without_device(lib):
    import paper_1712_01294_gb300 as gz
    p = gz.default_params()
    assert abs(p.gamma - 5.0 / 3.0) < 1e-15 and p.ngb == 32.0 and p.cfl == 0.2
    assert p.precision == gz.GZ_MIXED32 and p.max_ngb == 128 and p.hancock == 1
    assert lib.gz_default_params(None) == gz.GZ_E_INVAL
    h = C.c_void_p()
    counts = (C.c_int64 * 2)(10, 0)  # an empty box is rejected before any device work
    assert lib.gz_create(C.byref(p), 2, C.cast(counts, C.c_void_p), None, C.byref(h)) == gz.GZ_E_INVAL
    assert lib.gz_create(C.byref(p), 0, C.cast(counts, C.c_void_p), None, C.byref(h)) == gz.GZ_E_INVAL
    bad = gz.default_params(gamma=1.0)
    counts = (C.c_int64 * 1)(100)
    assert lib.gz_create(C.byref(bad), 1, C.cast(counts, C.c_void_p), None, C.byref(h)) == gz.GZ_E_INVAL
    bad = gz.default_params(h_lim=0.7)
    assert lib.gz_create(C.byref(bad), 1, C.cast(counts, C.c_void_p), None, C.byref(h)) == gz.GZ_E_INVAL
    assert lib.gz_density(None, None, None, None) == gz.GZ_E_INVAL
    assert lib.gz_step(None, None, 0.0, None) == gz.GZ_E_INVAL
    assert lib.gz_get_status(None, None, None, None, 0) == gz.GZ_E_INVAL
    assert lib.gz_destroy(None) == gz.GZ_E_INVAL
    assert lib.gz_version().startswith(b"gz-mfm")


def test_product_package_does_not_use_the_oracle():
    pkg = os.path.join(ROOT, "paper_1712_01294_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", txt, flags=re.M), f
                assert "gz_oracle" not in txt and "libgz_oracle" not in txt, f
