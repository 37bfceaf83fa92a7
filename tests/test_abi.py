"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function that include/*.h declares; argument errors are reported before any
GPU work (these calls need no device)."""
import ctypes
import glob
import os
import re

import pytest

from paper_2603_05447_gb300 import _build, gpe

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(?:int|void|double)\s+\*?\s*(gpe_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return gpe.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["gpe_grid_create_dense", "gpe_grid_create_analytic", "gpe_step_imag",
                     "gpe_step_real", "gpe_observables", "gpe_state_load", "gpe_state_store"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    missing = [n for n in declared_functions() if n not in gpe._SIGS or not hasattr(gpe, n)]
    assert not missing, missing


def test_version_and_argument_errors_without_gpu(lib):
    assert gpe.gpe_version() >= 100
    out = ctypes.c_void_p()
    assert lib.gpe_grid_create_analytic(None, None, 1.0, None, ctypes.byref(out), None) == gpe.GPE_ERR_ARG
    assert "box is NULL" in gpe.last_error()
    box = gpe.make_box(0, 4, 4, 0.1)
    pot = gpe.make_potential(gpe.GPE_POT_HARMONIC, 1, 1, 1)
    assert lib.gpe_grid_create_analytic(ctypes.byref(box), ctypes.byref(pot), 1.0, None,
                                        ctypes.byref(out), None) == gpe.GPE_ERR_ARG
    box = gpe.make_box(8, 8, 8, 0.1)
    bad = gpe.make_potential(7)
    assert lib.gpe_grid_create_analytic(ctypes.byref(box), ctypes.byref(bad), 1.0, None,
                                        ctypes.byref(out), None) == gpe.GPE_ERR_ARG
    assert "unknown potential kind" in gpe.last_error()
    with pytest.raises(gpe.GpeError) as e:
        gpe.gpe_grid_create_analytic(box, bad, 1.0)
    assert e.value.code == gpe.GPE_ERR_ARG


def test_struct_layouts_match_header():
    assert ctypes.sizeof(gpe.gpe_box) == 3 * 8 + 6 * 8
    assert ctypes.sizeof(gpe.gpe_grid_opts) == 8 * 4
    assert ctypes.sizeof(gpe.gpe_potential) == 8 + 8 * 8
    assert ctypes.sizeof(gpe.gpe_real_params) == 2 * 8 + 4 * 4 + 8 + 16 * 8
    assert ctypes.sizeof(gpe.gpe_obs) == 7 * 8
    assert ctypes.sizeof(gpe.gpe_grid_info) == 4 * 8 + 6 * 4 + 8 + ctypes.sizeof(gpe.gpe_box)


def header_structs():
    """Field names, in order, of every `typedef struct name {...} name;` in
    include/*.h (arrays keep their name)."""
    out = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"typedef\s+struct\s+(\w+)\s*\{(.*?)\}\s*(\w+)\s*;", text, flags=re.S):
            names = []
            for decl in m.group(2).split(";"):
                decl = decl.strip()
                if not decl:
                    continue
                # `type a, b[4]` or `const type *p`: each declarator's name is
                # its last identifier once array bounds are dropped
                for part in decl.split(","):
                    names.append(re.findall(r"\w+", re.sub(r"\[.*?\]", "", part))[-1])
            out[m.group(3)] = names
    return out


def test_binding_structs_match_the_header_field_by_field():
    """A renamed or reordered field in the binding would silently drop a
    setting (ctypes accepts unknown attributes): compare names and order."""
    structs = header_structs()
    assert "gpe_grid_opts" in structs and "gpe_real_params" in structs and "gpe_ramp_pot" in structs
    for name, fields in structs.items():
        cls = getattr(gpe, name, None)
        assert cls is not None, f"the binding has no {name}"
        assert [f[0] for f in cls._fields_] == fields, name


def test_header_is_plain_c(tmp_path):
    """The boundary header compiles as C99 and as C++ (no torch or CUDA types
    in the signatures)."""
    import shutil
    import subprocess
    for cc, std, ext in (("gcc", "-std=c99", "c"), ("g++", "-std=c++17", "cpp")):
        if shutil.which(cc) is None:
            pytest.skip(f"{cc} not available")
        src = tmp_path / f"use.{ext}"
        src.write_text('#include "gpe.h"\nint main(void) { return 0; }\n')
        r = subprocess.run([cc, std, "-Wall", "-Wextra", "-Werror", "-fsyntax-only",
                            "-I" + os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
