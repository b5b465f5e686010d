"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/ifgf.h declares.  No compute call (no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(ifgf_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libifgf():
    from paper_2010_02857_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(libifgf):
    declared = _declared()
    assert "ifgf_plan_create" in declared and "ifgf_apply_adjoint" in declared
    for name in declared:
        assert hasattr(libifgf, name), name


def test_binding_mirrors_the_header():
    import paper_2010_02857_gb300 as pkg
    assert sorted(pkg.EXPORTS) == _declared()


def test_last_error_without_plan_is_safe(libifgf):
    libifgf.ifgf_last_error.restype = ctypes.c_char_p
    libifgf.ifgf_last_error.argtypes = [ctypes.c_void_p]
    assert isinstance(libifgf.ifgf_last_error(None), bytes)


def test_invalid_arguments_rejected_before_any_device_work(libifgf):
    import paper_2010_02857_gb300 as pkg
    import numpy as np
    pts = np.zeros((1, 3))
    with pytest.raises(pkg.IFGFError) as e:
        pkg.plan_create(pts, 1.0, 4)
    assert e.value.status == 1
    pts = np.random.default_rng(0).normal(size=(10, 3))
    for kw in [dict(levels=2), dict(levels=21), dict(kappa=-1.0), dict(p_radial=2, p_angular=2),
               dict(timeout_s=-1.0)]:
        args = dict(kappa=1.0, levels=4)
        args.update(kw)
        with pytest.raises(pkg.IFGFError) as e:
            pkg.plan_create(pts, args.pop("kappa"), args.pop("levels"), **args)
        assert e.value.status == 1


def test_plan_entry_points_reject_a_null_plan(libifgf):
    # every call that takes a plan returns IFGF_EINVAL (1) for NULL, without touching
    # the device
    P, i = ctypes.c_void_p, ctypes.c_int
    calls = [
        ("ifgf_plan_set_graphs", [P, i], (None, 1)),
        ("ifgf_plan_set_tiles", [P, i, i], (None, 0, 2)),
        ("ifgf_plan_autotune", [P, i, i, P, P, P], (None, 4, 1, None, None, None)),
        ("ifgf_plan_autotune_cached", [P, i, i, ctypes.c_char_p, P, P, P], (None, 4, 1, b"x", None, None, None)),
        ("ifgf_plan_tune_key", [P, i, ctypes.c_char_p, i], (None, 4, None, 0)),
        ("ifgf_plan_set_profiling", [P, i], (None, 1)),
        ("ifgf_apply", [P, P, P, i, P], (None, None, None, 1, None)),
        ("ifgf_apply_adjoint", [P, P, P, i, P], (None, None, None, 1, None)),
    ]
    for name, argtypes, args in calls:
        f = getattr(libifgf, name)
        f.argtypes = argtypes
        f.restype = ctypes.c_int
        assert f(*args) == 1, name
    # destroying NULL is a no-op, like free(NULL)
    libifgf.ifgf_plan_destroy.argtypes = [P]
    libifgf.ifgf_plan_destroy.restype = ctypes.c_int
    assert libifgf.ifgf_plan_destroy(None) == 0


def test_options_struct_layout_matches_header(tmp_path):
    # the ctypes mirror of ifgf_options must have the C layout of include/ifgf.h
    import shutil
    import subprocess
    import paper_2010_02857_gb300 as pkg
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "layout.c"
    fields = [f[0] for f in pkg.ifgf_options._fields_]
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"ifgf.h\"\nint main(void) {\n"
                   "  printf(\"%zu\", sizeof(ifgf_options));\n"
                   + "".join(f'  printf(" %zu", offsetof(ifgf_options, {f}));\n' for f in fields)
                   + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(root, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(pkg.ifgf_options)] + [getattr(pkg.ifgf_options, f).offset for f in fields]
    assert got == want
