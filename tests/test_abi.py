"""The C ABI (no GPU needed): the library builds for sm_103a, loads, and exports
every function include/rbfgb.h declares; the Python binding covers them all.
No compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(rbf_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("rbf_create", "rbf_set_nodes", "rbf_build_stencils", "rbf_compute_weights", "rbf_step",
                 "rbf_solve", "rbf_permeability", "rbf_drag"):
        assert must in names


def test_library_builds_loads_and_exports():
    import paper_2404_14195_gb300 as rbf
    path = rbf._build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    # the Python binding wraps every declared function
    assert set(declared_functions()) <= set(rbf.ABI)


def test_no_gpu_fails_loudly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import paper_2404_14195_gb300 as rbf
    rbf._build.build()
    with pytest.raises(rbf.RbfError):
        rbf.Solver(0)


@pytest.mark.parametrize("compiler,std,ext", [("gcc", "-std=c99", "c"), ("g++", "-std=c++11", "cpp")])
def test_header_compiles_for_c_and_cpp_callers(tmp_path, compiler, std, ext):
    """The boundary is plain C: the header alone compiles as C99 and C++11 with
    warnings as errors (no CUDA or torch types leak into it)."""
    import shutil
    import subprocess
    if shutil.which(compiler) is None:
        pytest.skip(f"{compiler} not found")
    src = tmp_path / f"use.{ext}"
    src.write_text('#include "rbfgb.h"\nint main(void) { return 0; }\n')
    r = subprocess.run([compiler, std, "-Wall", "-Wextra", "-Werror", "-pedantic", "-fsyntax-only",
                        "-I", os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_output_buffers_are_checked_before_any_call():
    """Result readers write a caller's buffer in place (a pinned host array, so the
    device-to-host copy lands there directly) only when it has the result's shape,
    float64 type and C layout; anything else is refused before the C ABI is called."""
    import numpy as np

    from paper_2404_14195_gb300 import _out
    a = _out(None, (5, 4))
    assert a.shape == (5, 4) and a.dtype == np.float64
    b = np.zeros((5, 4))
    assert _out(b, (5, 4)) is b
    for bad in (np.zeros((4, 5)), np.zeros((5, 4), np.float32), np.zeros((5, 8))[:, ::2], [[0.0] * 4] * 5):
        with pytest.raises(ValueError):
            _out(bad, (5, 4))
    ro = np.zeros((5, 4))
    ro.flags.writeable = False
    with pytest.raises(ValueError):
        _out(ro, (5, 4))
