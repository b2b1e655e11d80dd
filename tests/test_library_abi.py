"""The C-ABI library builds for sm_103a, loads, and exports every entry point of include/pum.h.

No GPU is needed: only calls that fail before touching a device are made here.
"""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "pum.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s+\**([a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2509_06744_gb300 import _lib
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["pum_assemble", "bfsai_setup", "cheb4_smooth", "vcycle_apply", "pcg_solve",
                     "pum_hier_from_bsr", "pum_create", "pum_destroy", "pum_hier_save", "pum_hier_load"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_library_built_for_sm103a():
    from paper_2509_06744_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_null_arguments_are_rejected_without_a_device(lib):
    from paper_2509_06744_gb300 import _lib
    assert lib.pum_create(None, 0, None) == _lib.PUM_ERR_INVALID_ARG
    assert lib.pum_destroy(None) == _lib.PUM_ERR_INVALID_ARG
    assert lib.pum_hier_destroy(None) == _lib.PUM_ERR_INVALID_ARG
    assert lib.pum_last_error(None) == b"NULL context"
    assert lib.pum_launch_count(None) == 0
    n = C.c_int32()
    assert lib.pum_hier_levels(None, C.byref(n)) == _lib.PUM_ERR_INVALID_ARG
    # batches validate their arrays before any device work
    assert lib.pum_solve_batch(None, 1, None, 1, None, None, None, 0, None) == _lib.PUM_ERR_INVALID_ARG
    fp, sp = _lib.FsaiParams(), _lib.SmootherParams()
    assert lib.pum_setup_batch(None, 0, None, 0, C.byref(fp), C.byref(sp), None) == _lib.PUM_ERR_INVALID_ARG


def test_missing_device_is_an_error_not_a_fallback(lib):
    """On a machine without a CUDA device the library refuses to create a context."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2509_06744_gb300 import Context, PumError
    with pytest.raises(PumError):
        Context(0)


# C struct of include/pum.h -> ctypes mirror in the binding
_STRUCTS = {"pum_bsr_view": "BsrView", "pum_bsr_host": "BsrHost", "pum_problem": "Problem",
            "bfsai_params": "FsaiParams", "smoother_params": "SmootherParams", "pcg_report": "PcgReport",
            "pum_level_info": "LevelInfo"}


def _c_layout(tmp_path):
    """sizeof and field offsets of the header's structs, from a C program compiled with gcc."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    from paper_2509_06744_gb300 import _lib
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "pum.h"', "int main(void) {"]
    for cname, pyname in _STRUCTS.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in getattr(_lib, pyname)._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {(a, b): int(c) for a, b, c in (line.split() for line in out.splitlines())}


def test_struct_layouts_match_the_header(tmp_path):
    """Every ctypes mirror has the C struct's field names, offsets and size (a field added on one
    side only, or in another order, fails here)."""
    from paper_2509_06744_gb300 import _lib
    c = _c_layout(tmp_path)
    for cname, pyname in _STRUCTS.items():
        py = getattr(_lib, pyname)
        assert C.sizeof(py) == c[(cname, "size")], cname
        for f, _ in py._fields_:
            assert getattr(py, f).offset == c[(cname, f)], f"{cname}.{f}"


def test_c_example_builds_against_the_library(tmp_path):
    """tests/c_example/solve_biharmonic.c uses only include/pum.h (and the CUDA runtime for its
    vectors): it compiles warning-free, links against libpum.so and, without a CUDA device, reports
    the failed pum_create (exit status 2) instead of crashing; with one it solves (exit status 0)."""
    import shutil
    import subprocess
    from paper_2509_06744_gb300 import _lib
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    if not shutil.which("gcc") or not os.path.exists(os.path.join(cuda, "include", "cuda_runtime.h")):
        pytest.skip("gcc or the CUDA headers are not available")
    _lib.load()  # builds the library when it is missing
    libdir = os.path.dirname(_lib.lib_path())
    exe = tmp_path / "solve_biharmonic"
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                        "-I", os.path.join(cuda, "include"), os.path.join(ROOT, "tests", "c_example", "solve_biharmonic.c"),
                        "-L", libdir, "-lpum", "-L", os.path.join(cuda, "lib64"), "-lcudart",
                        f"-Wl,-rpath,{libdir}", f"-Wl,-rpath,{os.path.join(cuda, 'lib64')}", "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    import torch
    if torch.cuda.is_available():
        assert run.returncode == 0, run.stderr
        assert "converged" in run.stdout
    else:
        assert run.returncode == 2, run.stderr
        assert "pum_create" in run.stderr
