"""CPU checks of the product library: it builds for sm_103a, loads, exports every
entry point the public header declares, and fails cleanly without a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2201_13240_gb300 import build as B
    B.build_lib()
    import paper_2201_13240_gb300 as wos
    return wos.load()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "wos.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(wos_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_entry_points():
    names = declared_symbols()
    for n in ("wos_create", "wos_destroy", "wos_problem_create", "wos_sigma_bar", "wos_solve",
              "wos_walk_estimates", "wos_finalize", "wos_solve_host"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_library_is_built_for_sm103a():
    import subprocess
    from paper_2201_13240_gb300 import build as B
    out = subprocess.run(["cuobjdump", "--list-elf", B.LIB], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def test_version_and_null_handles(lib):
    assert b"sm_103a" in lib.wos_version()
    assert lib.wos_destroy(None) == -1
    assert lib.wos_problem_destroy(None) == -1
    assert lib.wos_last_error(None) == b"null context"
    assert lib.wos_create(None, 0) == -1


def test_create_without_gpu_reports_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    assert lib.wos_create(C.byref(h), 0) == -3
    assert not h.value
