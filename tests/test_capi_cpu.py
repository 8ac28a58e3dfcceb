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
    """Every translation unit is compiled with one -gencode for sm_103a (no PTX for JIT)."""
    from paper_2201_13240_gb300 import build as B
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert "sm_103a" in open(os.path.join(ROOT, "paper_2201_13240_gb300", "csrc", "wos_jit.cu")).read()


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


# The calls of the problem statement (Sec. 3: a domain, the fields of eq. 1, a problem,
# its delta-tracking bound, per-point estimates, batches and the replay adjoint) and the
# exported name that provides each.  Two names differ from the plain problem-statement
# form because the descriptor-based calls of the same purpose keep the shorter names:
# assembling a problem from handles is wos_problem_assemble (wos_problem_create takes a
# description), and the solve returning (mean, var, count) is wos_solve_mean (wos_solve
# adds raw sums for checkpointing).
PROBLEM_STATEMENT_CALLS = {
    "wos_create": "wos_create",
    "wos_destroy": "wos_destroy",
    "wos_last_error": "wos_last_error",
    "wos_domain_box": "wos_domain_box",
    "wos_domain_sdf": "wos_domain_sdf",
    "wos_domain_mesh": "wos_domain_mesh",
    "wos_field_analytic": "wos_field_analytic",
    "wos_field_grid": "wos_field_grid",
    "wos_problem_create(domain, alpha, sigma, Phi, f, g)": "wos_problem_assemble",
    "wos_problem_sigma_bar": "wos_problem_sigma_bar",
    "wos_solve(..., mean, var, count, ...)": "wos_solve_mean",
    "wos_solve_batched": "wos_solve_batched",
    "wos_adjoint(..., grad_sigma_grid, grad_alpha_grid)": "wos_adjoint",
}


def test_problem_statement_calls_are_declared_and_exported(lib):
    names = declared_symbols()
    for call, name in PROBLEM_STATEMENT_CALLS.items():
        assert name in names, call
        assert hasattr(lib, name), call


def test_handle_constructors_validate_on_the_host(lib):
    """Domain and field constructors need no device and accept a NULL context."""
    import paper_2201_13240_gb300 as wos
    vp, dv = C.c_void_p, lambda *v: (C.c_double * max(1, len(v)))(*v)
    h = vp()
    assert lib.wos_domain_box(None, 3, dv(0, 0, 0), dv(1, 1, 1), C.byref(h)) == 0 and h.value
    assert lib.wos_domain_destroy(h) == 0
    assert lib.wos_domain_box(None, 4, dv(0, 0, 0), dv(1, 1, 1), C.byref(h)) == -1 and not h.value
    assert lib.wos_domain_box(None, 2, dv(0, 1), dv(1, 1), C.byref(h)) == -1
    assert lib.wos_domain_sdf(None, 2, 1, dv(0, 0, 0, 0.5), C.byref(h)) == 0
    lib.wos_domain_destroy(h)
    assert lib.wos_domain_sdf(None, 2, 1, dv(0, 0, 0, -0.5), C.byref(h)) == -1
    assert lib.wos_domain_sdf(None, 3, 2, dv(0, 0, 0, 0.7, 0.5), C.byref(h)) == -1  # inner > outer
    assert lib.wos_domain_sdf(None, 3, 0, dv(0, 0, 0, 1), C.byref(h)) == -1       # a box is not an SDF kind
    assert lib.wos_field_analytic(None, 1, dv(2.5), 1, C.byref(h)) == 0
    lib.wos_field_destroy(h)
    assert lib.wos_field_analytic(None, 1, dv(2.5, 1.0), 2, C.byref(h)) == -1
    terms = wos.pack_terms([{"c": 1.0, "atoms": [(1, 3.14, 0.0), (5, 1.0, 0.0)]}])
    assert lib.wos_field_analytic(None, 2, dv(*terms), len(terms), C.byref(h)) == 0
    lib.wos_field_destroy(h)
    bad = list(terms)
    bad[1] = 9.0  # no atom type 9
    assert lib.wos_field_analytic(None, 2, dv(*bad), len(bad), C.byref(h)) == -1
    assert lib.wos_field_analytic(None, 3, dv(*terms), len(terms) - 1, C.byref(h)) == -1
    res = (C.c_int32 * 3)(8, 8, 1)
    assert lib.wos_field_grid(None, 2, res, dv(0, 0), dv(1, 1), vp(16), 5, C.byref(h)) == 0
    lib.wos_field_destroy(h)
    assert lib.wos_field_grid(None, 2, res, dv(0, 0), dv(1, 1), vp(16), 3, C.byref(h)) == -1
    assert lib.wos_field_grid(None, 2, (C.c_int32 * 3)(1, 8, 1), dv(0, 0), dv(1, 1), vp(16), 4, C.byref(h)) == -1
    assert lib.wos_problem_assemble(None, None, None, None, None, None, None, C.byref(h)) == -1
