"""Problem-specialised walk kernels (runtime compilation), host side.

* The generated field code, compiled here by g++ in FP64, equals the oracle's field
  evaluation (value, gradient, Laplacian) for every atom type, constant and zero
  fields, a manufactured source and an extra drift: the code generator is pinned to
  the oracle's reading of the separable fields, independently of the CUDA path.
* NVRTC compiles the specialised kernel for sm_103a (no device needed) for 2D and
  3D problems, analytic, grid, mesh and CSG domains, the extra drift, both
  precisions and the plain / weight-window / gradient variants.
* Invalid descriptions are refused with WOS_EINVAL.
"""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

import workloads as W
from workloads import COS, COSH, EXP, LIN, QUAD, SIN, SINH

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2201_13240_gb300", "csrc")


@pytest.fixture(scope="module")
def wos():
    from paper_2201_13240_gb300 import build as B
    B.build_lib()
    import paper_2201_13240_gb300 as m
    return m


def all_atoms_problem():
    """3D problem whose fields use every atom type with non-trivial k and phi."""
    alpha = W.sst(W.term(2.0), W.term(0.3, (SIN, 1.7, 0.2), (COS, 0.9, -0.4)),
                  W.term(0.1, (EXP, 0.5, 0.1), None, (QUAD, 1.3, -0.2)),
                  W.term(0.05, (SINH, 0.8, 0.0), (COSH, 0.6, 0.3), (LIN, 2.0, 1.0)))
    phi = W.sst(W.term(0.7, (LIN, 1.0, 0.0), (SIN, 2.5, 0.3)), W.term(-0.2, None, None, (COSH, 1.1, -0.5)))
    sigma = W.sst(W.term(1.5), W.term(0.4, (QUAD, 0.7, 0.1), (EXP, -0.3, 0.0), (SINH, 1.2, 0.2)))
    u = W.sst(W.term(1.0, (EXP, 0.5, 0.0), (SIN, 3.1, 0.0), (COS, 3.1, 0.2)),
              W.term(0.3, (COSH, 0.4, 0.0), None, (LIN, 1.0, 0.5)))
    omega = [W.sst(W.term(0.5, None, (SIN, 6.2, 0.0))), W.sst(W.term(0.25, None, None, (COS, 6.2, 0.0))),
             W.const(0.5)]
    return W.problem(3, W.box([0, 0, 0], [1, 1, 1]), alpha, sigma, W.manufactured(), u, phi=phi, um=u,
                     omega=omega)


ANALYTIC = {
    "all_atoms": all_atoms_problem,
    "cube3d": W.cube3d_problem,
    "square2d": W.square2d_problem,
    "hifreq": W.hifreq_alpha_problem,
    "screened_ball": W.screened_ball_problem,
}

FIELD_IDS = {"alpha": 0, "phi": 1, "sigma": 2, "f": 3, "g": 4, "um": 5}

HARNESS = r"""
#define __device__
#define __forceinline__ inline
%(source)s
extern "C" void eval_field(int id, const double* x, double* out) {
  static wos::DevProblem<double> P;  // only grid fields read it
  wos::FieldVal<double> o = wos::jit_field<%(dim)d, double>(P, id, x[0], x[1], x[2], true);
  out[0] = o.v; out[1] = o.gx; out[2] = o.gy; out[3] = o.gz; out[4] = o.lap;
}
"""


def _host_fields(wos, desc, tmp_path, name):
    """The generated field code of desc compiled by g++ (FP64), as a callable."""
    src = (wos.jit_source(desc).replace('#include "wos_walk_impl.cuh"', '#include "wos_problem.cuh"')
           .replace('#include "wos_adjoint_impl.cuh"', ''))
    cpp = tmp_path / f"jit_{name}.cpp"
    so = tmp_path / f"jit_{name}.so"
    cpp.write_text(HARNESS % {"source": src, "dim": desc["dim"]})
    subprocess.run(["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-Wno-unknown-pragmas", "-I", CSRC,
                    "-o", str(so), str(cpp)], check=True)
    lib = C.CDLL(str(so))
    lib.eval_field.argtypes = [C.c_int, C.c_void_p, C.c_void_p]

    def ev(fid, x):
        xx = np.zeros(3)
        xx[: len(x)] = x
        out = np.zeros(5)
        lib.eval_field(fid, xx.ctypes.data, out.ctypes.data)
        return out
    return ev


def _oracle_field(orc, pk, F, x):
    from oracle import _dptr, _load
    xx = np.zeros(3)
    xx[: len(x)] = x
    v, lap = C.c_double(), C.c_double()
    g = np.zeros(3)
    rc = _load().orc_field_eval(pk.ptr, C.pointer(F), _dptr(xx), C.byref(v), _dptr(g), C.byref(lap))
    assert rc == 0
    return np.array([v.value, g[0], g[1], g[2], lap.value])


@pytest.mark.parametrize("name", list(ANALYTIC))
def test_generated_fields_equal_oracle_fields(wos, orc, tmp_path, name):
    desc = ANALYTIC[name]()
    dim = desc["dim"]
    ev = _host_fields(wos, desc, tmp_path, name)
    pk = orc.pack(desc)
    rng = np.random.default_rng(5)
    fields = [(n, FIELD_IDS[n], getattr(pk.P, n)) for n in ("alpha", "phi", "sigma", "g", "um")]
    fields += [(f"omega{d}", 6 + d, pk.P.omega[d]) for d in range(dim)]
    if desc["f"]["kind"] != "manufactured":
        fields.append(("f", FIELD_IDS["f"], pk.P.f))
    checked = 0
    for fname, fid, F in fields:
        for _ in range(25):
            x = rng.uniform(-0.9, 1.1, size=dim)
            got = ev(fid, x)
            want = _oracle_field(orc, pk, F, x)
            if dim == 2:
                got[3] = want[3] = 0.0
            scale = max(1.0, np.abs(want).max())
            assert np.all(np.abs(got - want) <= 1e-12 * scale), (fname, x, got, want)
            checked += 1
    assert checked >= 25 * 5


def test_generated_source_folds_the_constants(wos):
    src = wos.jit_source(W.cube3d_problem())
    assert "#define WOS_JIT_F_KIND 3" in src  # manufactured source
    body = src.split("case FLD_ALPHA")[1].split("case FLD_PHI")[0]
    # alpha = 1 + 0.3 (x^2 + y^2 + z^2): no sin/cos/exp, literals as hex floats
    assert "w_sincos" not in body and "w_exp" not in body and "R(0x1.3333333333333p-2)" in body
    # the interpreter's descriptors are not read for analytic fields
    assert "P.terms" not in src and "field_eval" not in src


def GRID_DESC():
    sigma = np.random.default_rng(1).uniform(0.5, 2.0, (32, 32, 32)).astype(np.float32)
    return W.inverse_problem(sigma)


COMPILE = {
    "cube3d": (W.cube3d_problem, ("plain", "window", "grad")),
    "square2d": (W.square2d_problem, ("plain", "window", "grad")),
    "cube3d_literal_drift": (W.cube3d_literal_problem, ("plain",)),
    "grids": (GRID_DESC, ("plain", "grad")),
    "mesh": (lambda: W.mesh_manufactured_problem(level=2), ("plain", "grad")),
    "csg": (W.csg_variable_problem, ("plain",)),
    "all_atoms": (all_atoms_problem, ("plain",)),
}


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("name", list(COMPILE))
def test_specialised_kernel_compiles_for_sm103a(wos, name, precision):
    mk, variants = COMPILE[name]
    rc, log, nbytes = wos.jit_compile(mk(), precision, variants)
    if rc == wos.WOS_EUNSUPPORTED and "not found" in log:
        pytest.skip(log)
    assert rc == wos.WOS_OK, log
    assert nbytes > 10000


def test_grid_fields_call_the_grid_evaluators(wos):
    src = wos.jit_source(GRID_DESC())
    sig = src.split("case FLD_SIGMA")[1].split("case FLD_F")[0]
    alp = src.split("case FLD_ALPHA")[1].split("case FLD_PHI")[0]
    assert "grid_linear<DIM>(P.sigma, x)" in sig
    assert "grid_bspline<DIM>(P.alpha, x, &o.v, g, &o.lap, deriv)" in alp


def test_invalid_descriptions_are_refused(wos):
    bad = W.cube3d_problem()
    bad["alpha"] = W.const(-1.0)
    with pytest.raises(wos.WosError) as e:
        wos.jit_source(bad)
    assert e.value.code == wos.WOS_EINVAL
    bad = W.cube3d_problem()
    bad["dim"] = 4
    rc, log, _ = wos.jit_compile(bad)
    assert rc == wos.WOS_EINVAL and "dim" in log
    with pytest.raises(KeyError):
        wos.spec_flags("fp16")


def test_batch_source_shares_uniform_fields_and_compiles(wos):
    """A batch's specialised program: fields that every problem shares are generated code
    (grids read the walk's own problem's grid), a field that differs between problems calls
    the field interpreter; both precisions compile for sm_103a (no device)."""
    probs, pts, offs, walks = W.batch_problems(6, seed=5, max_points=8, min_points=4, min_walks=8, max_walks=16)
    src = wos.jit_batch_source(probs)
    assert "field_eval<DIM>(P, P." not in src                       # all six fields shared
    assert "grid_bspline<DIM>(P.alpha" in src and "grid_linear<DIM>(P.sigma" in src
    assert "R(0x1.921fb54442d18p+1)" in src                         # g = cos(pi x) y folded in
    for prec in ("fp32", "fp64"):
        rc, log, nbytes = wos.jit_batch_compile(probs, prec)
        assert rc == 0 and nbytes > 0, log
    # a g that differs between problems keeps the interpreter for g only
    other = [dict(p) for p in probs]
    other[3]["g"] = W.sst(W.term(2.0, (COS, 3.0, 0.0), (LIN, 1.0, 0.0)))
    src = wos.jit_batch_source(other)
    assert "case FLD_G:\n    return field_eval<DIM>(P, P.g" in src
    assert "field_eval<DIM>(P, P.alpha" not in src
    rc, log, nbytes = wos.jit_batch_compile(other, "fp32")
    assert rc == 0, log
    # sources that differ in being manufactured cannot share one kernel
    mixed = [W.rounded_box_problem(), W.noise_annulus_problem()]
    rc, log, _ = wos.jit_batch_compile(mixed, "fp32")
    assert rc == wos.WOS_EUNSUPPORTED and "manufactured" in log


def test_adjoint_kernels_compile_for_the_inverse_problem(wos):
    """WOS_SPEC_ADJOINT compiles the sigma and alpha replay kernels with the problem's fields
    (both precisions, sm_103a, no device)."""
    desc = W.inverse_problem(W.inverse_sigma_grid())
    for prec in ("fp32", "fp64"):
        rc, log, nbytes = wos.jit_compile(desc, prec, ("plain", "adjoint"))
        assert rc == 0 and nbytes > 0, log
