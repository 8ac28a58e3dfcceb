"""Python wrapper of the FP64 CPU oracle (``oracle.cpp``).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
CPU-baseline leg of the benchmark.  The product package never imports it.
The oracle is plain double-precision C++ compiled here with g++; it shares no
source, header or helper with the CUDA path.  Problems are the plain dicts of
the ``workloads`` module, packed into the oracle's own ctypes structs.

Functions with no independent pin: none (see ``tests/test_oracle_*.py``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_FIELD_KINDS = {"zero": 0, "const": 1, "sst": 2, "manufactured": 3, "grid_linear": 4,
                "grid_bspline": 5}
_DOM_KINDS = {"box": 0, "ball": 1, "annulus": 2, "rounded_box": 3, "mesh": 4, "csg": 5}


def build(force: bool = False) -> str:
    """Compile liboracle.so with g++ (-O2, OpenMP) if it is missing or stale."""
    with _lock:
        fresh = os.path.exists(_LIB_PATH) and all(
            os.path.getmtime(_LIB_PATH) >= os.path.getmtime(s) for s in (_SRC, _HDR))
        if fresh and not force:
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["g++", "-std=c++17", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True, cwd=_HERE)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


class Term(C.Structure):
    _fields_ = [("c", C.c_double), ("type", C.c_int32 * 3), ("k", C.c_double * 3),
                ("phi", C.c_double * 3)]


class Field(C.Structure):
    _fields_ = [("kind", C.c_int32), ("nterms", C.c_int32), ("terms", C.POINTER(Term)),
                ("value", C.c_double), ("res", C.c_int32 * 3), ("lo", C.c_double * 3),
                ("hi", C.c_double * 3), ("data", C.POINTER(C.c_float))]


class CsgNode(C.Structure):
    _fields_ = [("prim", C.c_int32), ("op", C.c_int32), ("p", C.c_double * 8)]


class Domain(C.Structure):
    _fields_ = [("kind", C.c_int32), ("p", C.c_double * 16), ("verts", C.POINTER(C.c_float)),
                ("nverts", C.c_int64), ("tris", C.POINTER(C.c_int32)), ("ntris", C.c_int64),
                ("bvh", C.c_void_p), ("csg", C.POINTER(CsgNode)), ("ncsg", C.c_int32), ("grid_res", C.c_int32)]


class Problem(C.Structure):
    _fields_ = [("dim", C.c_int32), ("domain", Domain), ("alpha", Field), ("phi", Field),
                ("sigma", Field), ("f", Field), ("g", Field), ("um", Field), ("omega", Field * 3),
                ("drift_bound", C.c_double)]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = C.CDLL(_LIB_PATH)
    dp = C.POINTER(C.c_double)
    pp = C.POINTER(Problem)
    lib.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
    lib.orc_uniform.argtypes = [C.c_uint32]
    lib.orc_uniform.restype = C.c_double
    lib.orc_bessel.argtypes = [C.c_double, dp]
    for n in ("orc_green_G", "orc_green_cdf", "orc_green_pdf", "orc_green_inv"):
        getattr(lib, n).argtypes = [C.c_int, C.c_double, C.c_double, C.c_double]
        getattr(lib, n).restype = C.c_double
    lib.orc_mix_radius.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, dp]
    lib.orc_mix_radius.restype = C.c_double
    for n in ("orc_green_norm", "orc_green_poisson"):
        getattr(lib, n).argtypes = [C.c_int, C.c_double, C.c_double]
        getattr(lib, n).restype = C.c_double
    lib.orc_field_eval.argtypes = [pp, C.POINTER(Field), dp, dp, dp, dp]
    lib.orc_coeffs.argtypes = [pp, dp, dp]
    lib.orc_distance.argtypes = [pp, dp, dp]
    lib.orc_distance.restype = C.c_double
    lib.orc_walk.argtypes = [pp, dp, C.c_uint32, C.c_uint32, C.c_uint64, C.c_double,
                             C.c_double, C.c_int64, C.POINTER(C.c_int64),
                             C.POINTER(C.c_int32)]
    lib.orc_walk.restype = C.c_double
    lib.orc_solve.argtypes = [pp, dp, C.c_int64, C.POINTER(C.c_int32), C.c_int32, C.c_uint64,
                              C.c_uint64, C.c_double, C.c_double, C.c_int64, dp, dp,
                              C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.c_int]
    lib.orc_walks.argtypes = [pp, dp, C.c_int64, C.c_int32, C.c_uint64, C.c_uint64,
                              C.c_double, C.c_double, C.c_int64, dp, C.POINTER(C.c_int64),
                              C.c_int]
    lib.orc_sigma_bar.argtypes = [pp, C.c_int, dp, dp, dp]
    lib.orc_walk_ww.argtypes = [pp, dp, C.c_uint32, C.c_uint32, C.c_uint64, C.c_double, C.c_double,
                                C.c_int64, C.c_double, C.c_double, C.c_int, C.POINTER(C.c_int64),
                                C.POINTER(C.c_int32)]
    lib.orc_walk_ww.restype = C.c_double
    lib.orc_solve_ww.argtypes = [pp, dp, C.c_int64, C.c_int32, C.c_uint64, C.c_uint64, C.c_double,
                                 C.c_double, C.c_int64, C.c_double, C.c_double, C.c_int, dp, dp,
                                 C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.c_int]
    lib.orc_green_dlog.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double]
    lib.orc_green_dlog.restype = C.c_double
    lib.orc_green_grad_ratios.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, dp]
    lib.orc_walk_grad.argtypes = [pp, dp, C.c_uint32, C.c_uint32, C.c_uint64, C.c_double, C.c_double,
                                  C.c_int64, dp, C.POINTER(C.c_int64), C.POINTER(C.c_int32)]
    lib.orc_walk_grad.restype = C.c_double
    lib.orc_walks_grad.argtypes = [pp, dp, C.c_int64, C.c_int32, C.c_uint64, C.c_uint64, C.c_double, C.c_double,
                                   C.c_int64, dp, dp, C.POINTER(C.c_int64), C.c_int]
    lib.orc_offcentre_G.argtypes = [C.c_int, C.c_double, C.c_double, dp, dp]
    lib.orc_offcentre_G.restype = C.c_double
    lib.orc_offcentre_P.argtypes = [C.c_int, C.c_double, C.c_double, dp, dp]
    lib.orc_offcentre_P.restype = C.c_double
    lib.orc_uniforms21.argtypes = [C.POINTER(C.c_uint32), dp]
    lib.orc_series_G.argtypes = [C.c_int, C.c_double, C.c_double, dp, dp, C.c_int]
    lib.orc_series_G.restype = C.c_double
    lib.orc_series_P.argtypes = [C.c_int, C.c_double, C.c_double, dp, dp, C.c_int]
    lib.orc_series_P.restype = C.c_double
    lib.orc_nf_h.argtypes = [C.c_int, C.c_double]
    lib.orc_nf_h.restype = C.c_double
    lib.orc_nf_free_radius.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double]
    lib.orc_nf_free_radius.restype = C.c_double
    lib.orc_walk_nf.argtypes = [pp, dp, C.c_uint32, C.c_uint32, C.c_uint64, C.c_double, C.c_double, C.c_int64,
                                C.c_int64, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                C.POINTER(C.c_int32)]
    lib.orc_walk_nf.restype = C.c_double
    lib.orc_walks_nf.argtypes = [pp, dp, C.c_int64, C.c_int32, C.c_uint64, C.c_uint64, C.c_double, C.c_double,
                                 C.c_int64, C.c_int64, C.c_int32, dp, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                 C.c_int]
    lib.orc_mesh_prepare.argtypes = [pp]
    lib.orc_mesh_release.argtypes = [pp]
    lib.orc_mesh_distance_brute.argtypes = [pp, dp, dp]
    lib.orc_mesh_distance_brute.restype = C.c_double
    _lib = lib
    return lib


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


_mesh_cache = {}


class _Packed:
    """A workloads problem dict packed into the oracle's structs (keeps arrays alive).
    A mesh domain gets the oracle's BVH, built once per mesh and kept for the process."""

    def __init__(self, prob):
        self.keep = []
        P = Problem()
        P.dim = prob["dim"]
        dom = prob["domain"]
        P.domain.kind = _DOM_KINDS[dom["kind"]]
        for i, v in enumerate(dom["p"]):
            P.domain.p[i] = v
        for name in ("alpha", "phi", "sigma", "f", "g", "um"):
            self._field(getattr(P, name), prob[name])
        for d, fd in enumerate(prob.get("omega", [{"kind": "zero"}] * 3)):
            self._field(P.omega[d], fd)
        P.drift_bound = float(prob.get("drift_bound", 0.0))
        if dom["kind"] == "csg":
            prims = {"sphere": 0, "box": 1, "capsule": 2, "torus": 3, "halfspace": 4}
            ops = {"union": 0, "intersect": 1, "subtract": 2}
            arr = (CsgNode * len(dom["nodes"]))()
            for i, (prim, op, prm) in enumerate(dom["nodes"]):
                arr[i].prim, arr[i].op = prims[prim], ops[op]
                for k, v in enumerate(prm):
                    arr[i].p[k] = v
            self.keep.append(arr)
            P.domain.csg = C.cast(arr, C.POINTER(CsgNode))
            P.domain.ncsg = len(dom["nodes"])
        if dom["kind"] == "mesh":
            key = (id(dom["verts"]), id(dom["tris"]), int(dom.get("grid_res", 0)))
            if key not in _mesh_cache:
                verts = np.ascontiguousarray(dom["verts"], dtype=np.float32)
                tris = np.ascontiguousarray(dom["tris"], dtype=np.int32)
                M = Problem()
                M.dim = 3
                M.domain.kind = 4
                M.domain.verts = verts.ctypes.data_as(C.POINTER(C.c_float))
                M.domain.nverts = len(verts)
                M.domain.tris = tris.ctypes.data_as(C.POINTER(C.c_int32))
                M.domain.ntris = len(tris)
                M.domain.grid_res = int(dom.get("grid_res", 0))
                if _load().orc_mesh_prepare(C.pointer(M)) != 0:
                    raise ValueError("orc_mesh_prepare failed")
                _mesh_cache[key] = (verts, tris, M, dom["verts"], dom["tris"])
            verts, tris, M, _, _ = _mesh_cache[key]
            P.domain.verts, P.domain.nverts = M.domain.verts, M.domain.nverts
            P.domain.tris, P.domain.ntris = M.domain.tris, M.domain.ntris
            P.domain.bvh = M.domain.bvh
            P.domain.grid_res = M.domain.grid_res
        self.P = P
        self.ptr = C.pointer(P)

    def _field(self, F, fd):
        F.kind = _FIELD_KINDS[fd["kind"]]
        F.value = fd.get("value", 0.0)
        if fd["kind"] == "sst":
            terms = (Term * max(1, len(fd["terms"])))()
            for i, t in enumerate(fd["terms"]):
                terms[i].c = t["c"]
                for d, (ty, k, ph) in enumerate(t["atoms"]):
                    terms[i].type[d] = ty
                    terms[i].k[d] = k
                    terms[i].phi[d] = ph
            self.keep.append(terms)
            F.nterms = len(fd["terms"])
            F.terms = C.cast(terms, C.POINTER(Term))
        if fd["kind"].startswith("grid"):
            data = np.ascontiguousarray(fd["data"], dtype=np.float32)
            self.keep.append(data)
            for d in range(3):
                F.res[d] = fd["res"][d] if d < len(fd["res"]) else 1
                F.lo[d] = fd["lo"][d] if d < len(fd["lo"]) else 0.0
                F.hi[d] = fd["hi"][d] if d < len(fd["hi"]) else 0.0
            F.data = data.ctypes.data_as(C.POINTER(C.c_float))


def pack(prob):
    return _Packed(prob)


# ---------------------------------------------------------------------------
# thin call wrappers
# ---------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    lib = _load()
    c = (C.c_uint32 * 4)(*[int(v) & 0xffffffff for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xffffffff for v in key])
    o = (C.c_uint32 * 4)()
    lib.orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def uniform(x):
    return _load().orc_uniform(int(x) & 0xffffffff)


def bessel(x):
    o = (C.c_double * 4)()
    _load().orc_bessel(float(x), o)
    return tuple(o)


def green_G(dim, R, sb, r):
    return _load().orc_green_G(dim, R, sb, r)


def green_norm(dim, R, sb):
    return _load().orc_green_norm(dim, R, sb)


def green_poisson(dim, R, sb):
    return _load().orc_green_poisson(dim, R, sb)


def green_cdf(dim, R, sb, r):
    return _load().orc_green_cdf(dim, R, sb, r)


def green_pdf(dim, R, sb, r):
    return _load().orc_green_pdf(dim, R, sb, r)


def green_inv(dim, R, sb, u):
    return _load().orc_green_inv(dim, R, sb, u)


def mix_radius(dim, R, sb, ur, lam):
    """(r, weight) of the mixture ball sample with G/|G| weight lam (reading R22)."""
    w = C.c_double()
    r = _load().orc_mix_radius(dim, R, sb, ur, lam, C.byref(w))
    return r, w.value


def field_eval(prob, name, x, packed=None):
    pk = packed or pack(prob)
    F = getattr(pk.P, name)
    xx = np.zeros(3, dtype=np.float64)
    xx[: len(x)] = x
    v = C.c_double()
    g = np.zeros(3)
    lap = C.c_double()
    rc = _load().orc_field_eval(pk.ptr, C.pointer(F), _dptr(xx), C.byref(v), _dptr(g),
                                C.byref(lap))
    if rc != 0:
        raise ValueError("field_eval failed")
    return v.value, g[: prob["dim"]].copy(), lap.value


def coeffs(prob, x, packed=None):
    """(gamma, sigma', f', f, alpha) at x."""
    pk = packed or pack(prob)
    xx = np.zeros(3)
    xx[: len(x)] = x
    out = np.zeros(5)
    _load().orc_coeffs(pk.ptr, _dptr(xx), _dptr(out))
    return tuple(out)


def mesh_distance_brute(prob, x, packed=None):
    pk = packed or pack(prob)
    xx = np.zeros(3)
    xx[: len(x)] = x
    xb = np.zeros(3)
    d = _load().orc_mesh_distance_brute(pk.ptr, _dptr(xx), _dptr(xb))
    return d, xb


def distance(prob, x, packed=None):
    pk = packed or pack(prob)
    xx = np.zeros(3)
    xx[: len(x)] = x
    xb = np.zeros(3)
    d = _load().orc_distance(pk.ptr, _dptr(xx), _dptr(xb))
    return d, xb[: prob["dim"]].copy()


def walk(prob, x0, point, walk_id, seed, eps, sigma_bar, max_steps=1 << 20, packed=None):
    pk = packed or pack(prob)
    xx = np.zeros(3)
    xx[: len(x0)] = x0
    k = C.c_int64()
    fl = C.c_int32()
    u = _load().orc_walk(pk.ptr, _dptr(xx), point, walk_id, seed, eps, sigma_bar, max_steps,
                         C.byref(k), C.byref(fl))
    return u, k.value, fl.value


def solve(prob, pts, walks, seed, eps, sigma_bar, walk_offset=0, max_steps=1 << 20,
          accum=None, nthreads=0):
    """Run walks and accumulate (sum, sumsq, count); returns (accum, stats).

    pts: SoA [dim][npts] array.  walks: int (uniform) or int32 array [npts].
    stats: {steps, walks, capped, nonfinite}.
    """
    lib = _load()
    pk = pack(prob)
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    npts = pts.shape[1]
    if accum is None:
        accum = (np.zeros(npts), np.zeros(npts), np.zeros(npts, dtype=np.int64))
    s1, s2, cnt = accum
    stats = np.zeros(4, dtype=np.int64)
    if np.isscalar(walks):
        wp, wu = None, int(walks)
    else:
        warr = np.ascontiguousarray(walks, dtype=np.int32)
        wp, wu = warr.ctypes.data_as(C.POINTER(C.c_int32)), 0
    rc = lib.orc_solve(pk.ptr, _dptr(pts), npts, wp, wu, walk_offset, seed, eps, sigma_bar,
                       max_steps, _dptr(s1), _dptr(s2),
                       cnt.ctypes.data_as(C.POINTER(C.c_int64)),
                       stats.ctypes.data_as(C.POINTER(C.c_int64)), nthreads)
    if rc != 0:
        raise ValueError("orc_solve rejected its inputs")
    return accum, {"steps": int(stats[0]), "walks": int(stats[1]), "capped": int(stats[2]),
                   "nonfinite": int(stats[3])}


def walks(prob, pts, walks_per_point, seed, eps, sigma_bar, walk_offset=0, max_steps=1 << 20,
          nthreads=0):
    """Per-walk estimates [npts, walks] and step counts."""
    lib = _load()
    pk = pack(prob)
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    npts = pts.shape[1]
    uh = np.zeros((npts, walks_per_point))
    st = np.zeros((npts, walks_per_point), dtype=np.int64)
    rc = lib.orc_walks(pk.ptr, _dptr(pts), npts, walks_per_point, walk_offset, seed, eps,
                       sigma_bar, max_steps, _dptr(uh),
                       st.ctypes.data_as(C.POINTER(C.c_int64)), nthreads)
    if rc != 0:
        raise ValueError("orc_walks rejected its inputs")
    return uh, st


def sigma_bar(prob, m=None):
    """(sigma_bar, min sigma', max sigma') on an m^dim lattice."""
    if m is None:
        m = 256 if prob["dim"] == 2 else 64
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    _load().orc_sigma_bar(pack(prob).ptr, m, C.byref(a), C.byref(b), C.byref(c))
    return a.value, b.value, c.value


def finalize(accum):
    """mean, unbiased variance of one walk, standard error of the mean."""
    s1, s2, n = accum
    n = n.astype(np.float64)
    mean = s1 / n
    var = (s2 - n * mean * mean) / np.maximum(n - 1, 1)
    var = np.maximum(var, 0.0)
    return mean, var, np.sqrt(var / n)


def walk_ww(prob, x0, point, walk_id, seed, eps, sigma_bar, ww_lo, ww_hi, depth=8, max_steps=1 << 20,
            packed=None):
    """One walk with the Sec. 6 weight window: (estimate, steps over all branches, flags)."""
    pk = packed or pack(prob)
    xx = np.zeros(3)
    xx[: len(x0)] = x0
    k = C.c_int64()
    fl = C.c_int32()
    u = _load().orc_walk_ww(pk.ptr, _dptr(xx), point, walk_id, seed, eps, sigma_bar, max_steps, ww_lo, ww_hi,
                            depth, C.byref(k), C.byref(fl))
    return u, k.value, fl.value


def solve_ww(prob, pts, walks, seed, eps, sigma_bar, ww_lo, ww_hi, depth=8, walk_offset=0, max_steps=1 << 20,
             nthreads=0):
    lib = _load()
    pk = pack(prob)
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    npts = pts.shape[1]
    acc = (np.zeros(npts), np.zeros(npts), np.zeros(npts, dtype=np.int64))
    stats = np.zeros(4, dtype=np.int64)
    rc = lib.orc_solve_ww(pk.ptr, _dptr(pts), npts, int(walks), walk_offset, seed, eps, sigma_bar, max_steps,
                          ww_lo, ww_hi, depth, _dptr(acc[0]), _dptr(acc[1]),
                          acc[2].ctypes.data_as(C.POINTER(C.c_int64)),
                          stats.ctypes.data_as(C.POINTER(C.c_int64)), nthreads)
    if rc != 0:
        raise ValueError("orc_solve_ww rejected its inputs")
    return acc, {"steps": int(stats[0]), "walks": int(stats[1]), "capped": int(stats[2]),
                 "nonfinite": int(stats[3])}


def green_grad_ratios(dim, R, sb, r):
    """(|grad_x G| / G at distance r, |grad_x P| / P) at the ball centre (Supplemental 1.3)."""
    o = (C.c_double * 2)()
    _load().orc_green_grad_ratios(dim, R, sb, r, o)
    return o[0], o[1]


def walk_grad(prob, x0, point, walk_id, seed, eps, sigma_bar, max_steps=1 << 20, packed=None):
    """(u estimate, grad u estimate, steps, flags) of one walk (Supplemental Sec. 2)."""
    pk = packed or pack(prob)
    xx = np.zeros(3)
    xx[: len(x0)] = x0
    g = np.zeros(3)
    k = C.c_int64()
    fl = C.c_int32()
    u = _load().orc_walk_grad(pk.ptr, _dptr(xx), point, walk_id, seed, eps, sigma_bar, max_steps, _dptr(g),
                              C.byref(k), C.byref(fl))
    return u, g[: prob["dim"]].copy(), k.value, fl.value


def walks_grad(prob, pts, walks_per_point, seed, eps, sigma_bar, walk_offset=0, max_steps=1 << 20, nthreads=0):
    """Per-walk u [npts, walks], grad u [dim, npts, walks] and step counts."""
    lib = _load()
    pk = pack(prob)
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    dim, npts = pts.shape
    uh = np.zeros((npts, walks_per_point))
    gh = np.zeros((dim, npts, walks_per_point))
    st = np.zeros((npts, walks_per_point), dtype=np.int64)
    rc = lib.orc_walks_grad(pk.ptr, _dptr(pts), npts, walks_per_point, walk_offset, seed, eps, sigma_bar,
                            max_steps, _dptr(uh), _dptr(gh), st.ctypes.data_as(C.POINTER(C.c_int64)), nthreads)
    if rc != 0:
        raise ValueError("orc_walks_grad rejected its inputs")
    return uh, gh, st


def solve_grad(prob, pts, walks, seed, eps, sigma_bar, walk_offset=0):
    """Per point: mean u, its standard error, mean grad u [npts, dim] and their standard errors."""
    uh, gh, _ = walks_grad(prob, pts, walks, seed, eps, sigma_bar, walk_offset)
    n = float(walks)
    gs = np.moveaxis(gh, 0, -1)  # [npts, walks, dim]
    return (uh.mean(1), uh.std(1, ddof=1) / np.sqrt(n), gs.mean(1), gs.std(1, ddof=1) / np.sqrt(n))


def offcentre_G(dim, R, sb, u, v):
    """Approximate off-centred G(x, y) on the ball (Supplemental 1.2), u = x - c, v = y - c."""
    uu, vv = np.zeros(3), np.zeros(3)
    uu[:dim], vv[:dim] = u, v
    return _load().orc_offcentre_G(dim, R, sb, _dptr(uu), _dptr(vv))


def offcentre_P(dim, R, sb, u, v):
    """Approximate off-centred P(x, z) on the sphere (Supplemental 1.2), u = x - c, v = z - c."""
    uu, vv = np.zeros(3), np.zeros(3)
    uu[:dim], vv[:dim] = u, v
    return _load().orc_offcentre_P(dim, R, sb, _dptr(uu), _dptr(vv))


def uniforms21(words):
    """The six 21-bit uniforms of a 3D step from one Philox block (four uint32 words)."""
    w = np.ascontiguousarray(words, dtype=np.uint32)
    out = np.zeros(6)
    _load().orc_uniforms21(w.ctypes.data_as(C.POINTER(C.c_uint32)), _dptr(out))
    return out


def series_G(dim, R, sb, u, v, nterms=0):
    """Off-centred G(x, y) on the ball as the series of Supplemental 1.2 (nterms = 0: to rounding)."""
    uu, vv = np.zeros(3), np.zeros(3)
    uu[:dim], vv[:dim] = u, v
    return _load().orc_series_G(dim, R, sb, _dptr(uu), _dptr(vv), nterms)


def series_P(dim, R, sb, u, v, nterms=0):
    """Off-centred P(x, z) on the sphere as the series of Supplemental 1.2 (nterms = 0: to rounding)."""
    uu, vv = np.zeros(3), np.zeros(3)
    uu[:dim], vv[:dim] = u, v
    return _load().orc_series_P(dim, R, sb, _dptr(uu), _dptr(vv), nterms)


def nf_h(dim, t):
    """h(t) of the series walk's in-ball sampling: 1 - e^{-t}(1 + t) (3D), 1 - t K_1(t) (2D)."""
    return _load().orc_nf_h(dim, t)


def nf_free_radius(dim, sb, rm, u):
    """Distance r in [0, rm] with h(sqrt(sb) r) = u h(sqrt(sb) rm)."""
    return _load().orc_nf_free_radius(dim, sb, rm, u)


def walk_nf(prob, x0, point, walk_id, seed, eps, sigma_bar, max_steps=1 << 20, max_inner=1 << 16, packed=None,
            series_terms=0):
    """(u estimate, outer steps, inner iterations, flags) of one next-flight walk; series_terms > 0
    takes the series G and P with that many terms instead of the printed approximations."""
    pk = packed or pack(prob)
    xx = np.zeros(3)
    xx[: len(x0)] = x0
    k, m, fl = C.c_int64(), C.c_int64(), C.c_int32()
    u = _load().orc_walk_nf(pk.ptr, _dptr(xx), point, walk_id, seed, eps, sigma_bar, max_steps, max_inner,
                            series_terms, C.byref(k), C.byref(m), C.byref(fl))
    return u, k.value, m.value, fl.value


def walks_nf(prob, pts, walks_per_point, seed, eps, sigma_bar, walk_offset=0, max_steps=1 << 20,
             max_inner=1 << 16, nthreads=0, series_terms=0):
    """Per-walk next-flight estimates [npts, walks], outer steps and inner iterations."""
    lib = _load()
    pk = pack(prob)
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    npts = pts.shape[1]
    uh = np.zeros((npts, walks_per_point))
    st = np.zeros((npts, walks_per_point), dtype=np.int64)
    inn = np.zeros((npts, walks_per_point), dtype=np.int64)
    rc = lib.orc_walks_nf(pk.ptr, _dptr(pts), npts, walks_per_point, walk_offset, seed, eps, sigma_bar, max_steps,
                          max_inner, series_terms, _dptr(uh), st.ctypes.data_as(C.POINTER(C.c_int64)),
                          inn.ctypes.data_as(C.POINTER(C.c_int64)), nthreads)
    if rc != 0:
        raise ValueError("orc_walks_nf rejected its inputs")
    return uh, st, inn


def green_dlog(dim, R, sb, r):
    """|G'(r)/G(r)| of the centred Green's function on a ball of radius R."""
    return _load().orc_green_dlog(dim, R, sb, r)
