"""The device's closest-point query on a triangle mesh, compiled here by g++ from the same
header (FP64): the 4-wide BVH built by the library's host builder, traversed by the
kernels' `mesh_query`, must return the oracle's brute-force distance (a loop over every
triangle) and a closest point on the mesh at that distance, with and without the walk's
upper bound, for points inside, outside and near the surface (Sec. 7.1)."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2201_13240_gb300", "csrc")

HARNESS = r"""
#include <vector>
#include "wos_mesh.h"
#include "wos_problem.cuh"
static std::vector<wos::MeshNode4> g_wide;
static std::vector<float> g_tris;
static wos::DevProblem<double> g_P;
extern "C" int build(const float* v, long long nv, const int* t, long long nt, int* nwide, int* wdepth) {
  std::vector<wos::MeshNode> bin;
  int depth = 0;
  if (wos::mesh_build_bvh(v, nv, t, nt, &bin, &g_tris, &depth) != 0) return -1;
  wos::mesh_collapse4(bin, &g_wide, wdepth);
  // the top levels first, as the library uploads them; the queries read those nodes through
  // the staged-node path (here the same host array)
  g_P.mesh_top = wos::mesh_top_first(&g_wide, wos::kMeshTopLevels);
  *nwide = (int)g_wide.size();
  g_P.mesh_nodes = reinterpret_cast<const float*>(g_wide.data());
  g_P.mesh_tris = g_tris.data();
  return 0;
}
extern "C" int top_count() { return g_P.mesh_top; }
extern "C" void query(const double* x, double bound2, double* out) {
  wos::MeshHit<double> h = wos::mesh_query<double, false>(g_P, x[0], x[1], x[2], bound2, nullptr, nullptr, 0, 1.0,
                                                          nullptr, nullptr, g_P.mesh_nodes);
  out[0] = h.d; out[1] = h.x; out[2] = h.y; out[3] = h.z;
}
extern "C" void query_tol(const double* x, double bound2, const double* pb, double tau, double* out) {
  wos::MeshVisits v = {0ull, 0ull, 0u};
  wos::MeshHit<double> h = wos::mesh_query<double, false>(g_P, x[0], x[1], x[2], bound2, nullptr, nullptr, 0, tau,
                                                          pb, &v, g_P.mesh_nodes);
  out[0] = h.d; out[1] = h.x; out[2] = h.y; out[3] = h.z;
  out[4] = (double)v.nodes; out[5] = (double)v.tris; out[6] = (double)v.exhausted;
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    d = tmp_path_factory.mktemp("bvh")
    cpp, so = d / "bvh.cpp", d / "bvh.so"
    cpp.write_text(HARNESS)
    subprocess.run(["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-Wno-unknown-pragmas", "-I", CSRC, "-o", str(so),
                    str(cpp), os.path.join(CSRC, "wos_mesh.cpp")], check=True)
    L = C.CDLL(str(so))
    L.build.argtypes = [C.c_void_p, C.c_longlong, C.c_void_p, C.c_longlong, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.query.argtypes = [C.c_void_p, C.c_double, C.c_void_p]
    L.query_tol.argtypes = [C.c_void_p, C.c_double, C.c_void_p, C.c_double, C.c_void_p]
    return L


@pytest.mark.parametrize("level", [2, 4])
def test_wide_bvh_query_equals_brute_force(lib, orc, level):
    desc = W.mesh_manufactured_problem(level=level)
    verts = np.ascontiguousarray(desc["domain"]["verts"], dtype=np.float32)
    tris = np.ascontiguousarray(desc["domain"]["tris"], dtype=np.int32)
    nw, wd = C.c_int(), C.c_int()
    assert lib.build(verts.ctypes.data, len(verts), tris.ctypes.data, len(tris), C.byref(nw), C.byref(wd)) == 0
    assert nw.value >= 1 and 1 <= wd.value <= 15
    assert 1 <= lib.top_count() <= min(21, nw.value)
    pk = orc.pack(desc)
    rng = np.random.default_rng(level)
    pts = np.concatenate([W.uniform_in_ball(3, 120, [0, 0, 0], 0.95, level, 0.0).T.astype(np.float64),
                          rng.uniform(-1.3, 1.3, size=(60, 3)),
                          # near the surface: vertices pushed in and out a little
                          verts[rng.choice(len(verts), 40)].astype(np.float64) * rng.uniform(0.98, 1.02, (40, 1))])
    out = np.zeros(4)
    for x in pts:
        dref, _ = orc.mesh_distance_brute(desc, x, packed=pk)
        for bound2 in (np.inf, (dref * 1.5) ** 2 + 1e-12, dref ** 2 * (1 + 1e-9), 0.0):
            lib.query(x.ctypes.data, float(bound2), out.ctypes.data)
            assert abs(out[0] - abs(dref)) <= 1e-9 * max(1.0, abs(dref)), (x, bound2, out[0], dref)
            # the returned point is on the mesh at that distance
            assert abs(np.linalg.norm(out[1:] - x) - out[0]) <= 1e-9


@pytest.mark.parametrize("tol", [0.05, 0.1, 0.3])
def test_tolerance_query_certifies_a_radius(lib, orc, tol):
    """With tolerance tol the query returns r with (1 - tol) d <= r <= d (d the brute-force
    distance), a point on the mesh, and opens fewer nodes than the exact query; with the
    walk's bound from a boundary point pb it is still certified, and when nothing lies
    inside the bound pb itself is returned."""
    desc = W.mesh_manufactured_problem(level=4)
    verts = np.ascontiguousarray(desc["domain"]["verts"], dtype=np.float32)
    tris = np.ascontiguousarray(desc["domain"]["tris"], dtype=np.int32)
    nw, wd = C.c_int(), C.c_int()
    assert lib.build(verts.ctypes.data, len(verts), tris.ctypes.data, len(tris), C.byref(nw), C.byref(wd)) == 0
    pk = orc.pack(desc)
    tau = (1.0 - tol) ** 2
    rng = np.random.default_rng(7)
    pts = np.ascontiguousarray(W.uniform_in_ball(3, 80, [0, 0, 0], 0.88, 9, 0.0).T, dtype=np.float64)
    out, ex = np.zeros(7), np.zeros(7)
    nodes_tol = nodes_ex = tris_tol = tris_ex = 0.0
    for x in pts:
        dref, _ = orc.mesh_distance_brute(desc, x, packed=pk)
        lib.query_tol(x.ctypes.data, np.inf, None, 1.0, ex.ctypes.data)
        lib.query_tol(x.ctypes.data, np.inf, None, tau, out.ctypes.data)
        assert (1.0 - tol) * dref * (1 - 1e-12) <= out[0] <= dref * (1 + 1e-12), (x, out[0], dref)
        assert abs(orc.mesh_distance_brute(desc, out[1:4], packed=pk)[0]) <= 1e-9  # on the mesh
        assert out[6] == 0
        nodes_tol += out[4]
        nodes_ex += ex[4]
        tris_tol += out[5]
        tris_ex += ex[5]
        # a bound from another boundary point, as the walk passes the previous step's
        y = x + 0.3 * dref * rng.normal(size=3) / np.sqrt(3.0)
        lib.query_tol(y.ctypes.data, np.inf, None, 1.0, ex.ctypes.data)
        pb = np.ascontiguousarray(ex[1:4])
        b2 = float(np.sum((x - pb) ** 2))
        lib.query_tol(x.ctypes.data, b2, pb.ctypes.data, tau, out.ctypes.data)
        assert (1.0 - tol) * dref * (1 - 1e-12) <= out[0] <= dref * (1 + 1e-12)
        assert abs(orc.mesh_distance_brute(desc, out[1:4], packed=pk)[0]) <= 1e-9
    assert nodes_tol < nodes_ex and tris_tol < tris_ex
    # a bound at exactly the distance (pb the closest point): the result is pb or a point
    # as near, with a certified radius
    x = pts[0]
    dref, _ = orc.mesh_distance_brute(desc, x, packed=pk)
    lib.query_tol(x.ctypes.data, np.inf, None, 1.0, ex.ctypes.data)
    pb = np.ascontiguousarray(ex[1:4])
    lib.query_tol(x.ctypes.data, float(np.sum((x - pb) ** 2)), pb.ctypes.data, tau, out.ctypes.data)
    assert (1.0 - tol) * dref * (1 - 1e-12) <= out[0] <= dref * (1 + 1e-12)
    assert np.linalg.norm(out[1:4] - x) == pytest.approx(dref, abs=1e-9)
