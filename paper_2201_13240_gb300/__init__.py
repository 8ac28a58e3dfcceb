"""GB300 delta-tracking walk on spheres for variable-coefficient elliptic PDEs.

Thin Python binding of the C interface in ``include/wos.h`` (the library
``libwos.so`` built in-tree by ``paper_2201_13240_gb300.build``).  Every step of
a solve runs in the library's CUDA kernels; this module only marshals
arguments.  PyTorch provides device memory and the current stream.

It estimates the solution of Sawhney et al. 2022, Sec. 3 eq. 1,
``div(alpha grad u) + omega.grad u - sigma u = -f`` (u = g on the boundary,
omega = alpha grad Phi) with the delta-tracking walk on spheres (Sec. 5.1).
Problems are the plain dicts produced by the ``workloads`` module.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwos.so")

WOS_OK, WOS_EINVAL, WOS_ENOMEM, WOS_ECUDA, WOS_ETIMEOUT, WOS_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
WOS_FP32, WOS_FP64 = 0, 1
STAT_STEPS, STAT_WALKS, STAT_CAPPED, STAT_NONFINITE, STAT_OUTSIDE, STAT_INNER = range(6)
STAT_MESH_NODES, STAT_MESH_TRIS, STAT_EXHAUSTED = 6, 7, 8
STATS_WORDS = 9
WOS_SPEC_FP32, WOS_SPEC_FP64, WOS_SPEC_PLAIN, WOS_SPEC_WINDOW, WOS_SPEC_GRAD = 0x1, 0x2, 0x10, 0x20, 0x40
WOS_SPEC_ADJOINT = 0x80
_FIELD_KINDS = {"zero": 0, "const": 1, "sst": 2, "manufactured": 3, "grid_linear": 4, "grid_bspline": 5}
_DOM_KINDS = {"box": 0, "ball": 1, "annulus": 2, "rounded_box": 3, "mesh": 4, "csg": 5}
_CSG_PRIMS = {"sphere": 0, "box": 1, "capsule": 2, "torus": 3, "halfspace": 4}
_CSG_OPS = {"union": 0, "intersect": 1, "subtract": 2}


class WosError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"wos error {code}: {msg}")
        self.code = code


class Term(C.Structure):
    _fields_ = [("c", C.c_double), ("type", C.c_int32 * 3), ("k", C.c_double * 3), ("phi", C.c_double * 3)]


class FieldDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("nterms", C.c_int32), ("terms", C.POINTER(Term)), ("value", C.c_double),
                ("res", C.c_int32 * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("data", C.c_void_p)]


class CsgNode(C.Structure):
    _fields_ = [("prim", C.c_int32), ("op", C.c_int32), ("p", C.c_double * 8)]


class DomainDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("p", C.c_double * 16), ("verts", C.c_void_p), ("nverts", C.c_int64),
                ("tris", C.c_void_p), ("ntris", C.c_int64), ("csg", C.c_void_p), ("ncsg", C.c_int32),
                ("mesh_grid_res", C.c_int32), ("mesh_tol", C.c_double)]


class ViewDesc(C.Structure):
    _fields_ = [("eye", C.c_double * 3), ("look", C.c_double * 3), ("up", C.c_double * 3),
                ("fov_y_deg", C.c_double), ("plane_origin", C.c_double * 3), ("plane_u", C.c_double * 3),
                ("plane_v", C.c_double * 3), ("slice_nu", C.c_int32), ("slice_nv", C.c_int32),
                ("width", C.c_int32), ("height", C.c_int32), ("value_lo", C.c_double), ("value_hi", C.c_double)]


def view(plane_origin, plane_u, plane_v, slice_nu, slice_nv, width, height, value_range, eye=(0, 0, 5),
         look=(0, 0, 0), up=(0, 1, 0), fov_y_deg=40.0):
    """A wos_view: slice rectangle plane_origin + a plane_u + b plane_v, its slice grid, the
    image size, the colour range and (3D) a pinhole camera."""
    v = ViewDesc()
    for name, val in (("eye", eye), ("look", look), ("up", up), ("plane_origin", plane_origin),
                      ("plane_u", plane_u), ("plane_v", plane_v)):
        arr = getattr(v, name)
        for k in range(3):
            arr[k] = float(val[k]) if k < len(val) else 0.0
    v.fov_y_deg = float(fov_y_deg)
    v.slice_nu, v.slice_nv = int(slice_nu), int(slice_nv)
    v.width, v.height = int(width), int(height)
    v.value_lo, v.value_hi = float(value_range[0]), float(value_range[1])
    return v


class ProblemDesc(C.Structure):
    _fields_ = [("dim", C.c_int32), ("domain", DomainDesc), ("alpha", FieldDesc), ("phi", FieldDesc),
                ("sigma", FieldDesc), ("f", FieldDesc), ("g", FieldDesc), ("um", FieldDesc),
                ("omega", FieldDesc * 3), ("drift_bound", C.c_double)]


class Schedule(C.Structure):
    _fields_ = [("chunk", C.c_int32), ("blocks_per_sm", C.c_int32), ("regs_variant", C.c_int32),
                ("reserved", C.c_int32)]

    def as_dict(self):
        return {"chunk": self.chunk, "blocks_per_sm": self.blocks_per_sm, "regs_variant": self.regs_variant}


class Params(C.Structure):
    _fields_ = [("eps", C.c_double), ("sigma_bar", C.c_double), ("seed", C.c_uint64), ("walk_offset", C.c_uint64),
                ("max_steps", C.c_int64), ("precision", C.c_int32), ("ww_depth", C.c_int32), ("ww_lo", C.c_double),
                ("ww_hi", C.c_double)]


_lib = None


def load():
    """Load libwos.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2201_13240_gb300.build`")
    lib = C.CDLL(LIB_PATH)
    vp, i64, i32, dp = C.c_void_p, C.c_int64, C.c_int32, C.POINTER(C.c_double)
    lib.wos_create.argtypes = [C.POINTER(vp), C.c_int]
    lib.wos_destroy.argtypes = [vp]
    lib.wos_last_error.argtypes = [vp]
    lib.wos_last_error.restype = C.c_char_p
    lib.wos_version.restype = C.c_char_p
    lib.wos_problem_create.argtypes = [vp, C.POINTER(ProblemDesc), C.POINTER(vp)]
    lib.wos_problem_destroy.argtypes = [vp]
    lib.wos_sigma_bar.argtypes = [vp, vp, i32, dp, dp, dp, vp]
    lib.wos_solve.argtypes = [vp, vp, vp, i64, vp, i32, C.POINTER(Params), vp, vp, vp, vp, vp]
    lib.wos_walk_estimates.argtypes = [vp, vp, vp, i64, i32, C.POINTER(Params), vp, vp, vp, vp]
    lib.wos_finalize.argtypes = [vp, vp, vp, vp, i64, vp, vp, vp, vp]
    lib.wos_slice_points.argtypes = [vp, vp, C.POINTER(ViewDesc), vp, vp]
    lib.wos_render_slice.argtypes = [vp, vp, C.POINTER(ViewDesc), vp, vp, vp, vp, vp, vp]
    lib.wos_solve_nf.argtypes = [vp, vp, vp, i64, vp, i32, C.POINTER(Params), i64, i32, vp, vp, vp, vp, vp]
    lib.wos_walk_estimates_nf.argtypes = [vp, vp, vp, i64, i32, C.POINTER(Params), i64, i32, vp, vp, vp, vp]
    lib.wos_solve_grad.argtypes = [vp, vp, vp, i64, vp, i32, C.POINTER(Params), vp, vp, vp, vp, vp, vp, vp]
    lib.wos_walk_grad_estimates.argtypes = [vp, vp, vp, i64, i32, C.POINTER(Params), vp, vp, vp, vp, vp]
    lib.wos_solve_host.argtypes = [vp, vp, vp, i64, i32, C.POINTER(Params), vp, vp, vp, vp, vp]
    lib.wos_adjoint_sigma.argtypes = [vp, vp, vp, i64, i32, C.POINTER(Params), vp, vp, vp, vp]
    lib.wos_adjoint_alpha.argtypes = [vp, vp, vp, i64, i32, C.POINTER(Params), vp, vp, vp, vp]
    lib.wos_batch_create.argtypes = [vp, C.POINTER(vp), i32, vp, vp, C.POINTER(vp)]
    lib.wos_batch_destroy.argtypes = [vp]
    lib.wos_solve_batch.argtypes = [vp, vp, vp, vp, i32, C.POINTER(Params), vp, vp, vp, vp, vp]
    lib.wos_batch_set_schedule.argtypes = [vp, C.POINTER(Schedule)]
    lib.wos_batch_get_schedule.argtypes = [vp, C.POINTER(Schedule)]
    lib.wos_batch_autotune.argtypes = [vp, vp, vp, vp, i32, C.POINTER(Params), i32, C.POINTER(Schedule), dp, dp, vp]
    lib.wos_problem_specialize.argtypes = [vp, vp, i32]
    lib.wos_problem_specialized.argtypes = [vp, C.POINTER(i32)]
    lib.wos_jit_source.argtypes = [C.POINTER(ProblemDesc), C.c_char_p, i64, C.POINTER(i64)]
    lib.wos_jit_compile.argtypes = [C.POINTER(ProblemDesc), i32, C.c_char_p, i64, C.POINTER(i64)]
    # problem-statement calls: domain and field handles, assembly, mean / variance solves
    lib.wos_domain_box.argtypes = [vp, i32, dp, dp, C.POINTER(vp)]
    lib.wos_domain_sdf.argtypes = [vp, i32, i32, dp, C.POINTER(vp)]
    lib.wos_domain_mesh.argtypes = [vp, vp, i64, vp, i64, C.POINTER(vp)]
    lib.wos_domain_destroy.argtypes = [vp]
    lib.wos_field_analytic.argtypes = [vp, i32, dp, i32, C.POINTER(vp)]
    lib.wos_field_grid.argtypes = [vp, i32, C.POINTER(i32), dp, dp, vp, i32, C.POINTER(vp)]
    lib.wos_field_destroy.argtypes = [vp]
    lib.wos_problem_assemble.argtypes = [vp, vp, vp, vp, vp, vp, vp, C.POINTER(vp)]
    lib.wos_problem_sigma_bar.argtypes = [vp, vp, dp, dp, dp]
    lib.wos_solve_mean.argtypes = [vp, vp, vp, i64, vp, i32, C.POINTER(Params), vp, vp, vp, vp, vp]
    lib.wos_solve_batched.argtypes = [vp, C.POINTER(vp), i32, vp, vp, vp, vp, i32, C.POINTER(Params), vp, vp, vp,
                                      vp, vp]
    lib.wos_adjoint.argtypes = [vp, vp, vp, i64, i32, C.POINTER(Params), vp, vp, vp, vp, vp]
    lib.wos_measure_peak.argtypes = [vp, i32, vp, i64, dp, dp, vp]
    lib.wos_batch_specialize.argtypes = [vp, vp, i32]
    lib.wos_batch_specialized.argtypes = [vp, C.POINTER(i32), C.POINTER(i32)]
    lib.wos_jit_batch_source.argtypes = [C.POINTER(ProblemDesc), i32, C.c_char_p, i64, C.POINTER(i64)]
    lib.wos_jit_batch_compile.argtypes = [C.POINTER(ProblemDesc), i32, i32, C.c_char_p, i64, C.POINTER(i64)]
    _lib = lib
    return lib


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _points(pts, dim, device):
    """Validate a device point array [dim, npts] and return it as a contiguous float32 tensor."""
    import torch
    if not isinstance(pts, torch.Tensor) or not pts.is_cuda:
        raise TypeError("points must be a CUDA tensor of shape [dim, npts]")
    if pts.dim() != 2 or pts.shape[0] != dim:
        raise ValueError(f"points must have shape [{dim}, npts], got {tuple(pts.shape)}")
    if pts.dtype != torch.float32:
        raise TypeError("points must be float32")
    if pts.device.index != device:
        raise ValueError(f"points live on {pts.device}, the context on cuda:{device}")
    return pts.contiguous()


def params(eps, sigma_bar, seed=0, walk_offset=0, max_steps=1 << 20, precision="fp32", window=None):
    """window: None, or (lo, hi) or (lo, hi, depth) for the Sec. 6 weight window."""
    p = Params()
    if window is not None:
        p.ww_lo, p.ww_hi = float(window[0]), float(window[1])
        p.ww_depth = int(window[2]) if len(window) > 2 else 8
    p.eps = float(eps)
    p.sigma_bar = float(sigma_bar)
    p.seed = int(seed)
    p.walk_offset = int(walk_offset)
    p.max_steps = int(max_steps)
    p.precision = WOS_FP64 if precision in ("fp64", WOS_FP64) else WOS_FP32
    return p


def describe(desc, device=None):
    """The C description of a problem dict: (ProblemDesc, objects to keep alive, sigma grid
    address, alpha grid address).  Grid data goes to cuda:device, or stays in host memory when
    device is None (descriptions for wos_jit_source / wos_jit_compile, which never read it)."""
    D = ProblemDesc()
    keep = []
    ptrs = {"sigma": 0, "alpha": 0}
    D.dim = desc["dim"]
    D.drift_bound = float(desc.get("drift_bound", 0.0))
    D.domain.kind = _DOM_KINDS[desc["domain"]["kind"]]
    for i, v in enumerate(desc["domain"]["p"]):
        D.domain.p[i] = v
    if desc["domain"]["kind"] == "mesh":
        verts = np.ascontiguousarray(desc["domain"]["verts"], dtype=np.float32)
        tris = np.ascontiguousarray(desc["domain"]["tris"], dtype=np.int32)
        keep += [verts, tris]
        D.domain.verts, D.domain.nverts = verts.ctypes.data, len(verts)
        D.domain.tris, D.domain.ntris = tris.ctypes.data, len(tris)
        D.domain.mesh_grid_res = int(desc["domain"].get("grid_res", 0))
        D.domain.mesh_tol = float(desc["domain"].get("tol", 0.0))
    if desc["domain"]["kind"] == "csg":
        nodes = desc["domain"]["nodes"]
        arr = (CsgNode * max(1, len(nodes)))()
        for i, (prim, op, prm) in enumerate(nodes):
            arr[i].prim = _CSG_PRIMS[prim]
            arr[i].op = _CSG_OPS[op]
            for k, v in enumerate(prm):
                arr[i].p[k] = v
        keep.append(arr)
        D.domain.csg = C.cast(arr, C.c_void_p)
        D.domain.ncsg = len(nodes)
    omega = list(desc.get("omega", []))
    omega += [{"kind": "zero"}] * (3 - len(omega))
    slots = [(n, desc[n], getattr(D, n)) for n in ("alpha", "phi", "sigma", "f", "g", "um")]
    slots += [(f"omega{k}", omega[k], D.omega[k]) for k in range(3)]
    for name, fd, F in slots:
        F.kind = _FIELD_KINDS[fd["kind"]]
        F.value = fd.get("value", 0.0)
        if fd["kind"] == "sst":
            terms = (Term * max(1, len(fd["terms"])))()
            for i, t in enumerate(fd["terms"]):
                terms[i].c = t["c"]
                for d, (ty, k, ph) in enumerate(t["atoms"]):
                    terms[i].type[d], terms[i].k[d], terms[i].phi[d] = ty, k, ph
            keep.append(terms)
            F.nterms = len(fd["terms"])
            F.terms = C.cast(terms, C.POINTER(Term))
        if fd["kind"].startswith("grid"):
            data = fd["data"]
            if device is None:
                if not isinstance(data, np.ndarray):
                    data = data.detach().cpu().numpy()
                data = np.ascontiguousarray(data, dtype=np.float32)
                addr = data.ctypes.data
            else:
                import torch
                if not isinstance(data, torch.Tensor):
                    data = torch.as_tensor(np.ascontiguousarray(data, dtype=np.float32))
                data = data.to(device=f"cuda:{device}", dtype=torch.float32).contiguous()
                addr = data.data_ptr()
            keep.append(data)
            for d in range(3):
                F.res[d] = fd["res"][d] if d < len(fd["res"]) else 1
                F.lo[d] = fd["lo"][d] if d < len(fd["lo"]) else 0.0
                F.hi[d] = fd["hi"][d] if d < len(fd["hi"]) else 0.0
            F.data = addr
            if name in ptrs:
                ptrs[name] = addr
    return D, keep, ptrs["sigma"], ptrs["alpha"]


_SPEC_PRECISION = {"fp32": WOS_SPEC_FP32, "fp64": WOS_SPEC_FP64}
_SPEC_VARIANT = {"plain": WOS_SPEC_PLAIN, "window": WOS_SPEC_WINDOW, "grad": WOS_SPEC_GRAD,
                 "adjoint": WOS_SPEC_ADJOINT}


def spec_flags(precisions=("fp32",), variants=("plain",)):
    f = 0
    for p in ([precisions] if isinstance(precisions, str) else precisions):
        f |= _SPEC_PRECISION[p]
    for v in ([variants] if isinstance(variants, str) else variants):
        f |= _SPEC_VARIANT[v]
    return f


def jit_source(desc):
    """The generated program of the problem-specialised walk kernel (host only)."""
    lib = load()
    D, keep, _, _ = describe(desc)
    n = C.c_int64(0)
    rc = lib.wos_jit_source(C.byref(D), None, 0, C.byref(n))
    if rc != WOS_OK:
        buf = C.create_string_buffer(512)
        lib.wos_jit_source(C.byref(D), buf, 512, None)
        raise WosError(rc, buf.value.decode(errors="replace"))
    buf = C.create_string_buffer(n.value + 1)
    lib.wos_jit_source(C.byref(D), buf, n.value + 1, C.byref(n))
    return buf.value.decode()


def jit_compile(desc, precision="fp32", variants=("plain",)):
    """NVRTC compile of the specialised kernels (no device): (status, log, cubin bytes)."""
    lib = load()
    D, keep, _, _ = describe(desc)
    log = C.create_string_buffer(1 << 16)
    nbytes = C.c_int64(0)
    rc = lib.wos_jit_compile(C.byref(D), spec_flags(precision, variants), log, 1 << 16, C.byref(nbytes))
    return rc, log.value.decode(errors="replace"), nbytes.value


def _describe_many(descs):
    arr = (ProblemDesc * len(descs))()
    keep = []
    for i, d in enumerate(descs):
        D, k, _, _ = describe(d)
        arr[i] = D
        keep.append(k)
    return arr, keep


def jit_batch_source(descs):
    """The generated program of wos_batch_specialize for a list of problem dicts (host only)."""
    lib = load()
    arr, keep = _describe_many(descs)
    n = C.c_int64(0)
    rc = lib.wos_jit_batch_source(arr, len(descs), None, 0, C.byref(n))
    if rc != WOS_OK:
        buf = C.create_string_buffer(512)
        lib.wos_jit_batch_source(arr, len(descs), buf, 512, None)
        raise WosError(rc, buf.value.decode(errors="replace"))
    buf = C.create_string_buffer(n.value + 1)
    lib.wos_jit_batch_source(arr, len(descs), buf, n.value + 1, C.byref(n))
    return buf.value.decode()


def jit_batch_compile(descs, precision="fp32"):
    """NVRTC compile of a batch's specialised kernels (no device): (status, log, cubin bytes)."""
    lib = load()
    arr, keep = _describe_many(descs)
    log = C.create_string_buffer(1 << 16)
    nbytes = C.c_int64(0)
    rc = lib.wos_jit_batch_compile(arr, len(descs), spec_flags(precision), log, 1 << 16, C.byref(nbytes))
    return rc, log.value.decode(errors="replace"), nbytes.value


class Problem:
    """A problem uploaded to the device (owns the library handle)."""

    def __init__(self, ctx, desc):
        self.ctx = ctx
        self.dim = desc["dim"]
        D, self._keep, self._sigma_ptr, self._alpha_ptr = describe(desc, ctx.device)
        h = C.c_void_p()
        ctx._check(ctx.lib.wos_problem_create(ctx.handle, C.byref(D), C.byref(h)))
        self.handle = h
        ctx._children.add(self)

    def specialize(self, precisions=("fp32",), variants=("plain",)):
        """Compile and load the walk kernels specialised to this problem's fields (NVRTC;
        blocks for the compilation).  Later solves of the matching precision and variant
        launch them."""
        self.ctx._check(self.ctx.lib.wos_problem_specialize(self.ctx.handle, self.handle,
                                                            spec_flags(precisions, variants)))
        return self

    def specialized(self):
        """WOS_SPEC_* bits of the loaded specialised kernels."""
        f = C.c_int32(0)
        rc = self.ctx.lib.wos_problem_specialized(self.handle, C.byref(f))
        if rc != WOS_OK:
            raise WosError(rc, "wos_problem_specialized")
        return f.value

    def sigma_data_ptr(self):
        """Device address of the sigma grid the problem reads (0 if sigma is not a grid)."""
        return self._sigma_ptr

    def alpha_data_ptr(self):
        """Device address of the alpha grid the problem reads (0 if alpha is not a grid)."""
        return self._alpha_ptr

    def close(self):
        if getattr(self, "handle", None):
            self.ctx.lib.wos_problem_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _dvec(vals):
    arr = (C.c_double * max(1, len(vals)))(*[float(v) for v in vals])
    return arr


def pack_terms(terms):
    """Separable terms (workloads format) as the 10-double packing of wos_field_analytic."""
    out = []
    for t in terms:
        atoms = list(t["atoms"]) + [(0, 0.0, 0.0)] * (3 - len(t["atoms"]))
        out += [t["c"]] + [a[0] for a in atoms] + [a[1] for a in atoms] + [a[2] for a in atoms]
    return out


class Handle:
    """A domain or field handle of the problem-statement calls (owns it)."""

    def __init__(self, lib, h, destroy, keep=None, dim=0):
        self.lib, self.handle, self._destroy, self._keep, self.dim = lib, h, destroy, keep, dim

    def close(self):
        if getattr(self, "handle", None):
            self._destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent problems solved by one launch (owns the library handle)."""

    def __init__(self, ctx, problems, pt_offsets, sigma_bars):
        self.ctx = ctx
        self.problems = list(problems)  # keep the problems (and their grid tensors) alive
        self.dim = self.problems[0].dim
        offs = np.ascontiguousarray(pt_offsets, dtype=np.int64)
        sbs = np.ascontiguousarray(sigma_bars, dtype=np.float64)
        if len(offs) != len(self.problems) + 1 or len(sbs) != len(self.problems):
            raise ValueError("need nprob + 1 offsets and nprob sigma_bars")
        self.npts = int(offs[-1])
        handles = (C.c_void_p * len(self.problems))(*[p.handle.value for p in self.problems])
        h = C.c_void_p()
        ctx._check(ctx.lib.wos_batch_create(ctx.handle, handles, len(self.problems), offs.ctypes.data,
                                            sbs.ctypes.data, C.byref(h)))
        self.handle = h
        ctx._children.add(self)

    def schedule(self):
        """The batch's launch schedule (dict: chunk, blocks_per_sm, regs_variant)."""
        sc = Schedule()
        rc = self.ctx.lib.wos_batch_get_schedule(self.handle, C.byref(sc))
        if rc != WOS_OK:
            raise WosError(rc, "wos_batch_get_schedule")
        return sc.as_dict()

    def specialize(self, precisions=("fp32",)):
        """Compile the batched walk kernel with the fields every problem shares as code
        (NVRTC; blocks for the compilation); later solves launch it."""
        self.ctx._check(self.ctx.lib.wos_batch_specialize(self.ctx.handle, self.handle, spec_flags(precisions)))
        return self

    def specialized(self):
        """(WOS_SPEC_* bits of the loaded kernels, bits of the fields all problems share)."""
        f, u = C.c_int32(0), C.c_int32(0)
        rc = self.ctx.lib.wos_batch_specialized(self.handle, C.byref(f), C.byref(u))
        if rc != WOS_OK:
            raise WosError(rc, "wos_batch_specialized")
        return f.value, u.value

    def set_schedule(self, chunk=0, blocks_per_sm=0, regs_variant=0):
        sc = Schedule(int(chunk), int(blocks_per_sm), int(regs_variant), 0)
        rc = self.ctx.lib.wos_batch_set_schedule(self.handle, C.byref(sc))
        if rc != WOS_OK:
            raise WosError(rc, "invalid schedule")

    def close(self):
        if getattr(self, "handle", None):
            self.ctx.lib.wos_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """A library context on one CUDA device."""

    def __init__(self, device=0):
        import torch
        self.lib = load()
        self.device = int(device)
        torch.cuda.init()
        h = C.c_void_p()
        rc = self.lib.wos_create(C.byref(h), self.device)
        if rc != WOS_OK:
            raise WosError(rc, "wos_create failed")
        self.handle = h
        import weakref
        self._children = weakref.WeakSet()  # problems and batches: released before the context

    def _check(self, rc):
        if rc != WOS_OK:
            raise WosError(rc, self.lib.wos_last_error(self.handle).decode())

    def close(self):
        if getattr(self, "handle", None):
            for c in list(getattr(self, "_children", ())):
                c.close()
            self.lib.wos_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- measurement utilities ----
    def measure_peak(self, unit, l2_bytes=32 << 20, stream=None):
        """Measured rate of 'fp32_lanes' (lane ops/s), 'mufu' (ops/s) or 'l2_read' (bytes/s, from
        a zero-filled l2_bytes buffer); returns (rate, ms per launch)."""
        import torch
        which = {"fp32_lanes": 0, "mufu": 1, "l2_read": 2}[unit]
        buf = torch.zeros(l2_bytes // 4, dtype=torch.float32, device=f"cuda:{self.device}") if which == 2 else None
        r, ms = C.c_double(), C.c_double()
        self._check(self.lib.wos_measure_peak(self.handle, which, _ptr(buf), l2_bytes if buf is not None else 0,
                                              C.byref(r), C.byref(ms), _stream(stream)))
        return r.value, ms.value

    # ---- problem-statement calls (handles) ----
    def _handle(self, rc, h, destroy, keep=None, dim=0):
        self._check(rc)
        return Handle(self.lib, h, destroy, keep, dim)

    def domain_box(self, dim, lo, hi):
        h = C.c_void_p()
        return self._handle(self.lib.wos_domain_box(self.handle, int(dim), _dvec(lo), _dvec(hi), C.byref(h)), h,
                            self.lib.wos_domain_destroy, dim=dim)

    def domain_sdf(self, dim, kind, p):
        """kind: 'ball', 'annulus' or 'rounded_box'; p as wos_domain_desc.p for that kind."""
        h = C.c_void_p()
        return self._handle(self.lib.wos_domain_sdf(self.handle, int(dim), _DOM_KINDS[kind], _dvec(p), C.byref(h)),
                            h, self.lib.wos_domain_destroy, dim=dim)

    def domain_mesh(self, verts, tris):
        """verts: CUDA float32 [nv, 3], tris: CUDA int32 [nt, 3] (copied by the call)."""
        verts, tris = verts.contiguous(), tris.contiguous()
        h = C.c_void_p()
        return self._handle(self.lib.wos_domain_mesh(self.handle, _ptr(verts), verts.shape[0], _ptr(tris),
                                                     tris.shape[0], C.byref(h)), h, self.lib.wos_domain_destroy,
                            dim=3)

    def field_analytic(self, family, p=()):
        """family: 'zero', 'const' (p = [value]), 'sst' or 'manufactured' (p = pack_terms(...))."""
        h = C.c_void_p()
        return self._handle(self.lib.wos_field_analytic(self.handle, _FIELD_KINDS[family], _dvec(p), len(p),
                                                        C.byref(h)), h, self.lib.wos_field_destroy)

    def field_grid(self, dim, res, lo, hi, data, interp="grid_linear"):
        """data: CUDA float32 node values (x fastest), kept alive by the handle."""
        data = data.contiguous()
        r = (C.c_int32 * 3)(*[int(v) for v in list(res) + [1] * (3 - len(res))])
        h = C.c_void_p()
        return self._handle(self.lib.wos_field_grid(self.handle, int(dim), r, _dvec(lo), _dvec(hi), _ptr(data),
                                                    _FIELD_KINDS[interp], C.byref(h)), h,
                            self.lib.wos_field_destroy, keep=data, dim=dim)

    def field(self, fd, dim):
        """A handle for a workloads field dict (grid data uploaded to this context's device)."""
        import torch
        k = fd["kind"]
        if k in ("zero",):
            return self.field_analytic("zero")
        if k == "const":
            return self.field_analytic("const", [fd["value"]])
        if k == "sst":
            return self.field_analytic("sst", pack_terms(fd["terms"]))
        if k.startswith("grid"):
            data = fd["data"]
            if not isinstance(data, torch.Tensor):
                data = torch.as_tensor(np.ascontiguousarray(data, dtype=np.float32))
            data = data.to(device=f"cuda:{self.device}", dtype=torch.float32).contiguous()
            return self.field_grid(dim, fd["res"][:dim], fd["lo"][:dim], fd["hi"][:dim], data, k)
        raise ValueError(f"field kind {k} has no handle of its own")

    def problem_assemble(self, domain, alpha, sigma, phi, f, g):
        """A Problem from handles (phi may be None)."""
        h = C.c_void_p()
        self._check(self.lib.wos_problem_assemble(self.handle, domain.handle, alpha.handle, sigma.handle,
                                                  phi.handle if phi is not None else None, f.handle, g.handle,
                                                  C.byref(h)))
        p = Problem.__new__(Problem)
        p.ctx, p.dim, p.handle = self, domain.dim, h
        p._keep = [domain, alpha, sigma, phi, f, g]
        p._sigma_ptr = sigma._keep.data_ptr() if sigma._keep is not None else 0
        p._alpha_ptr = alpha._keep.data_ptr() if alpha._keep is not None else 0
        self._children.add(p)
        return p

    def problem_sigma_bar(self, prob):
        a, b, c = C.c_double(), C.c_double(), C.c_double()
        self._check(self.lib.wos_problem_sigma_bar(self.handle, prob.handle, C.byref(a), C.byref(b), C.byref(c)))
        return a.value, b.value, c.value

    def new_moments(self, npts):
        """Zeroed (mean, var, count) for solve_mean."""
        import torch
        dev = f"cuda:{self.device}"
        return (torch.zeros(npts, dtype=torch.float64, device=dev), torch.zeros(npts, dtype=torch.float64, device=dev),
                torch.zeros(npts, dtype=torch.int64, device=dev))

    def _walks(self, walks, npts):
        import torch
        if isinstance(walks, int):
            return None, walks, None
        if not (isinstance(walks, torch.Tensor) and walks.is_cuda and walks.dtype == torch.int32
                and walks.shape == (npts,)):
            raise TypeError("walks must be an int or a CUDA int32 tensor of shape [npts]")
        walks = walks.contiguous()
        return _ptr(walks), 0, walks

    def solve_mean(self, prob, pts, walks, eps, sigma_bar, seed=0, walk_offset=0, max_steps=1 << 20,
                   precision="fp32", moments=None, stats=None, stream=None):
        """Per-point (mean, var, count), merged into `moments` when its counts are non-zero."""
        pts = _points(pts, prob.dim, self.device)
        npts = pts.shape[1]
        if moments is None:
            moments = self.new_moments(npts)
        if stats is None:
            stats = self.new_stats()
        wp, wu, _w = self._walks(walks, npts)
        p = params(eps, sigma_bar, seed, walk_offset, max_steps, precision)
        self._check(self.lib.wos_solve_mean(self.handle, prob.handle, _ptr(pts), npts, wp, wu, C.byref(p),
                                            _ptr(moments[0]), _ptr(moments[1]), _ptr(moments[2]), _ptr(stats),
                                            _stream(stream)))
        return moments, stats

    def solve_batched(self, problems, pt_offsets, sigma_bars, pts, walks, eps, seed=0, walk_offset=0,
                      max_steps=1 << 20, precision="fp32", moments=None, stats=None, stream=None):
        """One-call batch (creates, runs and frees a batch): per-point (mean, var, count)."""
        offs = np.ascontiguousarray(pt_offsets, dtype=np.int64)
        sbs = None if sigma_bars is None else np.ascontiguousarray(sigma_bars, dtype=np.float64)
        dim = problems[0].dim
        pts = _points(pts, dim, self.device)
        npts = pts.shape[1]
        if moments is None:
            moments = self.new_moments(npts)
        if stats is None:
            stats = self.new_stats()
        wp, wu, _w = self._walks(walks, npts)
        handles = (C.c_void_p * len(problems))(*[q.handle.value for q in problems])
        p = params(eps, 1.0, seed, walk_offset, max_steps, precision)
        self._check(self.lib.wos_solve_batched(self.handle, handles, len(problems), offs.ctypes.data,
                                               None if sbs is None else sbs.ctypes.data, _ptr(pts), wp, wu,
                                               C.byref(p), _ptr(moments[0]), _ptr(moments[1]), _ptr(moments[2]),
                                               _ptr(stats), _stream(stream)))
        return moments, stats

    def adjoint(self, prob, pts, walks_uniform, eps, sigma_bar, grad_u, sigma_nodes=0, alpha_nodes=0, seed=0,
                walk_offset=0, max_steps=1 << 20, precision="fp32", stats=None, stream=None):
        """wos_adjoint: float32 gradients with respect to the sigma grid (sigma_nodes > 0) and the
        alpha grid (alpha_nodes > 0); either is None when not asked for."""
        import torch
        pts = _points(pts, prob.dim, self.device)
        dev = f"cuda:{self.device}"
        gs = torch.empty(sigma_nodes, dtype=torch.float32, device=dev) if sigma_nodes else None
        ga = torch.empty(alpha_nodes, dtype=torch.float32, device=dev) if alpha_nodes else None
        gu = grad_u.to(device=dev, dtype=torch.float64).contiguous()
        p = params(eps, sigma_bar, seed, walk_offset, max_steps, precision)
        self._check(self.lib.wos_adjoint(self.handle, prob.handle, _ptr(pts), pts.shape[1], int(walks_uniform),
                                         C.byref(p), _ptr(gu), _ptr(gs), _ptr(ga), _ptr(stats), _stream(stream)))
        return gs, ga

    # ---- calls ----
    def problem(self, desc, specialize=None):
        """Upload a problem; specialize = None, or (precisions, variants) for Problem.specialize."""
        p = Problem(self, desc)
        if specialize:
            p.specialize(*specialize)
        return p

    def sigma_bar(self, prob, m=None, stream=None):
        if m is None:
            m = 256 if prob.dim == 2 else 64
        a, b, c = C.c_double(), C.c_double(), C.c_double()
        self._check(self.lib.wos_sigma_bar(self.handle, prob.handle, int(m), C.byref(a), C.byref(b), C.byref(c),
                                           _stream(stream)))
        return a.value, b.value, c.value

    def new_accum(self, npts):
        import torch
        dev = f"cuda:{self.device}"
        return (torch.zeros(npts, dtype=torch.float64, device=dev), torch.zeros(npts, dtype=torch.float64, device=dev),
                torch.zeros(npts, dtype=torch.int64, device=dev))

    def new_stats(self):
        import torch
        # the library adds unsigned 64-bit words; counts stay far below 2^63
        return torch.zeros(STATS_WORDS, dtype=torch.int64, device=f"cuda:{self.device}")

    def solve(self, prob, pts, walks, eps, sigma_bar, seed=0, walk_offset=0, max_steps=1 << 20, precision="fp32",
              accum=None, stats=None, stream=None, window=None):
        """Add walks to the accumulators (sum, sumsq, count); pts: cuda float32 [dim, npts]."""
        import torch
        pts = _points(pts, prob.dim, self.device)
        npts = pts.shape[1]
        if accum is None:
            accum = self.new_accum(npts)
        if not (accum[0].dtype == torch.float64 and accum[1].dtype == torch.float64 and accum[2].dtype == torch.int64
                and all(t.is_cuda and t.is_contiguous() and t.shape == (npts,) for t in accum)):
            raise TypeError("accumulators must be contiguous CUDA (float64, float64, int64) tensors of length npts")
        if stats is None:
            stats = self.new_stats()
        if isinstance(walks, int):
            wp, wu = None, walks
        else:
            if not (isinstance(walks, torch.Tensor) and walks.is_cuda and walks.dtype == torch.int32
                    and walks.shape == (npts,)):
                raise TypeError("walks must be an int or a CUDA int32 tensor of shape [npts]")
            walks = walks.contiguous()
            wp, wu = _ptr(walks), 0
        p = params(eps, sigma_bar, seed, walk_offset, max_steps, precision, window)
        self._check(self.lib.wos_solve(self.handle, prob.handle, _ptr(pts), npts, wp, wu, C.byref(p),
                                       _ptr(accum[0]), _ptr(accum[1]), _ptr(accum[2]), _ptr(stats),
                                       _stream(stream)))
        return accum, stats

    def walk_estimates(self, prob, pts, walks_per_point, eps, sigma_bar, seed=0, walk_offset=0, max_steps=1 << 20,
                       precision="fp32", stream=None, window=None):
        import torch
        pts = _points(pts, prob.dim, self.device)
        npts = pts.shape[1]
        dev = f"cuda:{self.device}"
        uhat = torch.empty((npts, walks_per_point), dtype=torch.float64, device=dev)
        steps = torch.empty((npts, walks_per_point), dtype=torch.int64, device=dev)
        stats = self.new_stats()
        p = params(eps, sigma_bar, seed, walk_offset, max_steps, precision, window)
        self._check(self.lib.wos_walk_estimates(self.handle, prob.handle, _ptr(pts), npts, int(walks_per_point),
                                                C.byref(p), _ptr(uhat), _ptr(steps), _ptr(stats), _stream(stream)))
        return uhat, steps, stats

    def slice_points(self, prob, v, stream=None):
        """The slice grid's points, CUDA float32 [dim, slice_nu * slice_nv]."""
        import torch
        pts = torch.empty((prob.dim, v.slice_nu * v.slice_nv), dtype=torch.float32, device=f"cuda:{self.device}")
        self._check(self.lib.wos_slice_points(self.handle, prob.handle, C.byref(v), _ptr(pts), _stream(stream)))
        return pts

    def render_slice(self, prob, v, accum, with_value=False, with_depth=False, stream=None):
        """RGBA8 image [height, width, 4] (CUDA uint8) of the view, and optionally the per-pixel
        value and depth buffers."""
        import torch
        dev = f"cuda:{self.device}"
        n = v.slice_nu * v.slice_nv
        if not (accum[0].shape == (n,) and accum[2].shape == (n,)):
            raise ValueError("accumulators must have one entry per slice point")
        img = torch.empty((v.height, v.width, 4), dtype=torch.uint8, device=dev)
        val = torch.empty((v.height, v.width), dtype=torch.float32, device=dev) if with_value else None
        dep = torch.empty((v.height, v.width), dtype=torch.float32, device=dev) if with_depth else None
        self._check(self.lib.wos_render_slice(self.handle, prob.handle, C.byref(v), _ptr(accum[0]), _ptr(accum[2]),
                                              _ptr(img), _ptr(val), _ptr(dep), _stream(stream)))
        return img, val, dep

    def solve_nf(self, prob, pts, walks, eps, sigma_bar, seed=0, walk_offset=0, max_steps=1 << 20,
                 max_inner=1 << 16, precision="fp32", accum=None, stats=None, stream=None, series_terms=8):
        """Next-flight walks (Sec. 5.2) added to the accumulators; stats 'steps' counts balls
        (distance queries), 'inner' the in-ball iterations.  series_terms = N in 1..64 takes the
        off-centred kernels as their series with N terms (in-ball points from the free-space
        kernel); 0 the printed approximations with uniform in-ball points."""
        import torch
        pts = _points(pts, prob.dim, self.device)
        npts = pts.shape[1]
        if accum is None:
            accum = self.new_accum(npts)
        if not (accum[0].dtype == torch.float64 and accum[1].dtype == torch.float64 and accum[2].dtype == torch.int64
                and all(t.is_cuda and t.is_contiguous() and t.shape == (npts,) for t in accum)):
            raise TypeError("accumulators must be contiguous CUDA (float64, float64, int64) tensors of length npts")
        if stats is None:
            stats = self.new_stats()
        if isinstance(walks, int):
            wp, wu = None, walks
        else:
            if not (isinstance(walks, torch.Tensor) and walks.is_cuda and walks.dtype == torch.int32
                    and walks.shape == (npts,)):
                raise TypeError("walks must be an int or a CUDA int32 tensor of shape [npts]")
            walks = walks.contiguous()
            wp, wu = _ptr(walks), 0
        p = params(eps, sigma_bar, seed, walk_offset, max_steps, precision)
        self._check(self.lib.wos_solve_nf(self.handle, prob.handle, _ptr(pts), npts, wp, wu, C.byref(p),
                                          int(max_inner), int(series_terms), _ptr(accum[0]), _ptr(accum[1]),
                                          _ptr(accum[2]),
                                          _ptr(stats), _stream(stream)))
        return accum, stats

    def walk_estimates_nf(self, prob, pts, walks_per_point, eps, sigma_bar, seed=0, walk_offset=0,
                          max_steps=1 << 20, max_inner=1 << 16, precision="fp32", stream=None, series_terms=8):
        import torch
        pts = _points(pts, prob.dim, self.device)
        npts = pts.shape[1]
        dev = f"cuda:{self.device}"
        uhat = torch.empty((npts, walks_per_point), dtype=torch.float64, device=dev)
        steps = torch.empty((npts, walks_per_point), dtype=torch.int64, device=dev)
        stats = self.new_stats()
        p = params(eps, sigma_bar, seed, walk_offset, max_steps, precision)
        self._check(self.lib.wos_walk_estimates_nf(self.handle, prob.handle, _ptr(pts), npts, int(walks_per_point),
                                                   C.byref(p), int(max_inner), int(series_terms), _ptr(uhat),
                                                   _ptr(steps),
                                                   _ptr(stats), _stream(stream)))
        return uhat, steps, stats

    def solve_grad(self, prob, pts, walks, eps, sigma_bar, seed=0, walk_offset=0, max_steps=1 << 20,
                   precision="fp32", accum=None, grad_accum=None, stats=None, stream=None):
        """Add walks' estimates of u and grad u (Supplemental Sec. 2).  Returns (accum, grad_accum,
        stats) with grad_accum = (sum, sumsq) of shape [dim, npts] float64; finalize_grad reads them."""
        import torch
        pts = _points(pts, prob.dim, self.device)
        npts = pts.shape[1]
        if accum is None:
            accum = self.new_accum(npts)
        if grad_accum is None:
            dev = f"cuda:{self.device}"
            grad_accum = tuple(torch.zeros((prob.dim, npts), dtype=torch.float64, device=dev) for _ in range(2))
        if not all(t.is_cuda and t.is_contiguous() and t.dtype == torch.float64 and t.shape == (prob.dim, npts)
                   for t in grad_accum):
            raise TypeError("gradient accumulators must be contiguous CUDA float64 tensors of shape [dim, npts]")
        if not (accum[0].dtype == torch.float64 and accum[1].dtype == torch.float64 and accum[2].dtype == torch.int64
                and all(t.is_cuda and t.is_contiguous() and t.shape == (npts,) for t in accum)):
            raise TypeError("accumulators must be contiguous CUDA (float64, float64, int64) tensors of length npts")
        if stats is None:
            stats = self.new_stats()
        if isinstance(walks, int):
            wp, wu = None, walks
        else:
            if not (isinstance(walks, torch.Tensor) and walks.is_cuda and walks.dtype == torch.int32
                    and walks.shape == (npts,)):
                raise TypeError("walks must be an int or a CUDA int32 tensor of shape [npts]")
            walks = walks.contiguous()
            wp, wu = _ptr(walks), 0
        p = params(eps, sigma_bar, seed, walk_offset, max_steps, precision)
        self._check(self.lib.wos_solve_grad(self.handle, prob.handle, _ptr(pts), npts, wp, wu, C.byref(p),
                                            _ptr(accum[0]), _ptr(accum[1]), _ptr(accum[2]), _ptr(grad_accum[0]),
                                            _ptr(grad_accum[1]), _ptr(stats), _stream(stream)))
        return accum, grad_accum, stats

    def finalize_grad(self, grad_accum, count, stream=None):
        """Per-component mean, variance and standard error [dim, npts] of the gradient estimate."""
        outs = [self.finalize((grad_accum[0][d], grad_accum[1][d], count), stream) for d in range(grad_accum[0].shape[0])]
        import torch
        return tuple(torch.stack([o[k] for o in outs]) for k in range(3))

    def walk_grad_estimates(self, prob, pts, walks_per_point, eps, sigma_bar, seed=0, walk_offset=0,
                            max_steps=1 << 20, precision="fp32", stream=None):
        """Per-walk (u, grad u [dim, npts, walks], steps, stats)."""
        import torch
        pts = _points(pts, prob.dim, self.device)
        npts = pts.shape[1]
        dev = f"cuda:{self.device}"
        uhat = torch.empty((npts, walks_per_point), dtype=torch.float64, device=dev)
        ghat = torch.empty((prob.dim, npts, walks_per_point), dtype=torch.float64, device=dev)
        steps = torch.empty((npts, walks_per_point), dtype=torch.int64, device=dev)
        stats = self.new_stats()
        p = params(eps, sigma_bar, seed, walk_offset, max_steps, precision)
        self._check(self.lib.wos_walk_grad_estimates(self.handle, prob.handle, _ptr(pts), npts, int(walks_per_point),
                                                     C.byref(p), _ptr(uhat), _ptr(ghat), _ptr(steps), _ptr(stats),
                                                     _stream(stream)))
        return uhat, ghat, steps, stats

    def finalize(self, accum, stream=None):
        import torch
        n = accum[0].shape[0]
        if not all(t.is_cuda and t.is_contiguous() and t.shape == (n,) for t in accum):
            raise TypeError("accumulators must be contiguous CUDA tensors of one length")
        mean, var, se = (torch.empty(n, dtype=torch.float64, device=accum[0].device) for _ in range(3))
        self._check(self.lib.wos_finalize(self.handle, _ptr(accum[0]), _ptr(accum[1]), _ptr(accum[2]), n,
                                          _ptr(mean), _ptr(var), _ptr(se), _stream(stream)))
        return mean, var, se

    def batch(self, problems, pt_offsets, sigma_bars):
        return Batch(self, problems, pt_offsets, sigma_bars)

    def solve_batch(self, batch, pts, walks, eps, seed=0, walk_offset=0, max_steps=1 << 20, precision="fp32",
                    accum=None, stats=None, stream=None):
        """One launch over every problem of the batch; pts: cuda float32 [dim, npts of the batch]."""
        import torch
        pts = _points(pts, batch.dim, self.device)
        npts = pts.shape[1]
        if npts != batch.npts:
            raise ValueError(f"the batch has {batch.npts} points, got {npts}")
        if accum is None:
            accum = self.new_accum(npts)
        if stats is None:
            stats = self.new_stats()
        if isinstance(walks, int):
            wp, wu = None, walks
        else:
            if not (isinstance(walks, torch.Tensor) and walks.is_cuda and walks.dtype == torch.int32
                    and walks.shape == (npts,)):
                raise TypeError("walks must be an int or a CUDA int32 tensor of shape [npts]")
            wp, wu = _ptr(walks.contiguous()), 0
        p = params(eps, 1.0, seed, walk_offset, max_steps, precision)
        self._check(self.lib.wos_solve_batch(self.handle, batch.handle, _ptr(pts), wp, wu, C.byref(p),
                                             _ptr(accum[0]), _ptr(accum[1]), _ptr(accum[2]), _ptr(stats),
                                             _stream(stream)))
        return accum, stats

    def batch_autotune(self, batch, pts, walks, eps, seed=0, trial_shift=4, precision="fp32", stream=None):
        """Time candidate launch schedules of the batch on trial walks (walks >> trial_shift)
        and keep the fastest in the batch: (schedule dict, best trial ms, default trial ms)."""
        import torch
        pts = _points(pts, batch.dim, self.device)
        if isinstance(walks, int):
            wp, wu = None, walks
        else:
            if not (isinstance(walks, torch.Tensor) and walks.is_cuda and walks.dtype == torch.int32
                    and walks.shape == (pts.shape[1],)):
                raise TypeError("walks must be an int or a CUDA int32 tensor of shape [npts]")
            wp, wu = _ptr(walks.contiguous()), 0
        p = params(eps, 1.0, seed, 0, 1 << 20, precision)
        sc = Schedule()
        best, dflt = C.c_double(), C.c_double()
        self._check(self.lib.wos_batch_autotune(self.handle, batch.handle, _ptr(pts), wp, wu, C.byref(p),
                                                int(trial_shift), C.byref(sc), C.byref(best), C.byref(dflt),
                                                _stream(stream)))
        return sc.as_dict(), best.value, dflt.value

    def adjoint_sigma(self, prob, pts, walks, grad_u, grad_sigma, eps, sigma_bar, seed=0, walk_offset=0,
                      max_steps=1 << 20, precision="fp32", stats=None, stream=None):
        """Add d(sum_p grad_u[p] mean_p)/d(sigma grid) to grad_sigma (CUDA float64, grid-sized)."""
        import torch
        pts = _points(pts, prob.dim, self.device)
        npts = pts.shape[1]
        if not (grad_u.is_cuda and grad_u.dtype == torch.float64 and grad_u.shape == (npts,)):
            raise TypeError("grad_u must be a CUDA float64 tensor of shape [npts]")
        if not (grad_sigma.is_cuda and grad_sigma.dtype == torch.float64 and grad_sigma.is_contiguous()):
            raise TypeError("grad_sigma must be a contiguous CUDA float64 tensor")
        grad_u = grad_u.contiguous()
        p = params(eps, sigma_bar, seed, walk_offset, max_steps, precision)
        self._check(self.lib.wos_adjoint_sigma(self.handle, prob.handle, _ptr(pts), npts, int(walks), C.byref(p),
                                               _ptr(grad_u), _ptr(grad_sigma), _ptr(stats), _stream(stream)))
        return grad_sigma

    def adjoint_alpha(self, prob, pts, walks, grad_u, grad_alpha, eps, sigma_bar, seed=0, walk_offset=0,
                      max_steps=1 << 20, precision="fp32", stats=None, stream=None):
        """Add d(sum_p grad_u[p] mean_p)/d(alpha B-spline grid) to grad_alpha (CUDA float64, grid-sized)."""
        import torch
        pts = _points(pts, prob.dim, self.device)
        npts = pts.shape[1]
        if not (grad_u.is_cuda and grad_u.dtype == torch.float64 and grad_u.shape == (npts,)):
            raise TypeError("grad_u must be a CUDA float64 tensor of shape [npts]")
        if not (grad_alpha.is_cuda and grad_alpha.dtype == torch.float64 and grad_alpha.is_contiguous()):
            raise TypeError("grad_alpha must be a contiguous CUDA float64 tensor")
        grad_u = grad_u.contiguous()
        p = params(eps, sigma_bar, seed, walk_offset, max_steps, precision)
        self._check(self.lib.wos_adjoint_alpha(self.handle, prob.handle, _ptr(pts), npts, int(walks), C.byref(p),
                                               _ptr(grad_u), _ptr(grad_alpha), _ptr(stats), _stream(stream)))
        return grad_alpha

    def solve_host(self, prob, pts_host, walks, eps, sigma_bar, seed=0, walk_offset=0, max_steps=1 << 20,
                   precision="fp32", out=None, stream=None):
        """Host arrays in, host arrays out (copies inside the call).  pts_host: float32 [dim, npts]
        numpy array or pinned torch tensor; out: optional (mean, var, se, stats) host buffers."""
        import torch
        if isinstance(pts_host, np.ndarray):
            pts_host = torch.from_numpy(np.ascontiguousarray(pts_host, dtype=np.float32))
        if pts_host.is_cuda or pts_host.dtype != torch.float32 or pts_host.dim() != 2 or pts_host.shape[0] != prob.dim:
            raise TypeError(f"host points must be a float32 CPU array of shape [{prob.dim}, npts]")
        pts_host = pts_host.contiguous()
        npts = pts_host.shape[1]
        if out is None:
            out = (torch.empty(npts, dtype=torch.float64), torch.empty(npts, dtype=torch.float64),
                   torch.empty(npts, dtype=torch.float64), torch.zeros(STATS_WORDS, dtype=torch.int64))
        if not all(t.numel() >= n for t, n in zip(out, (npts, npts, npts, STATS_WORDS))):
            raise ValueError("host output buffers are too small")
        p = params(eps, sigma_bar, seed, walk_offset, max_steps, precision)
        self._check(self.lib.wos_solve_host(self.handle, prob.handle, C.c_void_p(pts_host.data_ptr()), npts,
                                            int(walks), C.byref(p), C.c_void_p(out[0].data_ptr()),
                                            C.c_void_p(out[1].data_ptr()), C.c_void_p(out[2].data_ptr()),
                                            C.c_void_p(out[3].data_ptr()), _stream(stream)))
        return out


def stats_dict(stats):
    s = [int(v) for v in stats.cpu().tolist()]
    return {"steps": s[0], "walks": s[1], "capped": s[2], "nonfinite": s[3], "outside": s[4], "inner": s[5],
            "mesh_nodes": s[6], "mesh_tris": s[7], "exhausted": s[8]}


class SliceView:
    """Progressive solve on a slice plane (Sec. 7.2): each frame adds `walks` walks per slice
    point (continuing the Philox streams through walk_offset) and renders the view; `edit`
    swaps the problem and discards the accumulated walks."""

    def __init__(self, ctx, prob, v, eps, sigma_bar, seed=0):
        self.ctx, self.prob, self.view, self.eps, self.sigma_bar, self.seed = ctx, prob, v, eps, sigma_bar, seed
        self.pts = ctx.slice_points(prob, v)
        self.accum = ctx.new_accum(self.pts.shape[1])
        self.stats = ctx.new_stats()
        self.frames = 0

    def frame(self, walks=1, render=True, stream=None):
        self.ctx.solve(self.prob, self.pts, walks, self.eps, self.sigma_bar, seed=self.seed,
                       walk_offset=self.frames, accum=self.accum, stats=self.stats, stream=stream)
        self.frames += walks
        return self.ctx.render_slice(self.prob, self.view, self.accum, stream=stream)[0] if render else None

    def edit(self, prob, sigma_bar=None):
        self.prob = prob
        if sigma_bar is not None:
            self.sigma_bar = sigma_bar
        for t in self.accum:
            t.zero_()
        self.stats.zero_()
        self.frames = 0


def write_ppm(path, rgba):
    """Write an RGBA8 image (array or tensor [h, w, 4]) as a binary PPM file."""
    a = rgba.cpu().numpy() if hasattr(rgba, "cpu") else np.asarray(rgba)
    h, w = a.shape[:2]
    with open(path, "wb") as f:
        f.write(b"P6\n%d %d\n255\n" % (w, h))
        f.write(np.ascontiguousarray(a[:, :, :3]).tobytes())
