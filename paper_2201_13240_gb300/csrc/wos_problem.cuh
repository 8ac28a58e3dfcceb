// wos_problem.cuh -- device description of one PDE problem and its point-wise
// evaluation: coefficient fields, the transformation to a screened Poisson
// equation, and the distance to the domain boundary.
//
//   PDE (Sec. 3, eq. 1): div(alpha grad u) + omega . grad u - sigma u = -f,
//                        u = g on the boundary, omega = alpha grad(Phi).
//   Transform (Sec. 4.1 eq. 7-8, App. A):
//     gamma = 1/2 ln alpha + 1/2 Phi,  U = e^gamma u,
//     sigma' = sigma/alpha + Lap(gamma) + |grad gamma|^2,
//     f' = e^gamma f / alpha,  g' = e^gamma g,  Lap U - sigma' U = -f'.
#pragma once

#if !defined(__CUDACC_RTC__)
#include <stdint.h>
#include <string.h>
#endif

#include "wos_math.cuh"

#if defined(__CUDACC__)
#define WOS_FIELD_FN __host__ __device__ __noinline__
#else
#define WOS_FIELD_FN inline
#endif

namespace wos {

enum AtomType { A_ONE = 0, A_SIN = 1, A_COS = 2, A_EXP = 3, A_SINH = 4, A_COSH = 5, A_LIN = 6, A_QUAD = 7 };
enum FieldKind { F_ZERO = 0, F_CONST = 1, F_SST = 2, F_MANUFACTURED = 3, F_GRID_LINEAR = 4, F_GRID_BSPLINE = 5 };
enum DomainKind { D_BOX = 0, D_BALL = 1, D_ANNULUS = 2, D_ROUNDED_BOX = 3, D_MESH = 4, D_CSG = 5 };
enum CsgPrim { C_SPHERE = 0, C_BOX = 1, C_CAPSULE = 2, C_TORUS = 3, C_HALFSPACE = 4 };
enum CsgOp { C_UNION = 0, C_INTERSECT = 1, C_SUBTRACT = 2 };
constexpr int kMaxCsg = 16;
constexpr double kDriftSigmaBar = 50.0;  // sigma_bar >= this times max |omega/alpha|^2 (extra drift)

template <typename R>
struct CsgNode {
  int32_t prim;
  int32_t op;
  R p[8];
};

constexpr int kMaxTerms = 96;  // separable terms over all fields of one problem

template <typename R>
struct DevTerm {
  R c;
  R k[3];
  R phi[3];
  int32_t type[3];
};

template <typename R>
struct DevField {
  int32_t kind;
  int32_t nterms;
  int32_t first;  // first term in DevProblem::terms
  int32_t pad;
  R value;
  R lo[3];
  R inv_h[3];     // grid: 1 / node spacing
  int32_t res[3];
  int32_t pad2;
  const float* data;  // grid values, x fastest, device memory owned by the caller
};

template <typename R>
struct DevProblem {
  int32_t dim;
  int32_t domain_kind;
  int32_t nterms;
  int32_t pad;
  R dom[16];
  DevField<R> alpha, phi, sigma, f, g, um;
  DevField<R> omega[3];     // extra drift (any vector field); has_drift when any is not ZERO
  int32_t has_drift;
  int32_t pad5;
  alignas(16) const float* mesh_nodes;  // BVH: 32 floats per 4-wide node (see wos_mesh.h), device
  const float* mesh_tris;   // 12 floats per triangle in leaf order, device
  int32_t ncsg;
  int32_t mg_res;           // mesh distance grid: nodes per axis (0: none)
  int32_t mesh_top;         // the first mesh_top nodes are the tree's top levels (staged in shared memory)
  int32_t pad3;
  const R* mgrid;           // exact distances at the grid nodes, x fastest, device
  const void* mg_pad_ptr;   // keeps the 16-byte layout
  R mg_lo[3], mg_h[3], mg_inv_h[3];
  R mg_thresh;              // use the grid's lower bound when it is at least this
  R mesh_tau;               // mesh queries: squared radius factor (1 - tol)^2 (1: exact radii)
  R drift_bound;            // extra drift: B >= max |omega / alpha| (0: none), for per-ball bounds
  CsgNode<R> csg[kMaxCsg];
  DevTerm<R> terms[kMaxTerms];
};

// ---------------------------------------------------------------------------
// separable terms: c * prod_i h_i(k_i x_i + phi_i)
// ---------------------------------------------------------------------------
template <typename R>
WOS_HD void atom(int type, R k, R ph, R x, R* h, R* h1, R* h2) {
  R t = k * x + ph;
  switch (type) {
    case A_SIN: {
      R s, c;
      w_sincos(t, &s, &c);
      *h = s; *h1 = k * c; *h2 = -k * k * s;
      break;
    }
    case A_COS: {
      R s, c;
      w_sincos(t, &s, &c);
      *h = c; *h1 = -k * s; *h2 = -k * k * c;
      break;
    }
    case A_EXP: {
      R e = w_exp(t);
      *h = e; *h1 = k * e; *h2 = k * k * e;
      break;
    }
    case A_SINH:
    case A_COSH: {
      R e = w_exp(t), ei = w_div(R(1), e);
      R sh = R(0.5) * (e - ei), ch = R(0.5) * (e + ei);
      if (type == A_SINH) { *h = sh; *h1 = k * ch; *h2 = k * k * sh; }
      else { *h = ch; *h1 = k * sh; *h2 = k * k * ch; }
      break;
    }
    case A_LIN: *h = t; *h1 = k; *h2 = R(0); break;
    case A_QUAD: *h = t * t; *h1 = R(2) * k * t; *h2 = R(2) * k * k; break;
    default: *h = R(1); *h1 = R(0); *h2 = R(0); break;
  }
}

template <int DIM, typename R>
WOS_HD void sst_eval(const DevProblem<R>& P, const DevField<R>& F, const R* x, R* v, R* g, R* lap,
                     bool deriv) {
  R vv = R(0), ll = R(0), g0 = R(0), g1 = R(0), g2 = R(0);
#pragma unroll 1
  for (int n = 0; n < F.nterms; ++n) {
    const DevTerm<R>& T = P.terms[F.first + n];
    R h[3] = {R(1), R(1), R(1)}, h1[3] = {R(0), R(0), R(0)}, h2[3] = {R(0), R(0), R(0)};
    // a constant atom is skipped by a test that is uniform across the warp (every lane
    // reads the same term); measured 12% faster than dispatching it
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      if (T.type[i] == A_ONE) continue;
      atom(T.type[i], T.k[i], T.phi[i], x[i], &h[i], &h1[i], &h2[i]);
    }
    R p01 = h[0] * h[1];
    vv += T.c * p01 * h[2];
    if (deriv) {
      g0 += T.c * h1[0] * h[1] * h[2];
      g1 += T.c * h[0] * h1[1] * h[2];
      g2 += T.c * p01 * h1[2];
      ll += T.c * (h2[0] * h[1] * h[2] + h[0] * h2[1] * h[2] + p01 * h2[2]);
    }
  }
  *v = vv;
  if (deriv) {
    g[0] = g0; g[1] = g1; g[2] = g2;
    *lap = ll;
  }
}

// node-centred multilinear interpolation, clamped to the grid box
template <int DIM, typename R>
WOS_HD R grid_linear(const DevField<R>& F, const R* x) {
  int i0[3] = {0, 0, 0};
  R t[3] = {R(0), R(0), R(0)};
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    R s = (x[d] - F.lo[d]) * F.inv_h[d];
    s = w_fmin(w_fmax(s, R(0)), R(F.res[d] - 1));
    int i = (int)s;
    if (i > F.res[d] - 2) i = F.res[d] - 2;
    i0[d] = i;
    t[d] = s - R(i);
  }
  const float* base = F.data + i0[0] + (int64_t)F.res[0] * (i0[1] + (int64_t)F.res[1] * (DIM == 3 ? i0[2] : 0));
  int64_t sy = F.res[0], sz = (int64_t)F.res[0] * F.res[1];
  R v00 = R(base[0]) + t[0] * (R(base[1]) - R(base[0]));
  R v10 = R(base[sy]) + t[0] * (R(base[sy + 1]) - R(base[sy]));
  R v0 = v00 + t[1] * (v10 - v00);
  if (DIM == 2) return v0;
  R v01 = R(base[sz]) + t[0] * (R(base[sz + 1]) - R(base[sz]));
  R v11 = R(base[sz + sy]) + t[0] * (R(base[sz + sy + 1]) - R(base[sz + sy]));
  R v1 = v01 + t[1] * (v11 - v01);
  return v0 + t[2] * (v1 - v0);
}

template <typename R>
WOS_HD void bspline_w(R t, R* B, R* B1, R* B2) {
  R u = R(1) - t, t2 = t * t, t3 = t2 * t;
  B[0] = u * u * u * R(1.0 / 6.0);
  B[1] = (R(3) * t3 - R(6) * t2 + R(4)) * R(1.0 / 6.0);
  B[2] = (R(-3) * t3 + R(3) * t2 + R(3) * t + R(1)) * R(1.0 / 6.0);
  B[3] = t3 * R(1.0 / 6.0);
  B1[0] = R(-0.5) * u * u;
  B1[1] = R(0.5) * (R(3) * t2 - R(4) * t);
  B1[2] = R(0.5) * (R(-3) * t2 + R(2) * t + R(1));
  B1[3] = R(0.5) * t2;
  B2[0] = u;
  B2[1] = R(3) * t - R(2);
  B2[2] = R(-3) * t + R(1);
  B2[3] = t;
}

// uniform cubic B-spline with the node values as control points; control
// indices clamped to the grid (constant extension) so the field stays C^2
template <int DIM, typename R>
WOS_HD void grid_bspline(const DevField<R>& F, const R* x, R* v, R* g, R* lap, bool deriv) {
  int ib[3] = {0, 0, 0};
  R B[3][4], B1[3][4], B2[3][4];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
#pragma unroll
    for (int a = 0; a < 4; ++a) { B[d][a] = (a == 0) ? R(1) : R(0); B1[d][a] = R(0); B2[d][a] = R(0); }
  }
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    R s = (x[d] - F.lo[d]) * F.inv_h[d];
    R fs = floor(s);
    ib[d] = (int)fs - 1;
    bspline_w(s - fs, B[d], B1[d], B2[d]);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      B1[d][a] *= F.inv_h[d];
      B2[d][a] *= F.inv_h[d] * F.inv_h[d];
    }
  }
  int idx[3][4];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      int j = ib[d] + a;
      int hi = (d < DIM) ? F.res[d] - 1 : 0;
      j = j < 0 ? 0 : (j > hi ? hi : j);
      idx[d][a] = j;
    }
  }
  R vv = R(0), g0 = R(0), g1 = R(0), g2 = R(0), ll = R(0);
  const int n2 = (DIM == 3) ? 4 : 1;
  for (int c2 = 0; c2 < n2; ++c2) {
#pragma unroll
    for (int c1 = 0; c1 < 4; ++c1) {
      const float* row = F.data + (int64_t)F.res[0] * (idx[1][c1] + (int64_t)F.res[1] * idx[2][c2]);
      R r = R(0), r1 = R(0), r2 = R(0);
#pragma unroll
      for (int c0 = 0; c0 < 4; ++c0) {
        R val = R(row[idx[0][c0]]);
        r += val * B[0][c0];
        r1 += val * B1[0][c0];
        r2 += val * B2[0][c0];
      }
      R b1 = B[1][c1], b2 = B[2][c2];
      vv += r * b1 * b2;
      if (deriv) {
        g0 += r1 * b1 * b2;
        g1 += r * B1[1][c1] * b2;
        g2 += r * b1 * B1[2][c2];
        ll += r2 * b1 * b2 + r * B2[1][c1] * b2 + r * b1 * B2[2][c2];
      }
    }
  }
  *v = vv;
  if (deriv) {
    g[0] = g0; g[1] = g1; g[2] = g2;
    *lap = ll;
  }
}

// value, gradient and Laplacian of a field at a point
template <typename R>
struct FieldVal {
  R v, gx, gy, gz, lap;
};

// value (and gradient / Laplacian when deriv) of a plain field.  On the device it
// is one out-of-line function taking and returning registers: a step evaluates
// several fields, and inlining the separable-term and B-spline code at every
// call site made the walk kernel too large for the instruction cache.
template <int DIM, typename R>
WOS_FIELD_FN FieldVal<R> field_eval(const DevProblem<R>& P, const DevField<R>& F, R x0, R x1, R x2, bool deriv) {
  FieldVal<R> o = {R(0), R(0), R(0), R(0), R(0)};
  const R x[3] = {x0, x1, x2};
  R g[3] = {R(0), R(0), R(0)};
  switch (F.kind) {
    case F_CONST: o.v = F.value; return o;
    case F_SST: sst_eval<DIM>(P, F, x, &o.v, g, &o.lap, deriv); break;
    case F_GRID_LINEAR: o.v = grid_linear<DIM>(F, x); return o;  // piecewise linear: no second derivative
    case F_GRID_BSPLINE: grid_bspline<DIM>(F, x, &o.v, g, &o.lap, deriv); break;
    default: return o;
  }
  o.gx = g[0];
  o.gy = g[1];
  o.gz = g[2];
  return o;
}

// Fields as the walk kernel reads them.  A kernel compiled at run time for one
// problem (WOS_JIT_FIELDS) evaluates each of its fields by generated straight-line
// code with the problem's constants folded in (jit_field, emitted after this
// header); every other kernel interprets the field descriptors.
enum FieldId { FLD_ALPHA = 0, FLD_PHI = 1, FLD_SIGMA = 2, FLD_F = 3, FLD_G = 4, FLD_UM = 5, FLD_OMEGA0 = 6 };
#if defined(WOS_JIT_FIELDS)
template <int DIM, typename R>
__device__ __forceinline__ FieldVal<R> jit_field(const DevProblem<R>& P, int id, R x0, R x1, R x2, bool deriv);
#define WOS_FIELD(P, ID, F, x0, x1, x2, deriv) jit_field<DIM, R>(P, ID, x0, x1, x2, deriv)
#define WOS_F_KIND(P) (WOS_JIT_F_KIND)
#else
#define WOS_FIELD(P, ID, F, x0, x1, x2, deriv) field_eval<DIM>(P, F, x0, x1, x2, deriv)
#define WOS_F_KIND(P) ((P).f.kind)
#endif

// Transformed coefficients at y: sigma'(y), f'(y) and gamma(y) (Sec. 4.1, App. A).
// DRIFT: the problem has an extra drift omega; sp then also holds b . grad gamma + div b
// (b = omega / alpha) and b_out receives b(y).
// The fields coeffs evaluated (alpha and Phi with gradient and Laplacian, sigma's value):
// the alpha adjoint reuses them for d sigma' / d alpha instead of evaluating them again.
template <typename R>
struct FieldsAt {
  FieldVal<R> A, Ph;
  R S;
};

template <int DIM, typename R, bool DRIFT = false>
WOS_HD void coeffs(const DevProblem<R>& P, const R* y, R* sp, R* fp, R* gamma_out = nullptr,
                   R* alpha_out = nullptr, R* b_out = nullptr, FieldsAt<R>* raw = nullptr) {
  FieldVal<R> A = WOS_FIELD(P, FLD_ALPHA, P.alpha, y[0], y[1], y[2], true);
  FieldVal<R> Ph = WOS_FIELD(P, FLD_PHI, P.phi, y[0], y[1], y[2], true);
  FieldVal<R> S = WOS_FIELD(P, FLD_SIGMA, P.sigma, y[0], y[1], y[2], false);
  const R ga[3] = {A.gx, A.gy, A.gz}, gp[3] = {Ph.gx, Ph.gy, Ph.gz};
  R f;
  if (WOS_F_KIND(P) == F_MANUFACTURED) {
    // eq. 1 solved for f at the manufactured u: f = -(alpha Lap u + grad alpha . grad u)
    //                                              - alpha grad Phi . grad u + sigma u
    FieldVal<R> U = WOS_FIELD(P, FLD_UM, P.um, y[0], y[1], y[2], true);
    const R gu[3] = {U.gx, U.gy, U.gz};
    R da = R(0), dp = R(0);
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      da += ga[d] * gu[d];
      dp += gp[d] * gu[d];
    }
    f = -(A.v * U.lap + da) - A.v * dp + S.v * U.v;
    if (DRIFT) {
#pragma unroll
      for (int d = 0; d < DIM; ++d) f -= WOS_FIELD(P, FLD_OMEGA0 + d, P.omega[d], y[0], y[1], y[2], false).v * gu[d];
    }
  } else {
    f = WOS_FIELD(P, FLD_F, P.f, y[0], y[1], y[2], false).v;
  }
  R ia = w_div(R(1), A.v);
  R na2 = R(0), ng2 = R(0);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    R gg = R(0.5) * (ga[d] * ia + gp[d]);
    ng2 += gg * gg;
    na2 += ga[d] * ga[d];
  }
  R lgam = R(0.5) * (A.lap * ia - na2 * ia * ia + Ph.lap);
  *sp = S.v * ia + lgam + ng2;
  R gam = R(0.5) * w_log(A.v) + R(0.5) * Ph.v;
  *fp = w_exp(gam) * f * ia;
  if (gamma_out) *gamma_out = gam;
  if (alpha_out) *alpha_out = A.v;
  if (raw) {
    raw->A = A;
    raw->Ph = Ph;
    raw->S = S.v;
  }
  if (DRIFT) {
    // sigma'' = sigma' + b . grad gamma; div b = div omega / alpha - omega . grad alpha / alpha^2
    R divw = R(0), wga = R(0), bg = R(0);
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      FieldVal<R> Wd = WOS_FIELD(P, FLD_OMEGA0 + d, P.omega[d], y[0], y[1], y[2], true);
      const R gw[3] = {Wd.gx, Wd.gy, Wd.gz};
      divw += gw[d];
      wga += Wd.v * ga[d];
      R bd = Wd.v * ia;
      bg += bd * R(0.5) * (ga[d] * ia + gp[d]);
      if (b_out) b_out[d] = bd;
    }
    *sp += bg + divw * ia - wga * ia * ia;
  }
}

template <int DIM, typename R>
WOS_HD R gamma_at(const DevProblem<R>& P, const R* x) {
  R a = WOS_FIELD(P, FLD_ALPHA, P.alpha, x[0], x[1], x[2], false).v;
  R ph = WOS_FIELD(P, FLD_PHI, P.phi, x[0], x[1], x[2], false).v;
  return R(0.5) * w_log(a) + R(0.5) * ph;
}

// grad gamma = (grad alpha / alpha + grad Phi) / 2 (Sec. 4.1, App. A)
template <int DIM, typename R>
WOS_HD void grad_gamma_at(const DevProblem<R>& P, const R* x, R* g) {
  FieldVal<R> A = WOS_FIELD(P, FLD_ALPHA, P.alpha, x[0], x[1], x[2], true);
  FieldVal<R> Ph = WOS_FIELD(P, FLD_PHI, P.phi, x[0], x[1], x[2], true);
  R ia = R(1) / A.v;
  g[0] = R(0.5) * (A.gx * ia + Ph.gx);
  g[1] = R(0.5) * (A.gy * ia + Ph.gy);
  g[2] = R(0.5) * (A.gz * ia + Ph.gz);
}

template <int DIM, typename R>
WOS_HD R g_at(const DevProblem<R>& P, const R* x) {
  return WOS_FIELD(P, FLD_G, P.g, x[0], x[1], x[2], false).v;
}

// ---------------------------------------------------------------------------
// triangle-mesh boundary: closest point through the BVH built at problem
// creation (Sec. 7.1).  Nodes and triangles are read through the read-only
// cache; the traversal keeps a per-lane stack of (node, squared box distance),
// visits the nearer child first and skips every box farther than the best
// triangle so far.
// ---------------------------------------------------------------------------
constexpr int kMeshStack = 32;  // entries of the traversal stack (a full stack repeats the pass: mesh_query)
constexpr int kMeshTopMax = 21;  // nodes of the BVH's top levels staged in shared memory (1 + 4 + 16)

struct F4 {
  float x, y, z, w;
};
WOS_HD F4 ld4(const float* p) {
#if defined(__CUDA_ARCH__)
  float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return F4{v.x, v.y, v.z, v.w};
#else
  return F4{p[0], p[1], p[2], p[3]};
#endif
}
WOS_HD int f_as_i(float f) {
#if defined(__CUDA_ARCH__)
  return __float_as_int(f);
#else
  int i;
  memcpy(&i, &f, 4);
  return i;
#endif
}

template <typename R>
WOS_HD R box_d2(const R* x, const F4& lo, const F4& hi) {
  R dx = w_fmax(w_fmax(R(lo.x) - x[0], x[0] - R(hi.x)), R(0));
  R dy = w_fmax(w_fmax(R(lo.y) - x[1], x[1] - R(hi.y)), R(0));
  R dz = w_fmax(w_fmax(R(lo.z) - x[2], x[2] - R(hi.z)), R(0));
  return dx * dx + dy * dy + dz * dz;
}

// Closest point of triangle (a, b, c) to p by its Voronoi regions (Ericson,
// Real-Time Collision Detection, Sec. 5.1.5): barycentric (v, w) of the point.
template <typename R>
WOS_HD void tri_closest(const R* p, const float* t, R* v_out, R* w_out, R* d2_out) {
  F4 A = ld4(t), B = ld4(t + 4), Cc = ld4(t + 8);
  R ab[3] = {R(B.x) - R(A.x), R(B.y) - R(A.y), R(B.z) - R(A.z)};
  R ac[3] = {R(Cc.x) - R(A.x), R(Cc.y) - R(A.y), R(Cc.z) - R(A.z)};
  R ap[3] = {p[0] - R(A.x), p[1] - R(A.y), p[2] - R(A.z)};
  R d1 = ab[0] * ap[0] + ab[1] * ap[1] + ab[2] * ap[2];
  R d2 = ac[0] * ap[0] + ac[1] * ap[1] + ac[2] * ap[2];
  R abab = ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2];
  R acac = ac[0] * ac[0] + ac[1] * ac[1] + ac[2] * ac[2];
  R abac = ab[0] * ac[0] + ab[1] * ac[1] + ab[2] * ac[2];
  R d3 = d1 - abab, d4 = d2 - abac;  // ab.(p-b), ac.(p-b)
  R d5 = d1 - abac, d6 = d2 - acac;  // ab.(p-c), ac.(p-c)
  R v, w;
  R vc = d1 * d4 - d3 * d2, vb = d5 * d2 - d1 * d6, va = d3 * d6 - d5 * d4;
  if (d1 <= R(0) && d2 <= R(0)) { v = R(0); w = R(0); }                       // vertex a
  else if (d3 >= R(0) && d4 <= d3) { v = R(1); w = R(0); }                    // vertex b
  else if (d6 >= R(0) && d5 <= d6) { v = R(0); w = R(1); }                    // vertex c
  else if (vc <= R(0) && d1 >= R(0) && d3 <= R(0)) { v = w_div(d1, d1 - d3); w = R(0); }   // edge ab
  else if (vb <= R(0) && d2 >= R(0) && d6 <= R(0)) { v = R(0); w = w_div(d2, d2 - d6); }   // edge ac
  else if (va <= R(0) && (d4 - d3) >= R(0) && (d5 - d6) >= R(0)) {                    // edge bc
    w = w_div(d4 - d3, (d4 - d3) + (d5 - d6));
    v = R(1) - w;
  } else {                                                                              // interior
    R den = w_div(R(1), va + vb + vc);
    v = vb * den;
    w = vc * den;
  }
  R q[3] = {ap[0] - ab[0] * v - ac[0] * w, ap[1] - ab[1] * v - ac[1] * w, ap[2] - ab[2] * v - ac[2] * w};
  *v_out = v;
  *w_out = w;
  *d2_out = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
}

template <typename R>
struct MeshHit {
  R d;        // a certified lower bound of the distance: the exact distance when tau = 1
  R x, y, z;  // the best boundary point found (NaN when none is known)
};

// Counters of one lane's mesh queries (BVH nodes visited, triangles tested, searches that
// found no boundary point), added to the walk statistics.
struct MeshVisits {
  unsigned long long nodes, tris;
  uint32_t exhausted;
};

// bound2: an upper bound of the squared distance (a known boundary point's), or
// infinity.  The search starts from it, slightly enlarged for rounding, so only
// boxes nearer than a known boundary point are opened.
// tau = 1 (exact): if rounding still hides every triangle, the search restarts
// without the bound, and the result does not depend on the bound.
// tau < 1 (a radius within a factor sqrt(tau) of the distance): a box is opened only
// if its squared distance is below tau times the best squared distance so far, and
// the query returns sqrt(tau * best).  Every box left closed then holds only triangles
// at squared distance >= tau * best, and every tested triangle is at >= best, so the
// returned value is a lower bound of the distance (the ball it spans lies in the
// domain, which keeps the walk's estimator unbiased) and at least sqrt(tau) times the
// distance.  When nothing is found inside the bound, the bound's own boundary point pb
// (if given) is the best point.  Deep inside a near-spherical surface almost every
// leaf lies within the exact search's bound; with tau < 1 the query stops at boxes
// that are small enough to be certified.
// The tree has 4-wide nodes of one 128-byte line (MeshNode4 in wos_mesh.h: child boxes
// as structure of arrays): a visit loads one line and tests four boxes, so a query
// follows half as many dependent loads as in the binary tree.  Leaf children nearer
// than the best triangle are tested at once; the nearest interior child is visited
// next and the others are pushed, farther first.  A full stack drops the entry and
// marks the pass; a marked pass is repeated from the root with the best distance found
// (still exact: every dropped node is seen again).
// SMEM: the stack lives in shared memory, entry k of this thread at sn[k * stride] and
// sd[k * stride] (a column per thread: no bank conflicts); otherwise in local memory.
// Kept in local memory by the walk kernels, the stack's divergent per-lane accesses
// were the largest memory traffic of a mesh walk.
struct I4 {
  int x, y, z, w;
};
WOS_HD I4 ld4i(const float* p) {
#if defined(__CUDA_ARCH__)
  int4 v = __ldg(reinterpret_cast<const int4*>(p));
  return I4{v.x, v.y, v.z, v.w};
#else
  I4 v;
  memcpy(&v, p, 16);
  return v;
#endif
}
// 16 bytes of a node staged in shared memory (plain loads: the address is a shared one)
WOS_HD F4 lds4(const float* p) {
#if defined(__CUDA_ARCH__)
  const float4 v = *reinterpret_cast<const float4*>(p);
  return F4{v.x, v.y, v.z, v.w};
#else
  return F4{p[0], p[1], p[2], p[3]};
#endif
}
WOS_HD I4 lds4i(const float* p) {
#if defined(__CUDA_ARCH__)
  const int4 v = *reinterpret_cast<const int4*>(p);
  return I4{v.x, v.y, v.z, v.w};
#else
  I4 v;
  memcpy(&v, p, 16);
  return v;
#endif
}
template <typename R>
WOS_HD R box_d2_1(const R* x, float lx, float ly, float lz, float hx, float hy, float hz) {
  R dx = w_fmax(w_fmax(R(lx) - x[0], x[0] - R(hx)), R(0));
  R dy = w_fmax(w_fmax(R(ly) - x[1], x[1] - R(hy)), R(0));
  R dz = w_fmax(w_fmax(R(lz) - x[2], x[2] - R(hz)), R(0));
  return dx * dx + dy * dy + dz * dz;
}

template <typename R, bool SMEM>
WOS_FIELD_FN MeshHit<R> mesh_query(const DevProblem<R>& P, R x0, R x1, R x2, R bound2, int* sn, R* sd,
                                   int stride, R tau = R(1), const R* pb = nullptr, MeshVisits* vis = nullptr,
                                   const float* top = nullptr) {
  const R x[3] = {x0, x1, x2};
  const float* nodes = P.mesh_nodes;
  const float* tris = P.mesh_tris;
  int loc_n[SMEM ? 1 : kMeshStack];
  R loc_d[SMEM ? 1 : kMeshStack];
  int* stk_n = SMEM ? sn : loc_n;
  R* stk_d = SMEM ? sd : loc_d;
  const int sst = SMEM ? stride : 1;
  const bool exact = !(tau < R(1));
  R best = R(INFINITY), bv = R(0), bw = R(0);
  int best_t = -1;
  const R slack = (sizeof(R) == 4) ? R(1e-5) : R(1e-12);
  const R start = (bound2 < R(INFINITY)) ? bound2 * (R(1) + slack) + R(1e-30) : R(INFINITY);
  unsigned long long n_nodes = 0, n_tris = 0;
  bool again = true;
  for (int pass = 0; pass < 8 && again; ++pass) {
    // pass 0 starts from the bound.  Exact: a pass that found nothing within it, or
    // dropped stack entries, is followed by one from the root with the best so far (or
    // none).  tau < 1: only a pass that dropped entries is repeated, from the best so far.
    if (pass == 0) best = start;
    else if (best_t < 0 && exact) best = R(INFINITY);
    again = false;
    int sp = 0;
    int node = 0;
    for (;;) {
      F4 lx, ly, lz, hx, hy, hz;
      I4 ch, cn;
      if (top != nullptr && node < P.mesh_top) {
        // one of the tree's top nodes, staged in shared memory by the kernel
        const float* nd = top + 32 * node;
        lx = lds4(nd); ly = lds4(nd + 4); lz = lds4(nd + 8);
        hx = lds4(nd + 12); hy = lds4(nd + 16); hz = lds4(nd + 20);
        ch = lds4i(nd + 24); cn = lds4i(nd + 28);
      } else {
        const float* nd = nodes + 32 * node;
        lx = ld4(nd); ly = ld4(nd + 4); lz = ld4(nd + 8);
        hx = ld4(nd + 12); hy = ld4(nd + 16); hz = ld4(nd + 20);
        ch = ld4i(nd + 24); cn = ld4i(nd + 28);
      }
      ++n_nodes;
      R d[4] = {box_d2_1(x, lx.x, ly.x, lz.x, hx.x, hy.x, hz.x), box_d2_1(x, lx.y, ly.y, lz.y, hx.y, hy.y, hz.y),
                box_d2_1(x, lx.z, ly.z, lz.z, hx.z, hy.z, hz.z), box_d2_1(x, lx.w, ly.w, lz.w, hx.w, hy.w, hz.w)};
      const int cc[4] = {ch.x, ch.y, ch.z, ch.w}, nc[4] = {cn.x, cn.y, cn.z, cn.w};
      // leaf children within the opening threshold: test them now (lowers best)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (nc[i] > 0 && d[i] < tau * best) {
          for (int j = 0; j < nc[i]; ++j) {
            R v, w, d2;
            tri_closest(x, tris + 12 * (cc[i] + j), &v, &w, &d2);
            if (d2 < best) { best = d2; best_t = cc[i] + j; bv = v; bw = w; }
          }
          n_tris += (unsigned long long)nc[i];
        }
      }
      const R thr = tau * best;
      // interior children within the threshold: sort by distance (others at infinity)
      R k[4];
      int c[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        k[i] = (nc[i] == 0 && d[i] < thr) ? d[i] : R(INFINITY);
        c[i] = cc[i];
      }
#define WOS_CSWAP(a, b)                                   \
  if (k[b] < k[a]) {                                      \
    R tk = k[a]; k[a] = k[b]; k[b] = tk;                  \
    int tc = c[a]; c[a] = c[b]; c[b] = tc;                \
  }
      WOS_CSWAP(0, 1) WOS_CSWAP(2, 3) WOS_CSWAP(0, 2) WOS_CSWAP(1, 3) WOS_CSWAP(1, 2)
#undef WOS_CSWAP
      // push the farther ones (farthest first, so the nearer are popped first)
#pragma unroll
      for (int i = 3; i >= 1; --i) {
        if (k[i] < thr) {
          if (sp < kMeshStack) {
            stk_n[sp * sst] = c[i];
            stk_d[sp * sst] = k[i];
            ++sp;
          } else {
            again = true;
          }
        }
      }
      if (k[0] < thr) {
        node = c[0];
        continue;
      }
      // pop the next node still within the threshold of the best triangle
      bool found = false;
      while (sp > 0) {
        --sp;
        if (stk_d[sp * sst] < tau * best) { node = stk_n[sp * sst]; found = true; break; }
      }
      if (!found) break;
    }
    if (best_t < 0 && exact) again = true;
  }
  MeshHit<R> h;
  if (vis != nullptr) {
    vis->nodes += n_nodes;
    vis->tris += n_tris;
  }
  if (best_t >= 0) {
    const float* t = tris + 12 * best_t;
    F4 A = ld4(t), B = ld4(t + 4), Cc = ld4(t + 8);
    h.x = R(A.x) + (R(B.x) - R(A.x)) * bv + (R(Cc.x) - R(A.x)) * bw;
    h.y = R(A.y) + (R(B.y) - R(A.y)) * bv + (R(Cc.y) - R(A.y)) * bw;
    h.z = R(A.z) + (R(B.z) - R(A.z)) * bv + (R(Cc.z) - R(A.z)) * bw;
    h.d = exact ? w_sqrt(best) : w_sqrt(tau * best);
  } else if (!exact && best < R(INFINITY)) {
    // nothing inside the bound: its own boundary point (when known) is the best point
    h.x = pb ? pb[0] : R(NAN);
    h.y = pb ? pb[1] : R(NAN);
    h.z = pb ? pb[2] : R(NAN);
    h.d = w_sqrt(tau * best);
  } else {
    // no boundary point found at all (eight passes of overflowing stacks, or a non-finite
    // point): counted, and the walk ends here (distance 0, closest point x)
    if (vis != nullptr) ++vis->exhausted;
    h.x = x0;
    h.y = x1;
    h.z = x2;
    h.d = R(0);
  }
  return h;
}

// ---------------------------------------------------------------------------
// distance to the boundary (positive inside) and closest boundary point
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// signed-distance CSG (Sec. 7.2): exact primitive distances combined by min / max.
// Returns sdf(x) (negative inside) and the gradient of the active primitive.
// ---------------------------------------------------------------------------
template <int DIM, typename R>
WOS_HD R csg_prim(const CsgNode<R>& N, const R* x, R* g) {
  const R* p = N.p;
#pragma unroll
  for (int d = 0; d < 3; ++d) g[d] = R(0);
  switch (N.prim) {
    case C_SPHERE: {
      R v[3] = {R(0), R(0), R(0)}, r2 = R(0);
#pragma unroll
      for (int d = 0; d < DIM; ++d) { v[d] = x[d] - p[d]; r2 += v[d] * v[d]; }
      R r = w_sqrt(r2);
      R inv = (r > R(0)) ? R(1) / r : R(0);
      if (!(r > R(0))) g[0] = R(1);
#pragma unroll
      for (int d = 0; d < DIM; ++d) g[d] += v[d] * inv;
      return r - p[3];
    }
    case C_BOX: {
      R rc = p[6], q[3] = {R(0), R(0), R(0)}, sg[3] = {R(1), R(1), R(1)}, out2 = R(0), qmax = R(-1e30);
      int imax = 0;
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        R rel = x[d] - p[d];
        sg[d] = (rel >= R(0)) ? R(1) : R(-1);
        q[d] = w_fabs(rel) - (p[3 + d] - rc);
        if (q[d] > R(0)) out2 += q[d] * q[d];
        if (q[d] > qmax) { qmax = q[d]; imax = d; }
      }
      if (out2 > R(0)) {
        R od = w_sqrt(out2);
#pragma unroll
        for (int d = 0; d < DIM; ++d) g[d] = (q[d] > R(0)) ? sg[d] * q[d] / od : R(0);
        return od - rc;
      }
#pragma unroll
      for (int d = 0; d < DIM; ++d) if (d == imax) g[d] = sg[d];
      return qmax - rc;
    }
    case C_CAPSULE: {
      R ab[3] = {R(0), R(0), R(0)}, ax[3] = {R(0), R(0), R(0)}, l2 = R(0), t = R(0);
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        ab[d] = p[3 + d] - p[d];
        ax[d] = x[d] - p[d];
        l2 += ab[d] * ab[d];
        t += ab[d] * ax[d];
      }
      t = (l2 > R(0)) ? w_fmin(w_fmax(t / l2, R(0)), R(1)) : R(0);
      R v[3] = {R(0), R(0), R(0)}, r2 = R(0);
#pragma unroll
      for (int d = 0; d < DIM; ++d) { v[d] = ax[d] - t * ab[d]; r2 += v[d] * v[d]; }
      R r = w_sqrt(r2);
      R inv = (r > R(0)) ? R(1) / r : R(0);
      if (!(r > R(0))) g[0] = R(1);
#pragma unroll
      for (int d = 0; d < DIM; ++d) g[d] += v[d] * inv;
      return r - p[6];
    }
    case C_TORUS: {
      if (DIM == 2) {  // a ring: distance to the circle of radius p[3], minus p[4]
        R v0 = x[0] - p[0], v1 = x[1] - p[1];
        R rr = w_sqrt(v0 * v0 + v1 * v1);
        R q = rr - p[3];
        R s = (q >= R(0)) ? R(1) : R(-1);
        R inv = (rr > R(0)) ? R(1) / rr : R(0);
        g[0] = s * v0 * inv;
        g[1] = s * v1 * inv;
        if (!(rr > R(0))) g[0] = R(-1);
        return w_fabs(q) - p[4];
      }
      R v0 = x[0] - p[0], v1 = x[1] - p[1], v2 = x[2] - p[2];
      R rr = w_sqrt(v0 * v0 + v1 * v1);
      R q0 = rr - p[3], q1 = v2;
      R ql = w_sqrt(q0 * q0 + q1 * q1);
      R invr = (rr > R(0)) ? R(1) / rr : R(0);
      R invq = (ql > R(0)) ? R(1) / ql : R(0);
      g[0] = q0 * invq * v0 * invr;
      g[1] = q0 * invq * v1 * invr;
      g[2] = q1 * invq;
      return ql - p[4];
    }
    case C_HALFSPACE: {
      R s = R(0);
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        s += p[3 + d] * (x[d] - p[d]);
        g[d] = p[3 + d];
      }
      return s;
    }
    default:
      return R(1e30);
  }
}

template <int DIM, typename R>
WOS_HD R csg_sdf(const DevProblem<R>& P, const R* x, R* g) {
  R d = csg_prim<DIM, R>(P.csg[0], x, g);
  for (int i = 1; i < P.ncsg; ++i) {
    R gi[3];
    R s = csg_prim<DIM, R>(P.csg[i], x, gi);
    const int op = P.csg[i].op;
    if (op == C_SUBTRACT) {
      s = -s;
#pragma unroll
      for (int k = 0; k < 3; ++k) gi[k] = -gi[k];
    }
    const bool take = (op == C_UNION) ? (s < d) : (s > d);
    if (take) {
      d = s;
#pragma unroll
      for (int k = 0; k < 3; ++k) g[k] = gi[k];
    }
  }
  return d;
}

// bound2 (meshes only): an upper bound of the squared distance, see mesh_query.
// MESH = false compiles the mesh case out (for kernels launched on analytic domains).
// tau, pb, vis (meshes only): see mesh_query; tau = 1 returns the exact distance.
template <int DIM, typename R, bool MESH = true>
WOS_HD R distance(const DevProblem<R>& P, const R* x, R* xb, R bound2 = R(INFINITY), int* stk_n = nullptr,
                  R* stk_d = nullptr, int stk_stride = 0, R tau = R(1), const R* pb = nullptr,
                  MeshVisits* vis = nullptr, const float* top = nullptr) {
#if defined(WOS_JIT_DOMAIN_KIND)
  // a kernel compiled for one problem with an analytic domain: its kind and parameters are
  // constants of the generated source
  const R p[16] = WOS_JIT_DOMAIN_PARAMS;
  constexpr int kind = WOS_JIT_DOMAIN_KIND;
#else
  const R* p = P.dom;
  const int kind = P.domain_kind;
#endif
#pragma unroll
  for (int d = 0; d < 3; ++d) xb[d] = (d < DIM) ? x[d] : R(0);
  switch (kind) {
    case D_BOX: {
      R best = x[0] - p[0];
      int bd = 0;
      R bv = p[0];
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        R dl = x[d] - p[d], dh = p[3 + d] - x[d];
        if (dl < best) { best = dl; bd = d; bv = p[d]; }
        if (dh < best) { best = dh; bd = d; bv = p[3 + d]; }
      }
#pragma unroll
      for (int d = 0; d < DIM; ++d) if (d == bd) xb[d] = bv;
      return best;
    }
    case D_BALL:
    case D_ANNULUS: {
      R v[3] = {R(0), R(0), R(0)}, r2 = R(0);
#pragma unroll
      for (int d = 0; d < DIM; ++d) { v[d] = x[d] - p[d]; r2 += v[d] * v[d]; }
      R r = w_sqrt(r2);
      R dist, rad;
      if (kind == D_BALL) {
        dist = p[3] - r;
        rad = p[3];
      } else {
        R din = r - p[3], dout = p[4] - r;
        dist = (din < dout) ? din : dout;
        rad = (din < dout) ? p[3] : p[4];
      }
      if (r == R(0)) { v[0] = R(1); r = R(1); }
      R s = w_div(rad, r);
#pragma unroll
      for (int d = 0; d < DIM; ++d) xb[d] = p[d] + v[d] * s;
      return dist;
    }
    case D_ROUNDED_BOX: {
      R rc = p[6];
      R rel[3], inner[3], q[3];
      R out2 = R(0), qmax = R(-1e30);
      int imax = 0;
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        rel[d] = x[d] - p[d];
        inner[d] = p[3 + d] - rc;
        q[d] = w_fabs(rel[d]) - inner[d];
        if (q[d] > R(0)) out2 += q[d] * q[d];
        if (q[d] > qmax) { qmax = q[d]; imax = d; }
      }
      if (out2 > R(0)) {
        R od = w_sqrt(out2);
        R s = w_div(rc, od);
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          R c = w_fmin(w_fmax(rel[d], -inner[d]), inner[d]);
          xb[d] = p[d] + c + (rel[d] - c) * s;
        }
        return rc - od;
      }
#pragma unroll
      for (int d = 0; d < DIM; ++d)
        if (d == imax) xb[d] = p[d] + ((rel[d] >= R(0)) ? p[3 + d] : -p[3 + d]);
      return rc - qmax;
    }
    case D_CSG: {
      // ball radius -sdf (a lower bound of the distance); closest point along the gradient
      R g[3];
      R sd = csg_sdf<DIM, R>(P, x, g);
#pragma unroll
      for (int d = 0; d < DIM; ++d) xb[d] = x[d] - sd * g[d];
      return -sd;
    }
    case D_MESH: {
      if (DIM != 3 || !MESH) return R(-1);
      if (P.mg_res > 0) {
        // distance grid: lower bound max_c (d(c) - |x - c|), upper bound min_c (d(c) + |x - c|)
        int i0[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          R sg = floor((x[d] - P.mg_lo[d]) * P.mg_inv_h[d]);
          int i = (int)w_fmin(w_fmax(sg, R(0)), R(P.mg_res - 2));
          i0[d] = i;
        }
        R lo_b = R(-INFINITY), hi_b = R(INFINITY);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          int ii = i0[0] + (c & 1), jj = i0[1] + ((c >> 1) & 1), kk = i0[2] + ((c >> 2) & 1);
          R e0 = x[0] - (P.mg_lo[0] + R(ii) * P.mg_h[0]);
          R e1 = x[1] - (P.mg_lo[1] + R(jj) * P.mg_h[1]);
          R e2 = x[2] - (P.mg_lo[2] + R(kk) * P.mg_h[2]);
          R dist = w_sqrt(e0 * e0 + e1 * e1 + e2 * e2);
          R dc = P.mgrid[ii + (int64_t)P.mg_res * (jj + (int64_t)P.mg_res * kk)];
          lo_b = w_fmax(lo_b, dc - dist);
          hi_b = w_fmin(hi_b, dc + dist);
        }
        if (lo_b >= P.mg_thresh) {
          // the walk is not in the shell; no boundary point is known (NaN: the next step's
          // query starts without a bound)
          xb[0] = xb[1] = xb[2] = R(NAN);
          return lo_b;
        }
        if (hi_b * hi_b < bound2) {
          bound2 = hi_b * hi_b;
          pb = nullptr;  // the grid's bound has no boundary point of its own
        }
      }
      MeshHit<R> h = (stk_n != nullptr)
                         ? mesh_query<R, true>(P, x[0], x[1], x[2], bound2, stk_n, stk_d, stk_stride, tau, pb, vis,
                                               top)
                         : mesh_query<R, false>(P, x[0], x[1], x[2], bound2, nullptr, nullptr, 0, tau, pb, vis, top);
      xb[0] = h.x;
      xb[1] = h.y;
      xb[2] = h.z;
      return h.d;
    }
    default:
      return R(-1);
  }
}

}  // namespace wos
