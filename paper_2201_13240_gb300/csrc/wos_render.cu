// wos_render.cu -- headless view of a progressive solve on a slice plane (Sec. 7.2:
// signed-distance geometry rendered by sphere tracing, the solution shown on a slice
// plane and refined by accumulating one walk per point per frame).
//
// wos_slice_points lays the slice grid out (cell centres of an nu x nv grid on the
// plane rectangle); the walks run through the ordinary solve entry points and add to
// per-point accumulators; wos_render_slice then draws, per pixel, a pinhole ray that
// is sphere-traced against the domain clipped by the slice plane (the part of the
// domain on the camera's side of the plane is cut away).  A ray that reaches the
// plane inside the domain shows the accumulated mean of its slice cell through a
// colour map; a ray that reaches the boundary shows g there, shaded by the surface
// normal.  2D problems show the slice grid directly (the plane is the domain's own
// plane).  The output is an RGBA8 image in device memory, plus optional per-pixel
// value (NaN off the slice) and ray depth (INFINITY on a miss) buffers.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <cmath>

#include "wos.h"
#include "wos_math.cuh"
#include "wos_problem.cuh"

namespace wos {
namespace {

struct View3 {
  double eye[3], fwd[3], right[3], up[3];
  double tan_half;
  double org[3], pu[3], pv[3], n[3];  // plane rectangle and its normal (towards the eye)
  double pu2, pv2;
  double lo, hi;
  double scale;                        // size of the domain box, for tolerances
  int nu, nv, width, height;
};

__device__ double sd_domain(const DevProblem<double>& P, const double* x) {
  double xb[3];
  return -distance<3, double, false>(P, x, xb);  // signed distance, negative inside
}

__device__ void colour_map(double t, double* c) {
  // a blue - white - red map on [0, 1]
  t = fmin(fmax(t, 0.0), 1.0);
  if (t < 0.5) {
    double s = t * 2.0;
    c[0] = 0.23 + 0.77 * s; c[1] = 0.30 + 0.70 * s; c[2] = 0.75 + 0.25 * s;
  } else {
    double s = (t - 0.5) * 2.0;
    c[0] = 1.0 - 0.29 * s; c[1] = 1.0 - 0.98 * s; c[2] = 1.0 - 0.85 * s;
  }
}

__device__ void put(uint8_t* rgba, int64_t i, const double* c) {
  for (int k = 0; k < 3; ++k) rgba[4 * i + k] = (uint8_t)fmin(255.0, fmax(0.0, c[k] * 255.0 + 0.5));
  rgba[4 * i + 3] = 255;
}

__global__ void render3_kernel(const DevProblem<double>* Pg, View3 V, const double* sum, const int64_t* count,
                               uint8_t* rgba, float* value, float* depth) {
  const DevProblem<double>& P = *Pg;
  int64_t npx = (int64_t)V.width * V.height;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npx; i += (int64_t)gridDim.x * blockDim.x) {
    int px = (int)(i % V.width), py = (int)(i / V.width);
    double sx = ((px + 0.5) / V.width * 2.0 - 1.0) * V.tan_half * V.width / V.height;
    double sy = (1.0 - (py + 0.5) / V.height * 2.0) * V.tan_half;
    double dir[3], nd = 0.0;
    for (int k = 0; k < 3; ++k) {
      dir[k] = V.fwd[k] + sx * V.right[k] + sy * V.up[k];
      nd += dir[k] * dir[k];
    }
    nd = sqrt(nd);
    for (int k = 0; k < 3; ++k) dir[k] /= nd;
    double c[3] = {0.08, 0.08, 0.10};
    float val = NAN, dep = INFINITY;
    // sphere-trace max(sdf_domain, sdf_keep): the domain behind the plane
    double t = 0.0, tmax = 1e3 * V.scale;
    const double tol = 1e-5 * V.scale;
    for (int it = 0; it < 512 && t < tmax; ++it) {
      double x[3];
      for (int k = 0; k < 3; ++k) x[k] = V.eye[k] + t * dir[k];
      double sd = sd_domain(P, x);
      double sp = 0.0;  // > 0 on the eye's side of the plane: cut away
      for (int k = 0; k < 3; ++k) sp += V.n[k] * (x[k] - V.org[k]);
      double s = fmax(sd, sp);
      if (s < tol) {
        dep = (float)t;
        if (sp >= sd) {
          // on the slice plane, inside the domain
          double r[3], a = 0.0, b = 0.0;
          for (int k = 0; k < 3; ++k) r[k] = x[k] - V.org[k];
          for (int k = 0; k < 3; ++k) { a += r[k] * V.pu[k]; b += r[k] * V.pv[k]; }
          a /= V.pu2;
          b /= V.pv2;
          if (a >= 0.0 && a < 1.0 && b >= 0.0 && b < 1.0) {
            int iu = min((int)(a * V.nu), V.nu - 1), iv = min((int)(b * V.nv), V.nv - 1);
            int64_t cell = (int64_t)iv * V.nu + iu;
            int64_t n = count[cell];
            if (n > 0) {
              double u = sum[cell] / (double)n;
              val = (float)u;
              colour_map((u - V.lo) / (V.hi - V.lo), c);
            } else {
              c[0] = c[1] = c[2] = 0.35;
            }
          } else {
            c[0] = c[1] = c[2] = 0.25;
          }
        } else {
          // boundary: g there, Lambert-shaded by the normal of the signed distance
          double h = 1e-4 * V.scale, g[3];
          for (int k = 0; k < 3; ++k) {
            double xp[3] = {x[0], x[1], x[2]}, xm[3] = {x[0], x[1], x[2]};
            xp[k] += h;
            xm[k] -= h;
            g[k] = sd_domain(P, xp) - sd_domain(P, xm);
          }
          double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]) + 1e-300;
          double lam = 0.0;
          for (int k = 0; k < 3; ++k) lam -= g[k] / gn * dir[k];
          lam = 0.25 + 0.75 * fmax(lam, 0.0);
          double gv = field_eval<3>(P, P.g, x[0], x[1], x[2], false).v;
          colour_map((gv - V.lo) / (V.hi - V.lo), c);
          for (int k = 0; k < 3; ++k) c[k] *= lam;
        }
        break;
      }
      t += fmax(s, tol);
    }
    put(rgba, i, c);
    if (value) value[i] = val;
    if (depth) depth[i] = dep;
  }
}

__global__ void render2_kernel(const DevProblem<double>* Pg, double o0, double o1, double u0, double v1, int nu,
                               int nv, int width, int height, double lo, double hi, const double* sum,
                               const int64_t* count, uint8_t* rgba, float* value) {
  const DevProblem<double>& P = *Pg;
  int64_t npx = (int64_t)width * height;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npx; i += (int64_t)gridDim.x * blockDim.x) {
    int px = (int)(i % width), py = (int)(i / width);
    double a = (px + 0.5) / width, b = 1.0 - (py + 0.5) / height;
    double x[3] = {o0 + a * u0, o1 + b * v1, 0.0}, xb[3];
    double c[3] = {0.08, 0.08, 0.10};
    float val = NAN;
    if (distance<2, double, false>(P, x, xb) > 0.0) {
      int iu = min((int)(a * nu), nu - 1), iv = min((int)(b * nv), nv - 1);
      int64_t cell = (int64_t)iv * nu + iu;
      int64_t n = count[cell];
      if (n > 0) {
        double u = sum[cell] / (double)n;
        val = (float)u;
        colour_map((u - lo) / (hi - lo), c);
      } else {
        c[0] = c[1] = c[2] = 0.35;
      }
    }
    put(rgba, i, c);
    if (value) value[i] = val;
  }
}

__global__ void slice_points_kernel(int dim, View3 V, float* pts) {
  int64_t n = (int64_t)V.nu * V.nv;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double a = ((i % V.nu) + 0.5) / V.nu, b = ((i / V.nu) + 0.5) / V.nv;
    for (int k = 0; k < dim; ++k) pts[(int64_t)k * n + i] = (float)(V.org[k] + a * V.pu[k] + b * V.pv[k]);
  }
}

double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
bool normalise(double* a) {
  double n = sqrt(dot3(a, a));
  if (!(n > 0.0) || !std::isfinite(n)) return false;
  for (int k = 0; k < 3; ++k) a[k] /= n;
  return true;
}

bool make_view(const wos_view* v, int dim, View3* V) {
  for (int k = 0; k < 3; ++k) {
    V->org[k] = v->plane_origin[k];
    V->pu[k] = v->plane_u[k];
    V->pv[k] = v->plane_v[k];
  }
  if (dim == 2) {
    V->pu[1] = V->pu[2] = 0.0;
    V->pv[0] = V->pv[2] = 0.0;
    V->org[2] = 0.0;
  }
  V->pu2 = dot3(V->pu, V->pu);
  V->pv2 = dot3(V->pv, V->pv);
  V->nu = v->slice_nu;
  V->nv = v->slice_nv;
  V->width = v->width;
  V->height = v->height;
  V->lo = v->value_lo;
  V->hi = v->value_hi;
  if (!(V->pu2 > 0.0) || !(V->pv2 > 0.0) || V->nu < 1 || V->nv < 1) return false;
  if (dim == 2) return true;
  cross3(V->pu, V->pv, V->n);
  if (!normalise(V->n)) return false;
  for (int k = 0; k < 3; ++k) {
    V->eye[k] = v->eye[k];
    V->fwd[k] = v->look[k] - v->eye[k];
  }
  if (!normalise(V->fwd)) return false;
  double up[3] = {v->up[0], v->up[1], v->up[2]};
  cross3(V->fwd, up, V->right);
  if (!normalise(V->right)) return false;
  cross3(V->right, V->fwd, V->up);
  V->tan_half = tan(0.5 * v->fov_y_deg * 3.14159265358979323846 / 180.0);
  if (!(V->tan_half > 0.0) || !std::isfinite(V->tan_half)) return false;
  // the plane normal points to the eye's side (that half is cut away)
  double r[3];
  for (int k = 0; k < 3; ++k) r[k] = V->eye[k] - V->org[k];
  if (dot3(r, V->n) < 0.0)
    for (int k = 0; k < 3; ++k) V->n[k] = -V->n[k];
  return true;
}

}  // namespace

int render_slice(const DevProblem<double>* dprob, const DevProblem<double>& host, int dim, const wos_view* view,
                 const double* sum, const int64_t* count, uint8_t* rgba, float* value, float* depth, int num_sms,
                 cudaStream_t st) {
  View3 V;
  if (!make_view(view, dim, &V)) return WOS_EINVAL;
  if (V.width < 1 || V.height < 1 || !(V.hi > V.lo)) return WOS_EINVAL;
  int64_t npx = (int64_t)V.width * V.height;
  int blocks = (int)((npx + 255) / 256);
  if (blocks > num_sms * 16) blocks = num_sms * 16;
  if (dim == 2) {
    render2_kernel<<<blocks, 256, 0, st>>>(dprob, V.org[0], V.org[1], V.pu[0], V.pv[1], V.nu, V.nv, V.width,
                                           V.height, V.lo, V.hi, sum, count, rgba, value);
  } else {
    double span2 = 0.0;
    for (int k = 0; k < 3; ++k) span2 += (host.dom[3 + k] - host.dom[k]) * (host.dom[3 + k] - host.dom[k]);
    V.scale = sqrt(span2) > 0.0 ? sqrt(span2) : 1.0;
    render3_kernel<<<blocks, 256, 0, st>>>(dprob, V, sum, count, rgba, value, depth);
  }
  return cudaGetLastError() == cudaSuccess ? WOS_OK : WOS_ECUDA;
}

int slice_points(int dim, const wos_view* view, float* pts, int num_sms, cudaStream_t st) {
  View3 V;
  if (!make_view(view, dim, &V)) return WOS_EINVAL;
  int64_t n = (int64_t)V.nu * V.nv;
  int blocks = (int)((n + 255) / 256);
  if (blocks > num_sms * 16) blocks = num_sms * 16;
  slice_points_kernel<<<blocks, 256, 0, st>>>(dim, V, pts);
  return cudaGetLastError() == cudaSuccess ? WOS_OK : WOS_ECUDA;
}

}  // namespace wos
