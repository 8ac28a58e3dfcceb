// wos_capi.cu -- implementation of the C interface declared in include/wos.h:
// context and problem lifetime, validation, the sigma_bar prepass, the walk
// launches, the finalize kernel and the host-buffer convenience entry point.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "wos.h"
#include "wos_internal.h"
#include "wos_mesh.h"
#include "wos_jit.h"
#include "wos_problem.cuh"

#include "wos_capi_state.h"

namespace {

constexpr int kScratchWords = 64;
constexpr int kScratchStats = 8;
constexpr int kScratchSigma = 24;

int fail(wos_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

int cuda_fail(wos_ctx* ctx, cudaError_t e, const char* what) {
  return fail(ctx, WOS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

struct DeviceGuard {
  int prev = -1;
  // errors of these calls are reported by the calls that follow; they are cleared here so
  // that they do not surface later in the caller's own CUDA error checks
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      prev = -1;
      (void)cudaGetLastError();
    }
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) (void)cudaGetLastError();
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev && cudaSetDevice(prev) != cudaSuccess)
      (void)cudaGetLastError();
  }
};

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

int check_field(const wos_field_desc& f, int dim, const char* name, bool is_source, bool needs_c2,
                std::string* why) {
  if (f.kind < WOS_FIELD_ZERO || f.kind > WOS_FIELD_GRID_BSPLINE) {
    *why = std::string(name) + ": unknown field kind";
    return WOS_EINVAL;
  }
  if (f.kind == WOS_FIELD_MANUFACTURED && !is_source) {
    *why = std::string(name) + ": only the source may be MANUFACTURED";
    return WOS_EINVAL;
  }
  if (needs_c2 && f.kind == WOS_FIELD_GRID_LINEAR) {
    *why = std::string(name) + ": needs a Laplacian; use CONST, SST or GRID_BSPLINE";
    return WOS_EINVAL;
  }
  if (f.kind == WOS_FIELD_SST) {
    if (f.nterms < 0 || f.nterms > wos::kMaxTerms || (f.nterms > 0 && f.terms == nullptr)) {
      *why = std::string(name) + ": bad term count or null terms";
      return WOS_EINVAL;
    }
    for (int n = 0; n < f.nterms; ++n) {
      const wos_term& t = f.terms[n];
      if (!std::isfinite(t.c)) { *why = std::string(name) + ": non-finite coefficient"; return WOS_EINVAL; }
      for (int d = 0; d < dim; ++d) {
        if (t.type[d] < WOS_ATOM_ONE || t.type[d] > WOS_ATOM_QUAD || !std::isfinite(t.k[d]) ||
            !std::isfinite(t.phi[d])) {
          *why = std::string(name) + ": bad atom";
          return WOS_EINVAL;
        }
      }
    }
  }
  if (f.kind == WOS_FIELD_CONST && !std::isfinite(f.value)) {
    *why = std::string(name) + ": non-finite constant";
    return WOS_EINVAL;
  }
  if (f.kind == WOS_FIELD_GRID_LINEAR || f.kind == WOS_FIELD_GRID_BSPLINE) {
    if (f.data == nullptr) { *why = std::string(name) + ": null grid data"; return WOS_EINVAL; }
    for (int d = 0; d < dim; ++d) {
      if (f.res[d] < 2 || !(f.hi[d] > f.lo[d]) || !std::isfinite(f.lo[d]) || !std::isfinite(f.hi[d])) {
        *why = std::string(name) + ": grid needs res >= 2 and hi > lo on every axis";
        return WOS_EINVAL;
      }
    }
  }
  return WOS_OK;
}

// every field of a description (the domain is checked by the caller)
int check_fields(const wos_problem_desc& d, bool* drift, std::string* why) {
  struct { const wos_field_desc* f; const char* n; bool src; bool c2; } fl[6] = {
      {&d.alpha, "alpha", false, true}, {&d.phi, "phi", false, true}, {&d.sigma, "sigma", false, false},
      {&d.f, "f", true, false},         {&d.g, "g", false, false},    {&d.um, "um", false, true}};
  int total_terms = 0;
  for (auto& x : fl) {
    if (check_field(*x.f, d.dim, x.n, x.src, x.c2, why) != WOS_OK) return WOS_EINVAL;
    if (x.f->kind == WOS_FIELD_SST) total_terms += x.f->nterms;
  }
  *drift = false;
  for (int k = 0; k < d.dim; ++k) {
    if (check_field(d.omega[k], d.dim, "omega", false, true, why) != WOS_OK) return WOS_EINVAL;
    if (d.omega[k].kind == WOS_FIELD_SST) total_terms += d.omega[k].nterms;
    if (d.omega[k].kind != WOS_FIELD_ZERO) *drift = true;
  }
  if (d.alpha.kind == WOS_FIELD_ZERO || (d.alpha.kind == WOS_FIELD_CONST && !(d.alpha.value > 0))) {
    *why = "alpha must be > 0";
    return WOS_EINVAL;
  }
  if (total_terms > wos::kMaxTerms) {
    *why = "more than 96 separable terms in total";
    return WOS_EINVAL;
  }
  return WOS_OK;
}

template <typename R>
void fill_field(DevProblem<R>& P, DevField<R>& F, const wos_field_desc& f, int dim) {
  std::memset(&F, 0, sizeof(F));
  F.kind = f.kind;
  F.value = R(f.value);
  F.first = P.nterms;
  if (f.kind == WOS_FIELD_SST) {
    F.nterms = f.nterms;
    for (int n = 0; n < f.nterms; ++n) {
      DevTerm<R>& T = P.terms[P.nterms++];
      T.c = R(f.terms[n].c);
      for (int d = 0; d < 3; ++d) {
        bool on = d < dim;
        T.type[d] = on ? f.terms[n].type[d] : wos::A_ONE;
        T.k[d] = on ? R(f.terms[n].k[d]) : R(0);
        T.phi[d] = on ? R(f.terms[n].phi[d]) : R(0);
      }
    }
  }
  if (f.kind == WOS_FIELD_GRID_LINEAR || f.kind == WOS_FIELD_GRID_BSPLINE) {
    for (int d = 0; d < 3; ++d) {
      F.res[d] = d < dim ? f.res[d] : 1;
      F.lo[d] = d < dim ? R(f.lo[d]) : R(0);
      F.inv_h[d] = d < dim ? R((f.res[d] - 1) / (f.hi[d] - f.lo[d])) : R(0);
    }
    F.data = f.data;
  }
}

template <typename R>
void fill_problem(DevProblem<R>& P, const wos_problem_desc& d) {
  std::memset(&P, 0, sizeof(P));
  P.dim = d.dim;
  P.domain_kind = d.domain.kind;
  for (int i = 0; i < 16; ++i) P.dom[i] = R(d.domain.p[i]);
  if (d.domain.kind == WOS_DOMAIN_CSG && d.domain.csg) {
    P.ncsg = d.domain.ncsg;
    for (int i = 0; i < d.domain.ncsg && i < wos::kMaxCsg; ++i) {
      const wos_csg_node& n = d.domain.csg[i];
      P.csg[i].prim = n.prim;
      P.csg[i].op = n.op;
      double q[8];
      for (int k = 0; k < 8; ++k) q[k] = n.p[k];
      if (n.prim == WOS_CSG_HALFSPACE) {  // unit normal
        double nn = 0;
        for (int k = 0; k < d.dim; ++k) nn += q[3 + k] * q[3 + k];
        nn = std::sqrt(nn);
        for (int k = 0; k < 3; ++k) q[3 + k] = (k < d.dim) ? q[3 + k] / nn : 0.0;
      }
      for (int k = 0; k < 8; ++k) P.csg[i].p[k] = R(q[k]);
    }
  }
  P.mesh_tau = R(1);
  if (d.domain.kind == WOS_DOMAIN_MESH) P.mesh_tau = R((1.0 - d.domain.mesh_tol) * (1.0 - d.domain.mesh_tol));
  fill_field(P, P.alpha, d.alpha, d.dim);
  fill_field(P, P.phi, d.phi, d.dim);
  fill_field(P, P.sigma, d.sigma, d.dim);
  fill_field(P, P.f, d.f, d.dim);
  fill_field(P, P.g, d.g, d.dim);
  fill_field(P, P.um, d.um, d.dim);
  P.has_drift = 0;
  P.drift_bound = R(d.drift_bound);
  for (int k = 0; k < 3; ++k) {
    if (k < d.dim) {
      fill_field(P, P.omega[k], d.omega[k], d.dim);
      if (d.omega[k].kind != WOS_FIELD_ZERO) P.has_drift = 1;
    } else {
      P.omega[k].kind = wos::F_ZERO;
    }
  }
}

void domain_bbox(const wos_problem* pr, double lo[3], double hi[3]) {
  const DevProblem<double>& P = pr->host64;
  if (P.domain_kind == wos::D_MESH) {
    for (int d = 0; d < 3; ++d) { lo[d] = pr->mesh_lo[d]; hi[d] = pr->mesh_hi[d]; }
    return;
  }
  const double* p = P.dom;
  for (int d = 0; d < 3; ++d) { lo[d] = 0.0; hi[d] = 0.0; }
  for (int d = 0; d < P.dim; ++d) {
    switch (P.domain_kind) {
      case wos::D_BOX:
      case wos::D_CSG: lo[d] = p[d]; hi[d] = p[3 + d]; break;
      case wos::D_BALL: lo[d] = p[d] - p[3]; hi[d] = p[d] + p[3]; break;
      case wos::D_ANNULUS: lo[d] = p[d] - p[4]; hi[d] = p[d] + p[4]; break;
      case wos::D_ROUNDED_BOX: lo[d] = p[d] - p[3 + d]; hi[d] = p[d] + p[3 + d]; break;
    }
  }
}

// ---------------------------------------------------------------------------
// kernels: sigma' range on a lattice, prefix sums of walks, finalize
// ---------------------------------------------------------------------------
__device__ void atomic_min_d(double* addr, double v) {
  unsigned long long* p = reinterpret_cast<unsigned long long*>(addr);
  unsigned long long old = *p;
  for (int it = 0; it < (1 << 20) && v < __longlong_as_double(old); ++it) {
    unsigned long long prev = atomicCAS(p, old, __double_as_longlong(v));
    if (prev == old) break;
    old = prev;
  }
}
__device__ void atomic_max_d(double* addr, double v) {
  unsigned long long* p = reinterpret_cast<unsigned long long*>(addr);
  unsigned long long old = *p;
  for (int it = 0; it < (1 << 20) && v > __longlong_as_double(old); ++it) {
    unsigned long long prev = atomicCAS(p, old, __double_as_longlong(v));
    if (prev == old) break;
    old = prev;
  }
}

// exact distances to the mesh at the nodes of an n^3 grid (FP64 queries)
__global__ void mesh_grid_kernel(const DevProblem<double>* Pg, int n, double lo0, double lo1, double lo2, double h0,
                                 double h1, double h2, double* out64, float* out32) {
  const DevProblem<double>& P = *Pg;
  int64_t total = (int64_t)n * n * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    double x0 = lo0 + (double)(i % n) * h0, x1 = lo1 + (double)((i / n) % n) * h1,
           x2 = lo2 + (double)(i / ((int64_t)n * n)) * h2;
    wos::MeshHit<double> hit = wos::mesh_query<double, false>(P, x0, x1, x2, INFINITY, nullptr, nullptr, 0);
    out64[i] = hit.d;
    out32[i] = (float)hit.d;
  }
}

template <int DIM>
__global__ void sigma_range_kernel(const DevProblem<double>* Pg, int m, double lo0, double lo1, double lo2,
                                   double h0, double h1, double h2,
                                   double* out /* min, max, alpha_min, count, max |omega/alpha|^2 */) {
  const DevProblem<double>& P = *Pg;
  int64_t total = (DIM == 3) ? (int64_t)m * m * m : (int64_t)m * m;
  double mn = INFINITY, mx = -INFINITY, amin = INFINITY, cnt = 0.0, b2max = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    double x[3] = {lo0 + (i % m + 0.5) * h0, lo1 + ((i / m) % m + 0.5) * h1,
                   DIM == 3 ? lo2 + (i / ((int64_t)m * m) + 0.5) * h2 : 0.0};
    double xb[3];
    if (!(wos::distance<DIM>(P, x, xb) > 0.0)) continue;
    double sp, fp;
    if (P.has_drift) wos::coeffs<DIM, double, true>(P, x, &sp, &fp);
    else wos::coeffs<DIM>(P, x, &sp, &fp);
    double a = wos::field_eval<DIM>(P, P.alpha, x[0], x[1], x[2], false).v;
    mn = fmin(mn, sp);
    mx = fmax(mx, sp);
    amin = fmin(amin, a);
    cnt += 1.0;
    if (P.has_drift) {
      double b2 = 0.0;
      for (int d = 0; d < DIM; ++d) {
        double w = wos::field_eval<DIM>(P, P.omega[d], x[0], x[1], x[2], false).v / a;
        b2 += w * w;
      }
      b2max = fmax(b2max, b2);
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    mn = fmin(mn, __shfl_down_sync(0xffffffffu, mn, off));
    mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, off));
    amin = fmin(amin, __shfl_down_sync(0xffffffffu, amin, off));
    cnt += __shfl_down_sync(0xffffffffu, cnt, off);
    b2max = fmax(b2max, __shfl_down_sync(0xffffffffu, b2max, off));
  }
  if ((threadIdx.x & 31) == 0 && cnt > 0.0) {
    atomic_min_d(&out[0], mn);
    atomic_max_d(&out[1], mx);
    atomic_min_d(&out[2], amin);
    atomicAdd(&out[3], cnt);
    atomic_max_d(&out[4], b2max);
  }
}

// inclusive prefix sums of max(walks, 0): one block, sequential over tiles of 1024
__global__ void walk_prefix_kernel(const int32_t* walks, int64_t n, int64_t* out) {
  __shared__ int64_t tile[1024];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < n; base += 1024) {
    int64_t i = base + threadIdx.x;
    int64_t v = (i < n) ? (int64_t)max(walks[i], 0) : 0;
    tile[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
      int64_t add = (threadIdx.x >= (unsigned)off) ? tile[threadIdx.x - off] : 0;
      __syncthreads();
      tile[threadIdx.x] += add;
      __syncthreads();
    }
    if (i < n) out[i] = tile[threadIdx.x] + carry;
    __syncthreads();
    if (threadIdx.x == 1023) carry += tile[1023];
    __syncthreads();
  }
}

// FP64 inverse radial CDF on the (a, u) grid of the FP32 Newton start table
template <int DIM>
__global__ void radial_table_kernel(float* tab) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= wos::kTabSize) return;
  int ia = i / wos::kTabU, iu = i % wos::kTabU;
  double a = ia * (double)wos::kTabDA, u = wos::tab_u_of_t((double)iu / (wos::kTabU - 1));
  double r = (iu == 0) ? 0.0 : (iu == wos::kTabU - 1) ? 1.0 : wos::sample_radius<DIM, double>(a, u);
  tab[i] = (float)r;
}

__global__ void finalize_kernel(const double* sum, const double* sumsq, const int64_t* count, int64_t n,
                                double* mean, double* var, double* se) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double c = (double)count[i];
    double m = sum[i] / c;
    double v = (sumsq[i] - c * m * m) / fmax(c - 1.0, 1.0);
    v = fmax(v, 0.0);
    if (mean) mean[i] = m;
    if (var) var[i] = v;
    if (se) se[i] = sqrt(v / c);
  }
}

// The FP32 Newton start table of one dimension, built (in FP64, tens of ms) when the
// first problem of that dimension is created, so that a context used for 3D problems
// only never pays for the 2D table.  Problem creation allocates and synchronises anyway;
// every later launch on any stream finds the table complete.
int ensure_radial_table(wos_ctx* ctx, int dim) {
  float*& tab = ctx->radial_tab[dim - 2];
  if (tab != nullptr) return WOS_OK;
  float* t = nullptr;
  cudaError_t e = cudaMalloc(&t, wos::kTabSize * sizeof(float));
  if (e != cudaSuccess) return fail(ctx, WOS_ENOMEM, std::string("cudaMalloc(radial table): ") + cudaGetErrorString(e));
  const int blocks = (wos::kTabSize + 127) / 128;
  if (dim == 2) radial_table_kernel<2><<<blocks, 128>>>(t);
  else radial_table_kernel<3><<<blocks, 128>>>(t);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaFree(t);
    return cuda_fail(ctx, e, "radial table kernel");
  }
  tab = t;
  return WOS_OK;
}

int validate_params(wos_ctx* ctx, const wos_params* prm) {
  if (!prm) return fail(ctx, WOS_EINVAL, "params is NULL");
  if (!finite_pos(prm->eps)) return fail(ctx, WOS_EINVAL, "eps must be finite and > 0");
  if (!finite_pos(prm->sigma_bar)) return fail(ctx, WOS_EINVAL, "sigma_bar must be finite and > 0");
  if (prm->max_steps < 1) return fail(ctx, WOS_EINVAL, "max_steps must be >= 1");
  if (prm->precision != WOS_FP32 && prm->precision != WOS_FP64)
    return fail(ctx, WOS_EINVAL, "precision must be WOS_FP32 or WOS_FP64");
  if (prm->ww_lo != 0.0) {
    if (!finite_pos(prm->ww_lo) || !(std::isfinite(prm->ww_hi) && prm->ww_hi > prm->ww_lo))
      return fail(ctx, WOS_EINVAL, "weight window needs 0 < ww_lo < ww_hi");
    if (prm->ww_depth < 1 || prm->ww_depth > 8) return fail(ctx, WOS_EINVAL, "ww_depth must be in 1..8");
  }
  return WOS_OK;
}

int no_window(wos_ctx* ctx, const wos_params* prm) {
  if (prm && prm->ww_lo != 0.0) return fail(ctx, WOS_EUNSUPPORTED, "this entry point has no weight window");
  return WOS_OK;
}

int launch(wos_ctx* ctx, const wos_problem* prob, const float* pts, int64_t npts, const int64_t* walk_end,
           int64_t walks_uniform, uint64_t total, const wos_params* prm, double* sum, double* sumsq,
           int64_t* count, uint64_t* stats, double* uhat, int64_t* steps, cudaStream_t st,
           double* gsum = nullptr, double* gsumsq = nullptr, double* ghat = nullptr, int64_t nf_max_inner = 0,
           int32_t nf_series = 0) {
  cudaError_t e = cudaMemsetAsync(ctx->scratch, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemsetAsync(work counter)");
  unsigned long long* st_ptr = reinterpret_cast<unsigned long long*>(stats);
  if (st_ptr == nullptr) {
    st_ptr = ctx->scratch + kScratchStats;
    e = cudaMemsetAsync(st_ptr, 0, wos::ST_WORDS * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemsetAsync(stats)");
  }
  wos::WalkLaunch L;
  std::memset(&L, 0, sizeof(L));
  L.dim = prob->dim;
  L.pts = pts;
  L.npts = npts;
  L.walk_end = walk_end;
  L.walks_uniform = walks_uniform;
  L.total_items = total;
  L.seed = prm->seed;
  L.walk_offset = prm->walk_offset;
  L.eps = prm->eps;
  L.sigma_bar = prm->sigma_bar;
  L.max_steps = prm->max_steps;
  L.sum = sum;
  L.sumsq = sumsq;
  L.count = reinterpret_cast<unsigned long long*>(count);
  L.stats = st_ptr;
  L.work_counter = ctx->scratch;
  L.uhat = uhat;
  L.steps_out = steps;
  L.radial_tab = ctx->radial_tab[prob->dim - 2];
  L.mesh = prob->host64.domain_kind == wos::D_MESH;
  L.ww_lo = prm->ww_lo;
  L.ww_hi = prm->ww_hi;
  L.ww_depth = prm->ww_depth;
  L.gsum = gsum;
  L.gsumsq = gsumsq;
  L.ghat = ghat;
  L.nf_max_inner = nf_max_inner;
  L.nf_series = nf_series;
  L.drift = prob->host64.has_drift;
  const bool nf = nf_max_inner > 0;
  if (L.drift && (nf || gsum || ghat || prm->ww_lo != 0.0))
    return fail(ctx, WOS_EUNSUPPORTED, "an extra drift (omega) works with the plain solve only");
  const bool fp64 = prm->precision == WOS_FP64;
  const int variant = (gsum || ghat) ? wos::kJitGrad : (prm->ww_lo != 0.0 ? wos::kJitWindow : wos::kJitPlain);
  cudaKernel_t spec = nf ? nullptr : prob->jit.kernel[fp64 ? 1 : 0][variant];
  if (spec != nullptr) {
    // the walk kernel compiled for this problem's fields
    L.problem = fp64 ? (const void*)prob->d64 : (const void*)prob->d32;
    L.problem_bytes = fp64 ? (int)sizeof(DevProblem<double>) : (int)sizeof(DevProblem<float>);
    e = wos::launch_walks_kernel(L, spec, fp64 ? 8 : 4, ctx->num_sms, st);
  } else if (fp64) {
    L.problem = prob->d64;
    L.problem_bytes = (int)sizeof(DevProblem<double>);
    e = nf ? wos::launch_nf_f64(L, ctx->num_sms, st) : wos::launch_walks_f64(L, ctx->num_sms, st);
  } else {
    L.problem = prob->d32;
    L.problem_bytes = (int)sizeof(DevProblem<float>);
    e = nf ? wos::launch_nf_f32(L, ctx->num_sms, st) : wos::launch_walks_f32(L, ctx->num_sms, st);
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "walk kernel launch");
  return WOS_OK;
}

template <typename T>
int grow(wos_ctx* ctx, T** buf, int64_t n, int64_t* cap, int64_t need) {
  if (need <= *cap) return WOS_OK;
  if (*buf) cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(buf), sizeof(T) * (size_t)(n > 0 ? n : 1));
  if (e != cudaSuccess) return fail(ctx, WOS_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  *cap = need;
  return WOS_OK;
}

}  // namespace

static_assert(sizeof(DevProblem<float>) % 16 == 0, "problem size must be a multiple of 16 bytes");
static_assert(sizeof(DevProblem<double>) % 16 == 0, "problem size must be a multiple of 16 bytes");

extern "C" {

const char* wos_version(void) { return "wos-gb300 0.1 (sm_103a)"; }

int wos_create(wos_ctx** out, int device) {
  if (!out) return WOS_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return WOS_ECUDA;
  wos_ctx* ctx = new wos_ctx();
  ctx->device = device;
  DeviceGuard g(device);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    delete ctx;
    return WOS_ECUDA;
  }
  ctx->num_sms = prop.multiProcessorCount;
  if (cudaMalloc(&ctx->scratch, kScratchWords * sizeof(unsigned long long)) != cudaSuccess) {
    delete ctx;
    return WOS_ENOMEM;
  }
  if (cudaMemset(ctx->scratch, 0, kScratchWords * sizeof(unsigned long long)) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    wos_destroy(ctx);
    return WOS_ECUDA;
  }
  // the FP32 radial start tables are built by the first problem of each dimension
  *out = ctx;
  return WOS_OK;
}

int wos_destroy(wos_ctx* ctx) {
  if (!ctx) return WOS_EINVAL;
  {
    DeviceGuard g(ctx->device);
    cudaFree(ctx->scratch);
    for (int k = 0; k < 2; ++k)
      if (ctx->radial_tab[k]) cudaFree(ctx->radial_tab[k]);
    if (ctx->walk_end) cudaFree(ctx->walk_end);
    if (ctx->h_pts) cudaFree(ctx->h_pts);
    if (ctx->h_acc) cudaFree(ctx->h_acc);
    if (ctx->h_count) cudaFree(ctx->h_count);
    if (ctx->mv_sum) cudaFree(ctx->mv_sum);
    if (ctx->mv_count) cudaFree(ctx->mv_count);
    if (ctx->adj_buf) cudaFree(ctx->adj_buf);
    if (ctx->adj_totals) cudaFree(ctx->adj_totals);
  }
  delete ctx;
  return WOS_OK;
}

const char* wos_last_error(const wos_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int wos_problem_create(wos_ctx* ctx, const wos_problem_desc* d, wos_problem** out) {
  if (!ctx) return WOS_EINVAL;
  if (!d || !out) return fail(ctx, WOS_EINVAL, "null description or output");
  *out = nullptr;
  if (d->dim != 2 && d->dim != 3) return fail(ctx, WOS_EINVAL, "dim must be 2 or 3");
  const double* p = d->domain.p;
  for (int i = 0; i < 16; ++i)
    if (!std::isfinite(p[i])) return fail(ctx, WOS_EINVAL, "non-finite domain parameter");
  switch (d->domain.kind) {
    case WOS_DOMAIN_BOX:
      for (int i = 0; i < d->dim; ++i)
        if (!(p[3 + i] > p[i])) return fail(ctx, WOS_EINVAL, "box: hi must exceed lo");
      break;
    case WOS_DOMAIN_BALL:
      if (!(p[3] > 0)) return fail(ctx, WOS_EINVAL, "ball: radius must be > 0");
      break;
    case WOS_DOMAIN_ANNULUS:
      if (!(p[3] >= 0 && p[4] > p[3])) return fail(ctx, WOS_EINVAL, "annulus: need 0 <= r_in < r_out");
      break;
    case WOS_DOMAIN_ROUNDED_BOX:
      for (int i = 0; i < d->dim; ++i)
        if (!(p[3 + i] > 0 && p[6] >= 0 && p[6] <= p[3 + i]))
          return fail(ctx, WOS_EINVAL, "rounded box: need half extents > 0 and 0 <= corner <= half");
      break;
    case WOS_DOMAIN_MESH:
      if (d->dim != 3) return fail(ctx, WOS_EINVAL, "mesh domains are 3D");
      if (!d->domain.verts || !d->domain.tris || d->domain.nverts < 3 || d->domain.ntris < 1)
        return fail(ctx, WOS_EINVAL, "mesh: need vertices and triangles");
      if (d->domain.mesh_grid_res != 0 && (d->domain.mesh_grid_res < 4 || d->domain.mesh_grid_res > 512))
        return fail(ctx, WOS_EINVAL, "mesh: grid resolution must be 0 or in 4..512");
      if (!(d->domain.mesh_tol >= 0.0 && d->domain.mesh_tol <= 0.5))
        return fail(ctx, WOS_EINVAL, "mesh: tolerance must be in [0, 0.5]");
      break;
    case WOS_DOMAIN_CSG: {
      if (!d->domain.csg || d->domain.ncsg < 1 || d->domain.ncsg > WOS_CSG_MAX_NODES)
        return fail(ctx, WOS_EINVAL, "csg: need 1..16 nodes");
      for (int i = 0; i < d->dim; ++i)
        if (!(p[3 + i] > p[i])) return fail(ctx, WOS_EINVAL, "csg: the bounding box needs hi > lo");
      for (int i = 0; i < d->domain.ncsg; ++i) {
        const wos_csg_node& n = d->domain.csg[i];
        for (int k = 0; k < 8; ++k)
          if (!std::isfinite(n.p[k])) return fail(ctx, WOS_EINVAL, "csg: non-finite parameter");
        if (n.prim < WOS_CSG_SPHERE || n.prim > WOS_CSG_HALFSPACE) return fail(ctx, WOS_EINVAL, "csg: unknown primitive");
        if (i > 0 && (n.op < WOS_CSG_UNION || n.op > WOS_CSG_SUBTRACT)) return fail(ctx, WOS_EINVAL, "csg: unknown operation");
        bool ok = true;
        switch (n.prim) {
          case WOS_CSG_SPHERE: ok = n.p[3] > 0; break;
          case WOS_CSG_BOX:
            for (int k = 0; k < d->dim; ++k) ok = ok && n.p[3 + k] > 0 && n.p[6] >= 0 && n.p[6] <= n.p[3 + k];
            break;
          case WOS_CSG_CAPSULE: ok = n.p[6] > 0; break;
          case WOS_CSG_TORUS: ok = n.p[3] > 0 && n.p[4] > 0; break;
          case WOS_CSG_HALFSPACE: {
            double nn = 0;
            for (int k = 0; k < d->dim; ++k) nn += n.p[3 + k] * n.p[3 + k];
            ok = nn > 0;
            break;
          }
        }
        if (!ok) return fail(ctx, WOS_EINVAL, "csg: invalid primitive parameters");
      }
      break;
    }
    default:
      return fail(ctx, WOS_EINVAL, "unknown domain kind");
  }
  std::string why;
  bool drift = false;
  int rc = check_fields(*d, &drift, &why);
  if (rc != WOS_OK) return fail(ctx, rc, why);
  if (!(d->drift_bound >= 0.0) || !std::isfinite(d->drift_bound))
    return fail(ctx, WOS_EINVAL, "drift_bound must be finite and >= 0");
  if (drift && d->domain.kind == WOS_DOMAIN_MESH)
    return fail(ctx, WOS_EUNSUPPORTED, "an extra drift (omega) on a mesh domain is not supported");

  wos_problem* pr = new wos_problem();
  pr->ctx = ctx;
  pr->device = ctx->device;
  pr->dim = d->dim;
  DevProblem<float>* h32 = new DevProblem<float>();
  fill_problem(*h32, *d);
  fill_problem(pr->host64, *d);
  DeviceGuard g(ctx->device);
  rc = ensure_radial_table(ctx, d->dim);
  if (rc != WOS_OK) {
    delete h32;
    delete pr;
    return rc;
  }
  cudaError_t e = cudaSuccess;
  if (d->domain.kind == WOS_DOMAIN_MESH) {
    std::vector<wos::MeshNode> nodes;
    std::vector<float> tri;
    if (wos::mesh_build_bvh(d->domain.verts, d->domain.nverts, d->domain.tris, d->domain.ntris, &nodes, &tri,
                            &pr->mesh_depth) != 0 || pr->mesh_depth > wos::kMeshStack - 2) {
      delete h32;
      delete pr;
      return fail(ctx, WOS_EINVAL, "mesh: index out of range, non-finite vertex, or hierarchy too deep");
    }
    for (int k = 0; k < 3; ++k) {
      pr->mesh_lo[k] = nodes[0].lo[k];
      pr->mesh_hi[k] = nodes[0].hi[k];
    }
    std::vector<wos::MeshNode4> wide;  // the device traverses 4-wide nodes
    int wide_depth = 0;
    wos::mesh_collapse4(nodes, &wide, &wide_depth);
    static_assert(1 + 4 + 16 <= wos::kMeshTopMax, "top levels staged in shared memory");
    const int ntop = std::min(wos::mesh_top_first(&wide, wos::kMeshTopLevels), wos::kMeshTopMax);
    h32->mesh_top = ntop;
    pr->host64.mesh_top = ntop;
    e = cudaMalloc(&pr->mesh_nodes, wide.size() * sizeof(wos::MeshNode4));
    if (e == cudaSuccess) e = cudaMalloc(&pr->mesh_tris, tri.size() * sizeof(float));
    if (e == cudaSuccess)
      e = cudaMemcpy(pr->mesh_nodes, wide.data(), wide.size() * sizeof(wos::MeshNode4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pr->mesh_tris, tri.data(), tri.size() * sizeof(float), cudaMemcpyHostToDevice);
    h32->mesh_nodes = pr->mesh_nodes;
    h32->mesh_tris = pr->mesh_tris;
    pr->host64.mesh_nodes = pr->mesh_nodes;
    pr->host64.mesh_tris = pr->mesh_tris;
  }
  if (e == cudaSuccess) e = cudaMalloc(&pr->d32, sizeof(DevProblem<float>));
  if (e == cudaSuccess) e = cudaMalloc(&pr->d64, sizeof(DevProblem<double>));
  if (e == cudaSuccess) e = cudaMemcpy(pr->d64, &pr->host64, sizeof(DevProblem<double>), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && d->domain.kind == WOS_DOMAIN_MESH && d->domain.mesh_grid_res > 0) {
    // distance grid over the vertex bounds of the triangles plus 2% of the largest extent
    const int n = d->domain.mesh_grid_res;
    double vlo[3] = {INFINITY, INFINITY, INFINITY}, vhi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t t = 0; t < 3 * d->domain.ntris; ++t) {
      const float* v = d->domain.verts + 3 * (int64_t)d->domain.tris[t];
      for (int k = 0; k < 3; ++k) {
        vlo[k] = std::fmin(vlo[k], (double)v[k]);
        vhi[k] = std::fmax(vhi[k], (double)v[k]);
      }
    }
    double ext = std::fmax(vhi[0] - vlo[0], std::fmax(vhi[1] - vlo[1], vhi[2] - vlo[2]));
    double glo[3], gh[3], diag2 = 0.0;
    for (int k = 0; k < 3; ++k) {
      glo[k] = vlo[k] - 0.02 * ext;
      gh[k] = (vhi[k] - vlo[k] + 0.04 * ext) / (n - 1);
      diag2 += gh[k] * gh[k];
    }
    size_t nn = (size_t)n * n * n;
    e = cudaMalloc(&pr->mgrid64, nn * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&pr->mgrid32, nn * sizeof(float));
    if (e == cudaSuccess) {
      mesh_grid_kernel<<<ctx->num_sms * 8, 128>>>(pr->d64, n, glo[0], glo[1], glo[2], gh[0], gh[1], gh[2],
                                                  pr->mgrid64, pr->mgrid32);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) {
      pr->host64.mg_res = n;
      pr->host64.mgrid = pr->mgrid64;
      h32->mg_res = n;
      h32->mgrid = pr->mgrid32;
      for (int k = 0; k < 3; ++k) {
        pr->host64.mg_lo[k] = glo[k];
        pr->host64.mg_h[k] = gh[k];
        pr->host64.mg_inv_h[k] = 1.0 / gh[k];
        h32->mg_lo[k] = (float)glo[k];
        h32->mg_h[k] = (float)gh[k];
        h32->mg_inv_h[k] = (float)(1.0 / gh[k]);
      }
      pr->host64.mg_thresh = 0.5 * std::sqrt(diag2);
      h32->mg_thresh = (float)(0.5 * std::sqrt(diag2));
      e = cudaMemcpy(pr->d64, &pr->host64, sizeof(DevProblem<double>), cudaMemcpyHostToDevice);
    }
  }
  pr->host32 = *h32;
  if (e == cudaSuccess) e = cudaMemcpy(pr->d32, h32, sizeof(DevProblem<float>), cudaMemcpyHostToDevice);
  delete h32;
  if (e != cudaSuccess) {
    if (pr->d32) cudaFree(pr->d32);
    if (pr->d64) cudaFree(pr->d64);
    if (pr->mesh_nodes) cudaFree(pr->mesh_nodes);
    if (pr->mesh_tris) cudaFree(pr->mesh_tris);
    if (pr->mgrid32) cudaFree(pr->mgrid32);
    if (pr->mgrid64) cudaFree(pr->mgrid64);
    delete pr;
    return cuda_fail(ctx, e, "problem upload");
  }
  *out = pr;
  return WOS_OK;
}

int wos_problem_destroy(wos_problem* pr) {
  if (!pr) return WOS_EINVAL;
  {
    DeviceGuard g(pr->device);
    cudaFree(pr->d32);
    cudaFree(pr->d64);
    if (pr->mesh_nodes) cudaFree(pr->mesh_nodes);
    if (pr->mesh_tris) cudaFree(pr->mesh_tris);
    if (pr->mgrid32) cudaFree(pr->mgrid32);
    if (pr->mgrid64) cudaFree(pr->mgrid64);
    wos::jit_release(&pr->jit);
  }
  delete pr;
  return WOS_OK;
}

int wos_sigma_bar(wos_ctx* ctx, const wos_problem* pr, int32_t m, double* sb, double* smin, double* smax,
                  void* stream) {
  if (!ctx) return WOS_EINVAL;
  if (!pr || !sb) return fail(ctx, WOS_EINVAL, "null problem or output");
  if (m < 2 || (pr->dim == 3 && m > 2048) || m > 1 << 16) return fail(ctx, WOS_EINVAL, "lattice size out of range");
  DeviceGuard g(ctx->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double init[5] = {INFINITY, -INFINITY, INFINITY, 0.0, 0.0};
  double* out = reinterpret_cast<double*>(ctx->scratch + kScratchSigma);
  cudaError_t e = cudaMemcpyAsync(out, init, sizeof(init), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "sigma_bar init");
  double lo[3], hi[3];
  domain_bbox(pr, lo, hi);
  double h[3];
  for (int d = 0; d < 3; ++d) h[d] = (hi[d] - lo[d]) / m;
  int blocks = ctx->num_sms * 4;
  if (pr->dim == 2)
    sigma_range_kernel<2><<<blocks, 256, 0, st>>>(pr->d64, m, lo[0], lo[1], lo[2], h[0], h[1], h[2], out);
  else
    sigma_range_kernel<3><<<blocks, 256, 0, st>>>(pr->d64, m, lo[0], lo[1], lo[2], h[0], h[1], h[2], out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "sigma_bar kernel");
  double res[5];
  e = cudaMemcpyAsync(res, out, sizeof(res), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "sigma_bar readback");
  if (!(res[3] > 0)) return fail(ctx, WOS_EINVAL, "no lattice node lies inside the domain");
  if (!(res[2] > 0)) return fail(ctx, WOS_EINVAL, "alpha <= 0 at a lattice node");
  if (!std::isfinite(res[0]) || !std::isfinite(res[1])) return fail(ctx, WOS_EINVAL, "sigma' is not finite");
  double diam2 = 0.0;
  for (int d = 0; d < pr->dim; ++d) diam2 += (hi[d] - lo[d]) * (hi[d] - lo[d]);
  double v = res[1] - res[0];
  if (res[1] > v) v = res[1];
  if (1e-3 / diam2 > v) v = 1e-3 / diam2;
  // an extra drift's null weights carry |G'/G| (dir . b) / sigma_bar, whose second moment
  // grows like |b|^2 / sigma_bar per null event: keep sigma_bar >= 50 max |b|^2
  if (wos::kDriftSigmaBar * res[4] > v) v = wos::kDriftSigmaBar * res[4];
  *sb = v;
  if (smin) *smin = res[0];
  if (smax) *smax = res[1];
  return WOS_OK;
}

int wos_solve(wos_ctx* ctx, const wos_problem* pr, const float* pts, int64_t npts, const int32_t* walks,
              int32_t walks_uniform, const wos_params* prm, double* sum, double* sumsq, int64_t* count,
              uint64_t* stats, void* stream) {
  if (!ctx) return WOS_EINVAL;
  if (!pr) return fail(ctx, WOS_EINVAL, "null problem");
  int rc = validate_params(ctx, prm);
  if (rc) return rc;
  if (npts < 0) return fail(ctx, WOS_EINVAL, "npts < 0");
  if (npts == 0) return WOS_OK;
  if (npts > 0xffffffffll) return fail(ctx, WOS_EINVAL, "more than 2^32 points in one call");
  if (!pts || !sum || !sumsq || !count) return fail(ctx, WOS_EINVAL, "null device array");
  if (!walks && walks_uniform < 0) return fail(ctx, WOS_EINVAL, "walks_uniform < 0");
  if (!walks && walks_uniform == 0) return WOS_OK;
  DeviceGuard g(ctx->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t* walk_end = nullptr;
  uint64_t total;
  if (walks) {
    rc = grow(ctx, &ctx->walk_end, npts, &ctx->walk_end_cap, npts);
    if (rc) return rc;
    walk_prefix_kernel<<<1, 1024, 0, st>>>(walks, npts, ctx->walk_end);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "walk prefix kernel");
    walk_end = ctx->walk_end;
    // the kernel reads the total from the last prefix entry; bound it by 2^31 per point
    total = ~0ull;
  } else {
    total = (uint64_t)npts * (uint64_t)walks_uniform;
  }
  return launch(ctx, pr, pts, npts, walk_end, walks_uniform, total, prm, sum, sumsq, count, stats, nullptr,
                nullptr, st);
}

int wos_solve_grad(wos_ctx* ctx, const wos_problem* pr, const float* pts, int64_t npts, const int32_t* walks,
                   int32_t walks_uniform, const wos_params* prm, double* sum, double* sumsq, int64_t* count,
                   double* grad_sum, double* grad_sumsq, uint64_t* stats, void* stream) {
  if (!ctx) return WOS_EINVAL;
  if (!pr) return fail(ctx, WOS_EINVAL, "null problem");
  int rc = validate_params(ctx, prm);
  if (rc) return rc;
  if ((rc = no_window(ctx, prm))) return rc;
  if (npts < 0) return fail(ctx, WOS_EINVAL, "npts < 0");
  if (npts == 0) return WOS_OK;
  if (npts > 0xffffffffll) return fail(ctx, WOS_EINVAL, "more than 2^32 points in one call");
  if (!pts || !sum || !sumsq || !count || !grad_sum || !grad_sumsq)
    return fail(ctx, WOS_EINVAL, "null device array");
  if (!walks && walks_uniform < 0) return fail(ctx, WOS_EINVAL, "walks_uniform < 0");
  if (!walks && walks_uniform == 0) return WOS_OK;
  DeviceGuard g(ctx->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t* walk_end = nullptr;
  uint64_t total;
  if (walks) {
    rc = grow(ctx, &ctx->walk_end, npts, &ctx->walk_end_cap, npts);
    if (rc) return rc;
    walk_prefix_kernel<<<1, 1024, 0, st>>>(walks, npts, ctx->walk_end);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "walk prefix kernel");
    walk_end = ctx->walk_end;
    total = ~0ull;
  } else {
    total = (uint64_t)npts * (uint64_t)walks_uniform;
  }
  return launch(ctx, pr, pts, npts, walk_end, walks_uniform, total, prm, sum, sumsq, count, stats, nullptr,
                nullptr, st, grad_sum, grad_sumsq, nullptr);
}

static_assert(WOS_NF_SERIES_MAX == wos::kNfSeriesMax, "series table size");

int wos_solve_nf(wos_ctx* ctx, const wos_problem* pr, const float* pts, int64_t npts, const int32_t* walks,
                 int32_t walks_uniform, const wos_params* prm, int64_t max_inner, int32_t series_terms,
                 double* sum, double* sumsq, int64_t* count, uint64_t* stats, void* stream) {
  if (!ctx) return WOS_EINVAL;
  if (!pr) return fail(ctx, WOS_EINVAL, "null problem");
  int rc = validate_params(ctx, prm);
  if (rc) return rc;
  if ((rc = no_window(ctx, prm))) return rc;
  if (max_inner < 1) return fail(ctx, WOS_EINVAL, "max_inner must be >= 1");
  if (series_terms < 0 || series_terms > WOS_NF_SERIES_MAX)
    return fail(ctx, WOS_EINVAL, "series_terms must be in [0, WOS_NF_SERIES_MAX]");
  if (npts < 0) return fail(ctx, WOS_EINVAL, "npts < 0");
  if (npts == 0) return WOS_OK;
  if (npts > 0xffffffffll) return fail(ctx, WOS_EINVAL, "more than 2^32 points in one call");
  if (!pts || !sum || !sumsq || !count) return fail(ctx, WOS_EINVAL, "null device array");
  if (!walks && walks_uniform < 0) return fail(ctx, WOS_EINVAL, "walks_uniform < 0");
  if (!walks && walks_uniform == 0) return WOS_OK;
  DeviceGuard g(ctx->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t* walk_end = nullptr;
  uint64_t total;
  if (walks) {
    rc = grow(ctx, &ctx->walk_end, npts, &ctx->walk_end_cap, npts);
    if (rc) return rc;
    walk_prefix_kernel<<<1, 1024, 0, st>>>(walks, npts, ctx->walk_end);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "walk prefix kernel");
    walk_end = ctx->walk_end;
    total = ~0ull;
  } else {
    total = (uint64_t)npts * (uint64_t)walks_uniform;
  }
  return launch(ctx, pr, pts, npts, walk_end, walks_uniform, total, prm, sum, sumsq, count, stats, nullptr,
                nullptr, st, nullptr, nullptr, nullptr, max_inner, series_terms);
}

int wos_walk_estimates_nf(wos_ctx* ctx, const wos_problem* pr, const float* pts, int64_t npts, int32_t wpp,
                          const wos_params* prm, int64_t max_inner, int32_t series_terms, double* uhat,
                          int64_t* steps, uint64_t* stats, void* stream) {
  if (!ctx) return WOS_EINVAL;
  if (!pr) return fail(ctx, WOS_EINVAL, "null problem");
  int rc = validate_params(ctx, prm);
  if (rc) return rc;
  if ((rc = no_window(ctx, prm))) return rc;
  if (max_inner < 1) return fail(ctx, WOS_EINVAL, "max_inner must be >= 1");
  if (series_terms < 0 || series_terms > WOS_NF_SERIES_MAX)
    return fail(ctx, WOS_EINVAL, "series_terms must be in [0, WOS_NF_SERIES_MAX]");
  if (npts < 0 || wpp < 0) return fail(ctx, WOS_EINVAL, "negative size");
  if (npts == 0 || wpp == 0) return WOS_OK;
  if (!pts || !uhat || !steps) return fail(ctx, WOS_EINVAL, "null device array");
  DeviceGuard g(ctx->device);
  return launch(ctx, pr, pts, npts, nullptr, wpp, (uint64_t)npts * (uint64_t)wpp, prm, nullptr, nullptr, nullptr,
                stats, uhat, steps, static_cast<cudaStream_t>(stream), nullptr, nullptr, nullptr, max_inner,
                series_terms);
}

int wos_walk_grad_estimates(wos_ctx* ctx, const wos_problem* pr, const float* pts, int64_t npts, int32_t wpp,
                            const wos_params* prm, double* uhat, double* grad_hat, int64_t* steps, uint64_t* stats,
                            void* stream) {
  if (!ctx) return WOS_EINVAL;
  if (!pr) return fail(ctx, WOS_EINVAL, "null problem");
  int rc = validate_params(ctx, prm);
  if (rc) return rc;
  if ((rc = no_window(ctx, prm))) return rc;
  if (npts < 0 || wpp < 0) return fail(ctx, WOS_EINVAL, "negative size");
  if (npts == 0 || wpp == 0) return WOS_OK;
  if (!pts || !uhat || !steps || !grad_hat) return fail(ctx, WOS_EINVAL, "null device array");
  DeviceGuard g(ctx->device);
  return launch(ctx, pr, pts, npts, nullptr, wpp, (uint64_t)npts * (uint64_t)wpp, prm, nullptr, nullptr,
                nullptr, stats, uhat, steps, static_cast<cudaStream_t>(stream), nullptr, nullptr, grad_hat);
}

int wos_walk_estimates(wos_ctx* ctx, const wos_problem* pr, const float* pts, int64_t npts, int32_t wpp,
                       const wos_params* prm, double* uhat, int64_t* steps, uint64_t* stats, void* stream) {
  if (!ctx) return WOS_EINVAL;
  if (!pr) return fail(ctx, WOS_EINVAL, "null problem");
  int rc = validate_params(ctx, prm);
  if (rc) return rc;
  if (npts < 0 || wpp < 0) return fail(ctx, WOS_EINVAL, "negative size");
  if (npts == 0 || wpp == 0) return WOS_OK;
  if (!pts || !uhat || !steps) return fail(ctx, WOS_EINVAL, "null device array");
  DeviceGuard g(ctx->device);
  return launch(ctx, pr, pts, npts, nullptr, wpp, (uint64_t)npts * (uint64_t)wpp, prm, nullptr, nullptr,
                nullptr, stats, uhat, steps, static_cast<cudaStream_t>(stream));
}

int wos_finalize(wos_ctx* ctx, const double* sum, const double* sumsq, const int64_t* count, int64_t npts,
                 double* mean, double* var, double* se, void* stream) {
  if (!ctx) return WOS_EINVAL;
  if (npts < 0) return fail(ctx, WOS_EINVAL, "npts < 0");
  if (npts == 0) return WOS_OK;
  if (!sum || !sumsq || !count) return fail(ctx, WOS_EINVAL, "null accumulator");
  DeviceGuard g(ctx->device);
  int64_t blocks = (npts + 255) / 256;
  if (blocks > ctx->num_sms * 32) blocks = ctx->num_sms * 32;
  finalize_kernel<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(sum, sumsq, count, npts, mean,
                                                                                   var, se);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "finalize kernel");
  return WOS_OK;
}

int wos_solve_host(wos_ctx* ctx, const wos_problem* pr, const float* pts_host, int64_t npts, int32_t walks_uniform,
                   const wos_params* prm, double* mean_host, double* var_host, double* se_host,
                   uint64_t* stats_host, void* stream) {
  if (!ctx) return WOS_EINVAL;
  if (!pr) return fail(ctx, WOS_EINVAL, "null problem");
  int rc = validate_params(ctx, prm);
  if (rc) return rc;
  if (npts < 0 || walks_uniform < 0) return fail(ctx, WOS_EINVAL, "negative size");
  if (npts == 0) return WOS_OK;
  if (!pts_host) return fail(ctx, WOS_EINVAL, "null host points");
  DeviceGuard g(ctx->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (npts > ctx->host_cap) {
    int64_t c1 = 0, c2 = 0, c3 = 0;
    if (ctx->h_pts) cudaFree(ctx->h_pts);
    if (ctx->h_acc) cudaFree(ctx->h_acc);
    if (ctx->h_count) cudaFree(ctx->h_count);
    ctx->h_pts = nullptr;
    ctx->h_acc = nullptr;
    ctx->h_count = nullptr;
    ctx->host_cap = 0;
    if ((rc = grow(ctx, &ctx->h_pts, 3 * npts, &c1, 1))) return rc;
    if ((rc = grow(ctx, &ctx->h_acc, 5 * npts, &c2, 1))) return rc;
    if ((rc = grow(ctx, &ctx->h_count, npts, &c3, 1))) return rc;
    ctx->host_cap = npts;
  }
  double* d_sum = ctx->h_acc;
  double* d_sumsq = d_sum + npts;
  double* d_mean = d_sumsq + npts;
  double* d_var = d_mean + npts;
  double* d_se = d_var + npts;
  unsigned long long* d_stats = ctx->scratch + kScratchStats;
  cudaError_t e = cudaMemcpyAsync(ctx->h_pts, pts_host, sizeof(float) * pr->dim * npts, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_sum, 0, 2 * sizeof(double) * npts, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->h_count, 0, sizeof(int64_t) * npts, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_stats, 0, wos::ST_WORDS * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "host solve staging");
  rc = wos_solve(ctx, pr, ctx->h_pts, npts, nullptr, walks_uniform, prm, d_sum, d_sumsq, ctx->h_count,
                 reinterpret_cast<uint64_t*>(d_stats), stream);
  if (rc) return rc;
  rc = wos_finalize(ctx, d_sum, d_sumsq, ctx->h_count, npts, d_mean, d_var, d_se, stream);
  if (rc) return rc;
  if (mean_host) e = cudaMemcpyAsync(mean_host, d_mean, sizeof(double) * npts, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && var_host) e = cudaMemcpyAsync(var_host, d_var, sizeof(double) * npts, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && se_host) e = cudaMemcpyAsync(se_host, d_se, sizeof(double) * npts, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && stats_host)
    e = cudaMemcpyAsync(stats_host, d_stats, wos::ST_WORDS * sizeof(uint64_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "host solve readback");
  return WOS_OK;
}

// ---- problem-specialised walk kernels (runtime compilation) ----
namespace {
const int32_t kSpecFlags =
    WOS_SPEC_FP32 | WOS_SPEC_FP64 | WOS_SPEC_PLAIN | WOS_SPEC_WINDOW | WOS_SPEC_GRAD | WOS_SPEC_ADJOINT;

int spec_variants(int32_t flags) {
  int vm = 0;
  if (flags & WOS_SPEC_PLAIN) vm |= 1 << wos::kJitPlain;
  if (flags & WOS_SPEC_WINDOW) vm |= 1 << wos::kJitWindow;
  if (flags & WOS_SPEC_GRAD) vm |= 1 << wos::kJitGrad;
  if (flags & WOS_SPEC_ADJOINT) vm |= 1 << wos::kJitAdjoint;
  return vm ? vm : 1 << wos::kJitPlain;
}

// the fields of a description, checked and filled as wos_problem_create does (no device)
int host_problem(const wos_problem_desc* d, DevProblem<double>* P, std::string* why) {
  if (d->dim != 2 && d->dim != 3) {
    *why = "dim must be 2 or 3";
    return WOS_EINVAL;
  }
  bool drift = false;
  int rc = check_fields(*d, &drift, why);
  if (rc != WOS_OK) return rc;
  fill_problem(*P, *d);
  return WOS_OK;
}

void copy_text(const std::string& t, char* buf, int64_t cap) {
  if (!buf || cap <= 0) return;
  size_t n = std::min((size_t)(cap - 1), t.size());
  std::memcpy(buf, t.data(), n);
  buf[n] = '\0';
}
}  // namespace

int wos_problem_specialize(wos_ctx* ctx, wos_problem* pr, int32_t flags) {
  if (!ctx) return WOS_EINVAL;
  if (!pr) return fail(ctx, WOS_EINVAL, "null problem");
  if (flags & ~kSpecFlags) return fail(ctx, WOS_EINVAL, "unknown specialisation flag");
  const int vm = spec_variants(flags);
  const bool want32 = (flags & WOS_SPEC_FP32) || !(flags & WOS_SPEC_FP64);
  const bool want64 = (flags & WOS_SPEC_FP64) != 0;
  DeviceGuard g(pr->device);
  std::string why;
  for (int fp64 = 0; fp64 < 2; ++fp64) {
    if (!(fp64 ? want64 : want32)) continue;
    int rc = wos::jit_specialise(&pr->jit, pr->host64, fp64 != 0, vm, &why);
    if (rc != WOS_OK) return fail(ctx, rc, "specialise: " + why);
  }
  return WOS_OK;
}

int wos_problem_specialized(const wos_problem* pr, int32_t* flags_out) {
  if (!pr || !flags_out) return WOS_EINVAL;
  int32_t f = 0;
  static const int32_t vbit[wos::kJitVariants] = {WOS_SPEC_PLAIN, WOS_SPEC_WINDOW, WOS_SPEC_GRAD};
  for (int p = 0; p < 2; ++p)
    for (int v = 0; v < wos::kJitVariants; ++v)
      if (pr->jit.kernel[p][v] != nullptr) f |= (p ? WOS_SPEC_FP64 : WOS_SPEC_FP32) | vbit[v];
  for (int p = 0; p < 2; ++p)
    if (pr->jit.adjoint[p][0][0] != nullptr) f |= (p ? WOS_SPEC_FP64 : WOS_SPEC_FP32) | WOS_SPEC_ADJOINT;
  *flags_out = f;
  return WOS_OK;
}

int wos_jit_source(const wos_problem_desc* d, char* buf, int64_t cap, int64_t* len) {
  if (!d) return WOS_EINVAL;
  std::unique_ptr<DevProblem<double>> P(new DevProblem<double>());
  std::string why;
  int rc = host_problem(d, P.get(), &why);
  if (rc != WOS_OK) {
    copy_text(why, buf, cap);
    return rc;
  }
  const std::string src = wos::jit_source(*P);
  if (len) *len = (int64_t)src.size();
  copy_text(src, buf, cap);
  return WOS_OK;
}

static int batch_info_of(const wos_problem_desc* descs, int32_t n, wos::BatchJitInfo* info, std::string* why) {
  if (!descs || n < 1) {
    *why = "need at least one description";
    return WOS_EINVAL;
  }
  std::vector<DevProblem<double>> h(n);
  for (int32_t i = 0; i < n; ++i) {
    int rc = host_problem(&descs[i], &h[i], why);
    if (rc != WOS_OK) return rc;
    if (descs[i].dim != descs[0].dim) {
      *why = "all problems of a batch must have one dimension";
      return WOS_EINVAL;
    }
  }
  wos::batch_jit_info(h.data(), n, info);
  return WOS_OK;
}

int wos_jit_batch_source(const wos_problem_desc* descs, int32_t n, char* buf, int64_t cap, int64_t* len) {
  std::unique_ptr<wos::BatchJitInfo> info(new wos::BatchJitInfo());
  std::string why;
  int rc = batch_info_of(descs, n, info.get(), &why);
  if (rc != WOS_OK) {
    copy_text(why, buf, cap);
    return rc;
  }
  const std::string src = wos::jit_source_batch(*info);
  if (len) *len = (int64_t)src.size();
  copy_text(src, buf, cap);
  return WOS_OK;
}

int wos_jit_batch_compile(const wos_problem_desc* descs, int32_t n, int32_t flags, char* log, int64_t log_cap,
                          int64_t* cubin_bytes) {
  if (flags & ~(WOS_SPEC_FP32 | WOS_SPEC_FP64 | WOS_SPEC_PLAIN)) return WOS_EINVAL;
  std::unique_ptr<wos::BatchJitInfo> info(new wos::BatchJitInfo());
  std::string why;
  int rc = batch_info_of(descs, n, info.get(), &why);
  if (rc != WOS_OK) {
    copy_text(why, log, log_cap);
    return rc;
  }
  std::vector<char> cubin;
  std::vector<std::string> lowered;
  rc = wos::jit_compile_batch(*info, (flags & WOS_SPEC_FP64) != 0, &cubin, &lowered, &why);
  copy_text(why, log, log_cap);
  if (cubin_bytes) *cubin_bytes = (int64_t)cubin.size();
  return rc;
}

int wos_jit_compile(const wos_problem_desc* d, int32_t flags, char* log, int64_t log_cap, int64_t* cubin_bytes) {
  if (!d || (flags & ~kSpecFlags)) return WOS_EINVAL;
  std::unique_ptr<DevProblem<double>> P(new DevProblem<double>());
  std::string why;
  int rc = host_problem(d, P.get(), &why);
  if (rc != WOS_OK) {
    copy_text(why, log, log_cap);
    return rc;
  }
  std::vector<char> cubin;
  std::vector<std::string> lowered;
  rc = wos::jit_compile(*P, (flags & WOS_SPEC_FP64) != 0, spec_variants(flags), &cubin, &lowered, &why);
  copy_text(why, log, log_cap);
  if (cubin_bytes) *cubin_bytes = (int64_t)cubin.size();
  return rc;
}

}  // extern "C"

namespace {
constexpr uint64_t kAdjChunkItems = 1ull << 24;  // walks per pair of passes (their totals: 64 or 128 MB)

// the context's buffer of walk totals, at least `bytes` long
int ensure_adj_totals(wos_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->adj_totals_bytes) return WOS_OK;
  // an earlier adjoint may still be reading the old buffer on some stream
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronise before growing the adjoint totals");
  if (ctx->adj_totals) cudaFree(ctx->adj_totals);
  ctx->adj_totals = nullptr;
  ctx->adj_totals_bytes = 0;
  e = cudaMalloc(&ctx->adj_totals, bytes);
  if (e != cudaSuccess) {
    ctx->adj_totals = nullptr;
    return fail(ctx, WOS_ENOMEM, std::string("cudaMalloc(adjoint totals): ") + cudaGetErrorString(e));
  }
  ctx->adj_totals_bytes = bytes;
  return WOS_OK;
}

// the two passes of the path-replay adjoint over chunks of at most kAdjChunkItems walks: pass 1
// stores each walk's total, pass 2 replays the walk from it and scatters.  The
// problem-specialised kernels run when loaded (WOS_SPEC_ADJOINT), else the generic ones.
int adjoint_run(wos_ctx* ctx, const wos_problem* pr, wos::AdjLaunch& L, bool fp64, cudaStream_t st) {
  L.problem = fp64 ? (const void*)pr->d64 : (const void*)pr->d32;
  L.problem_bytes = fp64 ? (int)sizeof(DevProblem<double>) : (int)sizeof(DevProblem<float>);
  L.work_counter = ctx->scratch;
  const uint64_t all = L.total_items;
  const size_t rb = fp64 ? sizeof(double) : sizeof(float);
  int rc = ensure_adj_totals(ctx, rb * (size_t)std::min<uint64_t>(all, kAdjChunkItems));
  if (rc) return rc;
  L.totals = ctx->adj_totals;
  for (uint64_t base = 0; base < all; base += kAdjChunkItems) {
    L.item_base = base;
    L.total_items = std::min<uint64_t>(all - base, kAdjChunkItems);
    for (int pass = 1; pass <= 2; ++pass) {
      L.pass = pass;
      cudaError_t e = cudaMemsetAsync(ctx->scratch, 0, sizeof(unsigned long long), st);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemsetAsync(work counter)");
      cudaKernel_t spec = pr->jit.adjoint[fp64 ? 1 : 0][L.alpha ? 1 : 0][pass - 1];
      if (spec != nullptr) e = wos::launch_adjoint_kernel(L, spec, (int)rb, ctx->num_sms, st);
      else e = fp64 ? wos::launch_adjoint_f64(L, ctx->num_sms, st) : wos::launch_adjoint_f32(L, ctx->num_sms, st);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "adjoint kernel launch");
    }
  }
  L.total_items = all;
  return WOS_OK;
}
}  // namespace

extern "C" int wos_adjoint_sigma(wos_ctx* ctx, const wos_problem* pr, const float* pts, int64_t npts,
                                 int32_t walks_uniform, const wos_params* prm, const double* grad_u,
                                 double* grad_sigma, uint64_t* stats, void* stream) {
  if (!ctx) return WOS_EINVAL;
  if (!pr) return fail(ctx, WOS_EINVAL, "null problem");
  int rc = validate_params(ctx, prm);
  if (rc) return rc;
  if ((rc = no_window(ctx, prm))) return rc;
  if (npts < 0 || walks_uniform < 0) return fail(ctx, WOS_EINVAL, "negative size");
  if (npts > 0xffffffffll) return fail(ctx, WOS_EINVAL, "more than 2^32 points in one call");
  if (npts == 0 || walks_uniform == 0) return WOS_OK;
  if (!pts || !grad_u || !grad_sigma) return fail(ctx, WOS_EINVAL, "null device array");
  const DevProblem<double>& H = pr->host64;
  if (H.has_drift) return fail(ctx, WOS_EUNSUPPORTED, "the adjoint has no extra-drift (omega) term");
  if (H.sigma.kind != wos::F_GRID_LINEAR)
    return fail(ctx, WOS_EUNSUPPORTED, "the sigma gradient needs sigma given as a multilinear grid");
  if (H.f.kind == wos::F_MANUFACTURED)
    return fail(ctx, WOS_EUNSUPPORTED, "a manufactured source depends on sigma; give f explicitly");
  DeviceGuard g(ctx->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  wos::AdjLaunch L;
  std::memset(&L, 0, sizeof(L));
  L.dim = pr->dim;
  L.pts = pts;
  L.npts = npts;
  L.walks_uniform = walks_uniform;
  L.total_items = (uint64_t)npts * (uint64_t)walks_uniform;
  L.seed = prm->seed;
  L.walk_offset = prm->walk_offset;
  L.eps = prm->eps;
  L.sigma_bar = prm->sigma_bar;
  L.max_steps = prm->max_steps;
  L.grad_u = grad_u;
  L.grad_sigma = grad_sigma;
  L.stats = reinterpret_cast<unsigned long long*>(stats);
  L.radial_tab = ctx->radial_tab[pr->dim - 2];
  return adjoint_run(ctx, pr, L, prm->precision == WOS_FP64, st);
}

namespace wos {
int render_slice(const DevProblem<double>* dprob, const DevProblem<double>& host, int dim, const wos_view* view,
                 const double* sum, const int64_t* count, uint8_t* rgba, float* value, float* depth, int num_sms,
                 cudaStream_t st);
int slice_points(int dim, const wos_view* view, float* pts, int num_sms, cudaStream_t st);
}  // namespace wos

extern "C" int wos_slice_points(wos_ctx* ctx, const wos_problem* pr, const wos_view* view, float* pts, void* stream) {
  if (!ctx) return WOS_EINVAL;
  if (!pr || !view || !pts) return fail(ctx, WOS_EINVAL, "null argument");
  if (view->slice_nu < 1 || view->slice_nv < 1) return fail(ctx, WOS_EINVAL, "empty slice grid");
  DeviceGuard g(ctx->device);
  int rc = wos::slice_points(pr->dim, view, pts, ctx->num_sms, static_cast<cudaStream_t>(stream));
  if (rc != WOS_OK) return fail(ctx, rc, "slice points: degenerate plane rectangle");
  return WOS_OK;
}

extern "C" int wos_render_slice(wos_ctx* ctx, const wos_problem* pr, const wos_view* view, const double* sum,
                                const int64_t* count, uint8_t* rgba, float* value, float* depth, void* stream) {
  if (!ctx) return WOS_EINVAL;
  if (!pr || !view || !sum || !count || !rgba) return fail(ctx, WOS_EINVAL, "null argument");
  if (pr->host64.domain_kind == wos::D_MESH)
    return fail(ctx, WOS_EUNSUPPORTED, "mesh distances are unsigned: no sphere tracing");
  if (view->width < 1 || view->height < 1 || view->slice_nu < 1 || view->slice_nv < 1 ||
      !(view->value_hi > view->value_lo))
    return fail(ctx, WOS_EINVAL, "bad view size or value range");
  DeviceGuard g(ctx->device);
  int rc = wos::render_slice(pr->d64, pr->host64, pr->dim, view, sum, count, rgba, value, depth, ctx->num_sms,
                             static_cast<cudaStream_t>(stream));
  if (rc != WOS_OK) return fail(ctx, rc, "render: degenerate camera or plane, or launch failure");
  return WOS_OK;
}

extern "C" int wos_adjoint_alpha(wos_ctx* ctx, const wos_problem* pr, const float* pts, int64_t npts,
                                 int32_t walks_uniform, const wos_params* prm, const double* grad_u,
                                 double* grad_alpha, uint64_t* stats, void* stream) {
  if (!ctx) return WOS_EINVAL;
  if (!pr) return fail(ctx, WOS_EINVAL, "null problem");
  int rc = validate_params(ctx, prm);
  if (rc) return rc;
  if ((rc = no_window(ctx, prm))) return rc;
  if (npts < 0 || walks_uniform < 0) return fail(ctx, WOS_EINVAL, "negative size");
  if (npts > 0xffffffffll) return fail(ctx, WOS_EINVAL, "more than 2^32 points in one call");
  if (npts == 0 || walks_uniform == 0) return WOS_OK;
  if (!pts || !grad_u || !grad_alpha) return fail(ctx, WOS_EINVAL, "null device array");
  const DevProblem<double>& H = pr->host64;
  if (H.has_drift) return fail(ctx, WOS_EUNSUPPORTED, "the adjoint has no extra-drift (omega) term");
  if (H.alpha.kind != wos::F_GRID_BSPLINE)
    return fail(ctx, WOS_EUNSUPPORTED, "the alpha gradient needs alpha given as a B-spline grid");
  if (H.f.kind == wos::F_MANUFACTURED)
    return fail(ctx, WOS_EUNSUPPORTED, "a manufactured source depends on alpha; give f explicitly");
  int64_t nodes = (int64_t)H.alpha.res[0] * H.alpha.res[1] * (pr->dim == 3 ? H.alpha.res[2] : 1);
  DeviceGuard g(ctx->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  wos::AdjLaunch L;
  std::memset(&L, 0, sizeof(L));
  L.dim = pr->dim;
  L.pts = pts;
  L.npts = npts;
  L.walks_uniform = walks_uniform;
  L.total_items = (uint64_t)npts * (uint64_t)walks_uniform;
  L.seed = prm->seed;
  L.walk_offset = prm->walk_offset;
  L.eps = prm->eps;
  L.sigma_bar = prm->sigma_bar;
  L.max_steps = prm->max_steps;
  L.grad_u = grad_u;
  L.grad_alpha = grad_alpha;
  L.alpha = 1;
  L.stats = reinterpret_cast<unsigned long long*>(stats);
  L.radial_tab = ctx->radial_tab[pr->dim - 2];
  // grids of up to 8192 nodes (64 KB of FP64) are accumulated per CTA in shared memory
  // the per-CTA copy is padded (row stride res0 + 1, plane stride (res0 + 1) res1 + 1)
  int64_t padded = ((int64_t)(H.alpha.res[0] + 1) * H.alpha.res[1] + 1) * (pr->dim == 3 ? H.alpha.res[2] : 1);
  L.priv_nodes = (nodes <= 8192) ? (int)padded : 0;
  return adjoint_run(ctx, pr, L, prm->precision == WOS_FP64, st);
}

extern "C" int wos_batch_create(wos_ctx* ctx, const wos_problem* const* probs, int32_t nprob,
                                const int64_t* pt_offsets, const double* sigma_bars, wos_batch** out) {
  if (!ctx) return WOS_EINVAL;
  if (!out || !probs || !pt_offsets || !sigma_bars || nprob < 1) return fail(ctx, WOS_EINVAL, "bad batch arguments");
  *out = nullptr;
  int dim = probs[0] ? probs[0]->dim : 0;
  if (pt_offsets[0] != 0) return fail(ctx, WOS_EINVAL, "point offsets must start at 0");
  for (int32_t i = 0; i < nprob; ++i) {
    if (!probs[i]) return fail(ctx, WOS_EINVAL, "null problem in batch");
    if (probs[i]->ctx != ctx) return fail(ctx, WOS_EINVAL, "problem of another context in batch");
    if (probs[i]->dim != dim) return fail(ctx, WOS_EINVAL, "all problems of a batch must have one dimension");
    if (probs[i]->host64.domain_kind == wos::D_MESH) return fail(ctx, WOS_EUNSUPPORTED, "mesh domains in a batch");
    if (probs[i]->host64.has_drift) return fail(ctx, WOS_EUNSUPPORTED, "extra-drift (omega) problems in a batch");
    if (pt_offsets[i + 1] < pt_offsets[i]) return fail(ctx, WOS_EINVAL, "point offsets must not decrease");
    if (!finite_pos(sigma_bars[i])) return fail(ctx, WOS_EINVAL, "sigma_bar of every problem must be > 0");
  }
  int64_t npts = pt_offsets[nprob];
  if (npts > 0xffffffffll) return fail(ctx, WOS_EINVAL, "more than 2^32 points in a batch");
  DeviceGuard g(ctx->device);
  wos_batch* b = new wos_batch();
  b->ctx = ctx;
  b->device = ctx->device;
  b->dim = dim;
  b->nprob = nprob;
  b->npts = npts;
  std::vector<DevProblem<float>> h32(nprob);
  std::vector<DevProblem<double>> h64(nprob);
  for (int32_t i = 0; i < nprob; ++i) {
    h32[i] = probs[i]->host32;
    h64[i] = probs[i]->host64;
  }
  // which fields every problem shares (the code wos_batch_specialize can compile in)
  wos::batch_jit_info(h64.data(), nprob, &b->jit_info);
  cudaError_t e = cudaMalloc(&b->d32, sizeof(DevProblem<float>) * nprob);
  if (e == cudaSuccess) e = cudaMalloc(&b->d64, sizeof(DevProblem<double>) * nprob);
  if (e == cudaSuccess) e = cudaMalloc(&b->offsets, sizeof(int64_t) * (nprob + 1));
  if (e == cudaSuccess) e = cudaMalloc(&b->sigma_bars, sizeof(double) * nprob);
  if (e == cudaSuccess) e = cudaMalloc(&b->walk_end, sizeof(int64_t) * (npts > 0 ? npts : 1));
  if (e == cudaSuccess) e = cudaMemcpy(b->d32, h32.data(), sizeof(DevProblem<float>) * nprob, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d64, h64.data(), sizeof(DevProblem<double>) * nprob, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->offsets, pt_offsets, sizeof(int64_t) * (nprob + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->sigma_bars, sigma_bars, sizeof(double) * nprob, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    wos_batch_destroy(b);
    return cuda_fail(ctx, e, "batch upload");
  }
  *out = b;
  return WOS_OK;
}

extern "C" int wos_batch_destroy(wos_batch* b) {
  if (!b) return WOS_EINVAL;
  {
    DeviceGuard g(b->device);
    if (b->d32) cudaFree(b->d32);
    if (b->d64) cudaFree(b->d64);
    if (b->offsets) cudaFree(b->offsets);
    if (b->sigma_bars) cudaFree(b->sigma_bars);
    if (b->walk_end) cudaFree(b->walk_end);
    wos::jit_release(&b->jit);
  }
  delete b;
  return WOS_OK;
}

extern "C" int wos_batch_specialize(wos_ctx* ctx, wos_batch* b, int32_t flags) {
  if (!ctx) return WOS_EINVAL;
  if (!b || b->ctx != ctx) return fail(ctx, WOS_EINVAL, "null batch or batch of another context");
  if (flags & ~(WOS_SPEC_FP32 | WOS_SPEC_FP64 | WOS_SPEC_PLAIN))
    return fail(ctx, WOS_EINVAL, "batches specialise the plain walk in FP32 and/or FP64 only");
  const bool f32 = (flags & WOS_SPEC_FP32) || !(flags & WOS_SPEC_FP64);
  const bool f64 = (flags & WOS_SPEC_FP64) != 0;
  DeviceGuard g(b->device);
  std::string why;
  for (int p = 0; p < 2; ++p) {
    if ((p == 0 && !f32) || (p == 1 && !f64)) continue;
    int rc = wos::jit_specialise_batch(&b->jit, b->jit_info, p == 1, &why);
    if (rc != WOS_OK) return fail(ctx, rc, why);
  }
  return WOS_OK;
}

extern "C" int wos_batch_specialized(const wos_batch* b, int32_t* flags_out, int32_t* uniform_fields) {
  if (!b || !flags_out) return WOS_EINVAL;
  int32_t f = 0;
  if (b->jit.kernel[0][0]) f |= WOS_SPEC_FP32 | WOS_SPEC_PLAIN;
  if (b->jit.kernel[1][0]) f |= WOS_SPEC_FP64 | WOS_SPEC_PLAIN;
  *flags_out = f;
  if (uniform_fields) *uniform_fields = (int32_t)b->jit_info.uniform;
  return WOS_OK;
}

namespace {
int solve_batch_impl(wos_ctx* ctx, const wos_batch* b, const wos_schedule& sched, const float* pts,
                     const int32_t* walks, int32_t walks_uniform, const wos_params* prm, double* sum, double* sumsq,
                     int64_t* count, uint64_t* stats, void* stream);

bool valid_schedule(const wos_schedule& s) {
  const bool chunk_ok = s.chunk == 0 || (s.chunk >= 32 && s.chunk <= 65536 && s.chunk % 32 == 0);
  return chunk_ok && s.blocks_per_sm >= 0 && s.blocks_per_sm <= 32 && (s.regs_variant == 0 || s.regs_variant == 1) &&
         s.reserved == 0;
}

__global__ void trial_walks_kernel(const int32_t* walks, int64_t n, int32_t uniform, int shift, int32_t* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t w = walks ? walks[i] : uniform;
    out[i] = (w > 0) ? max(1, w >> shift) : 0;
  }
}
}  // namespace

extern "C" int wos_batch_set_schedule(wos_batch* b, const wos_schedule* sched) {
  if (!b) return WOS_EINVAL;
  wos_schedule s = sched ? *sched : wos_schedule{0, 0, 0, 0};
  if (!valid_schedule(s)) return WOS_EINVAL;
  b->sched = s;
  return WOS_OK;
}

extern "C" int wos_batch_get_schedule(const wos_batch* b, wos_schedule* out) {
  if (!b || !out) return WOS_EINVAL;
  *out = b->sched;
  return WOS_OK;
}

extern "C" int wos_batch_autotune(wos_ctx* ctx, wos_batch* b, const float* pts, const int32_t* walks,
                                  int32_t walks_uniform, const wos_params* prm, int32_t trial_shift,
                                  wos_schedule* best_out, double* best_ms, double* default_ms, void* stream) {
  if (!ctx) return WOS_EINVAL;
  if (!b || b->ctx != ctx) return fail(ctx, WOS_EINVAL, "null batch or batch of another context");
  if (!prm || !pts) return fail(ctx, WOS_EINVAL, "null params or points");
  if (trial_shift < 0 || trial_shift > 16) return fail(ctx, WOS_EINVAL, "trial_shift must be in 0..16");
  if (!walks && walks_uniform <= 0) return fail(ctx, WOS_EINVAL, "walks_uniform must be > 0");
  if (b->npts == 0) return fail(ctx, WOS_EINVAL, "empty batch");
  DeviceGuard g(ctx->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // trial buffers: walks per point >> trial_shift (at least 1 where the walk count is > 0),
  // and accumulators; freed before returning
  const int64_t n = b->npts;
  int32_t* tw = nullptr;
  double* acc = nullptr;
  int64_t* cnt = nullptr;
  unsigned long long* stt = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&]() {
    if (tw) cudaFree(tw);
    if (acc) cudaFree(acc);
    if (cnt) cudaFree(cnt);
    if (stt) cudaFree(stt);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  if (cudaMalloc(&tw, sizeof(int32_t) * n) != cudaSuccess || cudaMalloc(&acc, 2 * sizeof(double) * n) != cudaSuccess ||
      cudaMalloc(&cnt, sizeof(int64_t) * n) != cudaSuccess ||
      cudaMalloc(&stt, wos::ST_WORDS * sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return fail(ctx, WOS_ENOMEM, "autotune trial buffers");
  }
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return fail(ctx, WOS_ECUDA, "autotune events");
  }
  trial_walks_kernel<<<ctx->num_sms * 4, 256, 0, st>>>(walks, n, walks_uniform, trial_shift, tw);
  if (cudaError_t el = cudaGetLastError(); el != cudaSuccess) {
    cleanup();
    return cuda_fail(ctx, el, "autotune trial walks");
  }
  // candidates: the kernel's own chunk rule and fixed chunks, at both register caps
  std::vector<wos_schedule> cand;
  const int32_t chunks[] = {0, 64, 128, 256, 512, 1024, 2048};
  for (int rv = 0; rv < 2; ++rv)
    for (int32_t c : chunks) cand.push_back(wos_schedule{c, 0, rv, 0});
  double best = 1e300, dflt = -1.0;
  wos_schedule best_s = cand[0];
  int rc = WOS_OK;
  for (size_t i = 0; i <= cand.size() && rc == WOS_OK; ++i) {
    // i == 0 warms up with the first candidate (untimed)
    const wos_schedule& sc = cand[i == 0 ? 0 : i - 1];
    cudaError_t em = cudaMemsetAsync(acc, 0, 2 * sizeof(double) * n, st);
    if (em == cudaSuccess) em = cudaMemsetAsync(cnt, 0, sizeof(int64_t) * n, st);
    if (em != cudaSuccess) {
      rc = cuda_fail(ctx, em, "autotune accumulators");
      break;
    }
    cudaEventRecord(e0, st);
    rc = solve_batch_impl(ctx, b, sc, pts, tw, 0, prm, acc, acc + n, cnt, reinterpret_cast<uint64_t*>(stt), stream);
    cudaEventRecord(e1, st);
    if (rc != WOS_OK) break;
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      rc = cuda_fail(ctx, cudaGetLastError(), "autotune trial");
      break;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (i == 0) continue;
    if (i == 1) dflt = ms;
    if (ms < best) {
      best = ms;
      best_s = sc;
    }
  }
  cleanup();
  if (rc != WOS_OK) return rc;
  b->sched = best_s;
  if (best_out) *best_out = best_s;
  if (best_ms) *best_ms = best;
  if (default_ms) *default_ms = dflt;
  return WOS_OK;
}

extern "C" int wos_solve_batch(wos_ctx* ctx, const wos_batch* b, const float* pts, const int32_t* walks,
                               int32_t walks_uniform, const wos_params* prm, double* sum, double* sumsq,
                               int64_t* count, uint64_t* stats, void* stream) {
  if (!ctx) return WOS_EINVAL;
  if (!b || b->ctx != ctx) return fail(ctx, WOS_EINVAL, "null batch or batch of another context");
  return solve_batch_impl(ctx, b, b->sched, pts, walks, walks_uniform, prm, sum, sumsq, count, stats, stream);
}

namespace {
int solve_batch_impl(wos_ctx* ctx, const wos_batch* b, const wos_schedule& sched, const float* pts,
                     const int32_t* walks, int32_t walks_uniform, const wos_params* prm, double* sum, double* sumsq,
                     int64_t* count, uint64_t* stats, void* stream) {
  if (!b || b->ctx != ctx) return fail(ctx, WOS_EINVAL, "null batch or batch of another context");
  if (!prm) return fail(ctx, WOS_EINVAL, "params is NULL");
  if (!finite_pos(prm->eps) || prm->max_steps < 1 || (prm->precision != WOS_FP32 && prm->precision != WOS_FP64))
    return fail(ctx, WOS_EINVAL, "eps must be > 0, max_steps >= 1, precision FP32 or FP64");
  if (prm->ww_lo != 0.0) return fail(ctx, WOS_EUNSUPPORTED, "batches have no weight window");
  if (!walks && walks_uniform < 0) return fail(ctx, WOS_EINVAL, "walks_uniform < 0");
  if (b->npts == 0 || (!walks && walks_uniform == 0)) return WOS_OK;
  if (!pts || !sum || !sumsq || !count) return fail(ctx, WOS_EINVAL, "null device array");
  DeviceGuard g(ctx->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t* walk_end = nullptr;
  uint64_t total;
  if (walks) {
    walk_prefix_kernel<<<1, 1024, 0, st>>>(walks, b->npts, b->walk_end);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "walk prefix kernel");
    walk_end = b->walk_end;
    total = ~0ull;
  } else {
    total = (uint64_t)b->npts * (uint64_t)walks_uniform;
  }
  cudaError_t e = cudaMemsetAsync(ctx->scratch, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemsetAsync(work counter)");
  unsigned long long* st_ptr = reinterpret_cast<unsigned long long*>(stats);
  if (st_ptr == nullptr) {
    st_ptr = ctx->scratch + kScratchStats;
    e = cudaMemsetAsync(st_ptr, 0, wos::ST_WORDS * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemsetAsync(stats)");
  }
  wos::WalkLaunch L;
  std::memset(&L, 0, sizeof(L));
  L.dim = b->dim;
  L.pts = pts;
  L.npts = b->npts;
  L.walk_end = walk_end;
  L.walks_uniform = walks_uniform;
  L.total_items = total;
  L.seed = prm->seed;
  L.walk_offset = prm->walk_offset;
  L.eps = prm->eps;
  L.sigma_bar = 1.0;  // per problem: sigma_bars
  L.max_steps = prm->max_steps;
  L.sum = sum;
  L.sumsq = sumsq;
  L.count = reinterpret_cast<unsigned long long*>(count);
  L.stats = st_ptr;
  L.work_counter = ctx->scratch;
  L.radial_tab = ctx->radial_tab[b->dim - 2];
  L.prob_offsets = b->offsets;
  L.sigma_bars = b->sigma_bars;
  L.nprob = b->nprob;
  L.chunk = (uint32_t)sched.chunk;
  L.blocks_per_sm = sched.blocks_per_sm;
  L.regs_variant = sched.regs_variant;
  const bool fp64 = prm->precision == WOS_FP64;
  L.probs = fp64 ? (const void*)b->d64 : (const void*)b->d32;
  cudaKernel_t spec = b->jit.kernel[fp64 ? 1 : 0][sched.regs_variant == 1 ? 1 : 0];
  if (spec != nullptr) e = wos::launch_walks_kernel(L, spec, fp64 ? 8 : 4, ctx->num_sms, st);  // wos_batch_specialize
  else e = fp64 ? wos::launch_walks_f64(L, ctx->num_sms, st) : wos::launch_walks_f32(L, ctx->num_sms, st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "batched walk kernel launch");
  return WOS_OK;
}
}  // namespace

// ===========================================================================
// Allocation-free solve.
//
// Some callers cannot allocate device memory at all: code running inside a
// host allocator hook or a memory-pool callback, plugins whose host program
// owns every allocation and forbids cudaMalloc/cudaFree, and programs that
// must not synchronise the device, which cudaFree does.  wos_solve_noalloc
// serves them.  It runs the same walk kernel as wos_solve, but the kernel's
// scratch (work counter, default statistics, the problem description and the
// per-point walk prefix sums) lives in the file-scope device array below
// instead of context memory.  That array is part of the module image, so every
// GPU that loads this library holds it (WOS_NOALLOC_SCRATCH_BYTES) until the
// process exits.
// ===========================================================================
namespace {

constexpr size_t kNaCounter = 0;        // work counter (8 bytes)
constexpr size_t kNaStats = 64;         // default statistics (WOS_STATS_WORDS x 8 bytes)
constexpr size_t kNaProblem = 256;      // DevProblem<float> or DevProblem<double>
constexpr size_t kNaProblemBytes = 16384;
constexpr size_t kNaPrefix = kNaProblem + kNaProblemBytes;  // int64 walk prefix sums
constexpr size_t kNaBytes = kNaPrefix + sizeof(int64_t) * (size_t)WOS_NOALLOC_MAX_VAR_POINTS;
static_assert(kNaBytes == WOS_NOALLOC_SCRATCH_BYTES, "header and scratch layout disagree");
static_assert(sizeof(DevProblem<double>) <= kNaProblemBytes, "problem does not fit the static scratch");
static_assert(kNaProblem % 256 == 0 && kNaPrefix % 256 == 0, "scratch regions must stay 256-byte aligned");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// The problem description reaches the scratch as a kernel argument: a by-value
// parameter is copied by the launch itself, so the host neither blocks (a pageable
// cudaMemcpyAsync waits for the stream) nor leaves a pointer to its own stack behind.
// One thread copies it with compile-time offsets (a dynamic index into the parameter
// block would make a per-thread local copy); it also zeroes the work counter and, when
// the caller passes no statistics array, the default statistics.
static_assert(sizeof(DevProblem<double>) + 64 <= 32764, "problem must fit the kernel parameter block");
template <typename Prob>
struct NaBlob {
  int4 w[sizeof(Prob) / 16];
};
template <typename Prob>
__global__ void noalloc_setup_kernel(const NaBlob<Prob> blob, int4* dst, unsigned long long* counter,
                                     unsigned long long* stats_zero) {
#pragma unroll
  for (int i = 0; i < (int)(sizeof(Prob) / 16); ++i) dst[i] = blob.w[i];
  *counter = 0ull;
  if (stats_zero != nullptr) {
#pragma unroll
    for (int i = 0; i < WOS_STATS_WORDS; ++i) stats_zero[i] = 0ull;
  }
}

template <typename Prob>
cudaError_t noalloc_setup(const wos_problem_desc& d, unsigned char* base, unsigned long long* stats_zero,
                          cudaStream_t st) {
  Prob h;
  fill_problem(h, d);
  NaBlob<Prob> blob;
  std::memcpy(&blob, &h, sizeof(Prob));
  noalloc_setup_kernel<Prob><<<1, 1, 0, st>>>(blob, reinterpret_cast<int4*>(base + kNaProblem),
                                              reinterpret_cast<unsigned long long*>(base + kNaCounter), stats_zero);
  return cudaGetLastError();
}

// validation without host allocation (no message strings)
bool na_field_ok(const wos_field_desc& f, int dim, bool is_source, bool needs_c2) {
  if (f.kind < WOS_FIELD_ZERO || f.kind > WOS_FIELD_GRID_BSPLINE) return false;
  if (f.kind == WOS_FIELD_MANUFACTURED && !is_source) return false;
  if (needs_c2 && f.kind == WOS_FIELD_GRID_LINEAR) return false;
  if (f.kind == WOS_FIELD_SST) {
    if (f.nterms < 0 || f.nterms > wos::kMaxTerms || (f.nterms > 0 && f.terms == nullptr)) return false;
    for (int n = 0; n < f.nterms; ++n) {
      if (!std::isfinite(f.terms[n].c)) return false;
      for (int d = 0; d < dim; ++d)
        if (f.terms[n].type[d] < WOS_ATOM_ONE || f.terms[n].type[d] > WOS_ATOM_QUAD ||
            !std::isfinite(f.terms[n].k[d]) || !std::isfinite(f.terms[n].phi[d]))
          return false;
    }
  }
  if (f.kind == WOS_FIELD_CONST && !std::isfinite(f.value)) return false;
  if (f.kind == WOS_FIELD_GRID_LINEAR || f.kind == WOS_FIELD_GRID_BSPLINE) {
    if (f.data == nullptr) return false;
    for (int d = 0; d < dim; ++d)
      if (f.res[d] < 2 || !(f.hi[d] > f.lo[d]) || !std::isfinite(f.lo[d]) || !std::isfinite(f.hi[d])) return false;
  }
  return true;
}

bool na_desc_ok(const wos_problem_desc* d) {
  if (d->dim != 2 && d->dim != 3) return false;
  const double* p = d->domain.p;
  for (int i = 0; i < 16; ++i)
    if (!std::isfinite(p[i])) return false;
  switch (d->domain.kind) {
    case WOS_DOMAIN_BOX:
      for (int i = 0; i < d->dim; ++i)
        if (!(p[3 + i] > p[i])) return false;
      break;
    case WOS_DOMAIN_BALL:
      if (!(p[3] > 0)) return false;
      break;
    case WOS_DOMAIN_ANNULUS:
      if (!(p[3] >= 0 && p[4] > p[3])) return false;
      break;
    case WOS_DOMAIN_ROUNDED_BOX:
      for (int i = 0; i < d->dim; ++i)
        if (!(p[3 + i] > 0 && p[6] >= 0 && p[6] <= p[3 + i])) return false;
      break;
    default:
      return false;
  }
  if (!na_field_ok(d->alpha, d->dim, false, true) || !na_field_ok(d->phi, d->dim, false, true) ||
      !na_field_ok(d->sigma, d->dim, false, false) || !na_field_ok(d->f, d->dim, true, false) ||
      !na_field_ok(d->g, d->dim, false, false) || !na_field_ok(d->um, d->dim, false, true))
    return false;
  if (d->alpha.kind == WOS_FIELD_ZERO) return false;
  if (d->alpha.kind == WOS_FIELD_CONST && !(d->alpha.value > 0)) return false;
  int total = 0;
  const wos_field_desc* fl[6] = {&d->alpha, &d->phi, &d->sigma, &d->f, &d->g, &d->um};
  for (auto* f : fl)
    if (f->kind == WOS_FIELD_SST) total += f->nterms;
  for (int k = 0; k < 3; ++k)
    if (k < d->dim && d->omega[k].kind != WOS_FIELD_ZERO) return false;  // the extra drift needs wos_solve
  return total <= wos::kMaxTerms;
}

}  // namespace

extern "C" int wos_solve_noalloc(const wos_problem_desc* desc, const float* pts, int64_t npts,
                                 const int32_t* walks, int32_t walks_uniform, const wos_params* prm,
                                 double* sum, double* sumsq, int64_t* count, uint64_t* stats, void* stream) {
  if (!desc || !prm) return WOS_EINVAL;
  if (prm->ww_lo != 0.0) return WOS_EUNSUPPORTED;
  if (!finite_pos(prm->eps) || !finite_pos(prm->sigma_bar) || prm->max_steps < 1 ||
      (prm->precision != WOS_FP32 && prm->precision != WOS_FP64))
    return WOS_EINVAL;
  if (!na_desc_ok(desc)) return WOS_EINVAL;
  if (npts < 0 || npts > 0xffffffffll) return WOS_EINVAL;
  if (walks != nullptr && npts > WOS_NOALLOC_MAX_VAR_POINTS) return WOS_EINVAL;  // prefix sums would not fit
  if (walks == nullptr && walks_uniform < 0) return WOS_EINVAL;
  if (npts == 0 || (walks == nullptr && walks_uniform == 0)) return WOS_OK;
  if (!pts || !sum || !sumsq || !count) return WOS_EINVAL;

  // The array's address on the current device.  In host code the name
  // g_noalloc_scratch is only a host-side stand-in, so the kernels get the address the
  // runtime reports.  It is resolved on every call (no allocation, not a stream
  // operation): a cached address would go stale if the host program reset the device
  // and the module were loaded again elsewhere.  The first call on a device also loads
  // the module there.
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return WOS_ECUDA;
  void* sym = nullptr;
  if (cudaGetSymbolAddress(&sym, g_noalloc_scratch) != cudaSuccess || sym == nullptr) return WOS_ECUDA;
  unsigned char* base = static_cast<unsigned char*>(sym);
  int num_sms = 0;
  if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return WOS_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  // problem description into the scratch, work counter (and default statistics) to zero
  const bool fp64 = prm->precision == WOS_FP64;
  const size_t pbytes = fp64 ? sizeof(DevProblem<double>) : sizeof(DevProblem<float>);
  unsigned long long* st_ptr = reinterpret_cast<unsigned long long*>(stats);
  unsigned long long* st_zero = nullptr;
  if (st_ptr == nullptr) st_ptr = st_zero = reinterpret_cast<unsigned long long*>(base + kNaStats);
  cudaError_t e = fp64 ? noalloc_setup<DevProblem<double>>(*desc, base, st_zero, st)
                       : noalloc_setup<DevProblem<float>>(*desc, base, st_zero, st);
  if (e != cudaSuccess) return WOS_ECUDA;

  const int64_t* walk_end = nullptr;
  uint64_t total;
  if (walks != nullptr) {
    int64_t* prefix = reinterpret_cast<int64_t*>(base + kNaPrefix);
    walk_prefix_kernel<<<1, 1024, 0, st>>>(walks, npts, prefix);
    if (cudaGetLastError() != cudaSuccess) return WOS_ECUDA;
    walk_end = prefix;
    total = ~0ull;
  } else {
    total = (uint64_t)npts * (uint64_t)walks_uniform;
  }

  wos::WalkLaunch L;
  std::memset(&L, 0, sizeof(L));
  L.problem = base + kNaProblem;
  L.problem_bytes = (int)pbytes;
  L.dim = desc->dim;
  L.pts = pts;
  L.npts = npts;
  L.walk_end = walk_end;
  L.walks_uniform = walks_uniform;
  L.total_items = total;
  L.seed = prm->seed;
  L.walk_offset = prm->walk_offset;
  L.eps = prm->eps;
  L.sigma_bar = prm->sigma_bar;
  L.max_steps = prm->max_steps;
  L.sum = sum;
  L.sumsq = sumsq;
  L.count = reinterpret_cast<unsigned long long*>(count);
  L.stats = st_ptr;
  L.work_counter = reinterpret_cast<unsigned long long*>(base + kNaCounter);
  L.radial_tab = nullptr;  // no tables here: the FP32 Newton starts from its closed-form guess
  e = fp64 ? wos::launch_walks_f64(L, num_sms, st) : wos::launch_walks_f32(L, num_sms, st);
  return e == cudaSuccess ? WOS_OK : WOS_ECUDA;
}
