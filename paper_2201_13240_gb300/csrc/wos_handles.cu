// wos_handles.cu -- the problem-statement calls of include/wos.h: domain and field
// handles (Sec. 3: the region Omega and the coefficient, source and boundary fields of
// eq. 1), problem assembly, the default delta-tracking bound (Sec. 5.1, Sec. 7.1),
// solves that return per-point means and variances (Sec. 2.2), one-call batches and
// the combined replay adjoint.  Every call is layered on the descriptor entry points
// (wos_problem_create, wos_sigma_bar, wos_solve, wos_batch_*, wos_adjoint_*), so a
// problem built from handles runs the same kernels as one built from a description.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "wos_capi_state.h"

struct wos_domain {
  int dim = 0;
  wos_domain_desc desc;        // mesh: verts / tris point into the vectors below
  std::vector<float> verts;    // host copy of a mesh's vertices
  std::vector<int32_t> tris;   // host copy of a mesh's triangles
};

struct wos_field {
  int dim = 0;                 // grids: their dimension; analytic fields: 0 (any)
  int family = 0;              // WOS_FIELD_* kind the caller asked for
  wos_field_desc desc;         // SST terms point into `terms`
  std::vector<wos_term> terms;
};

namespace {

int hfail(wos_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

int hcuda(wos_ctx* ctx, cudaError_t e, const char* what) {
  return hfail(ctx, WOS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool finite_all(const double* v, int n) {
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

struct HandleDeviceGuard {
  int prev = -1;
  explicit HandleDeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      prev = -1;
      (void)cudaGetLastError();
    }
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) (void)cudaGetLastError();
  }
  ~HandleDeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev && cudaSetDevice(prev) != cudaSuccess)
      (void)cudaGetLastError();
  }
};

// a closed, consistently oriented surface: every directed edge once, and its reverse too
bool mesh_closed(const std::vector<int32_t>& tris) {
  const size_t nt = tris.size() / 3;
  std::vector<uint64_t> dir;
  dir.reserve(3 * nt);
  for (size_t t = 0; t < nt; ++t)
    for (int e = 0; e < 3; ++e) {
      uint32_t a = (uint32_t)tris[3 * t + e], b = (uint32_t)tris[3 * t + (e + 1) % 3];
      if (a == b) return false;  // degenerate triangle
      dir.push_back(((uint64_t)a << 32) | b);
    }
  std::sort(dir.begin(), dir.end());
  for (size_t i = 1; i < dir.size(); ++i)
    if (dir[i] == dir[i - 1]) return false;  // an edge used twice in one direction
  for (uint64_t k : dir) {
    uint64_t rev = (k << 32) | (k >> 32);
    if (!std::binary_search(dir.begin(), dir.end(), rev)) return false;  // a boundary edge
  }
  return true;
}

// Chan, Golub and LeVeque's pairwise update of (mean, unbiased variance, count) with the
// raw sums of the new walks (n_b = cnt, sum, sumsq)
__global__ void merge_moments_kernel(const double* sum, const double* sumsq, const int64_t* cnt, int64_t n,
                                     double* mean, double* var, int64_t* count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t nb = cnt[i];
    if (nb <= 0) continue;
    const double db = (double)nb;
    const double mb = sum[i] / db;
    const double m2b = fmax(sumsq[i] - sum[i] * mb, 0.0);
    const int64_t na = count[i];
    double m, m2;
    if (na <= 0) {
      m = mb;
      m2 = m2b;
    } else {
      const double da = (double)na, ma = mean[i];
      const double m2a = (na > 1) ? var[i] * (da - 1.0) : 0.0;
      const double dn = da + db, delta = mb - ma;
      m = ma + delta * (db / dn);
      m2 = m2a + m2b + delta * delta * (da * db / dn);
    }
    const int64_t nt = (na > 0 ? na : 0) + nb;
    mean[i] = m;
    var[i] = (nt > 1) ? m2 / (double)(nt - 1) : 0.0;
    count[i] = nt;
  }
}

__global__ void to_float_kernel(const double* src, int64_t n, float* dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

int grid_blocks(const wos_ctx* ctx, int64_t n) {
  int64_t b = (n + 255) / 256;
  int64_t cap = (int64_t)ctx->num_sms * 8;
  return (int)std::max<int64_t>(1, std::min(b, cap));
}

// context-owned FP64 accumulators of at least npts points
int ensure_mv(wos_ctx* ctx, int64_t npts) {
  if (npts <= ctx->mv_cap) return WOS_OK;
  // an earlier call may still be reading the old buffers on some stream
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return hcuda(ctx, e, "synchronise before growing accumulators");
  if (ctx->mv_sum) cudaFree(ctx->mv_sum);
  if (ctx->mv_count) cudaFree(ctx->mv_count);
  ctx->mv_sum = nullptr;
  ctx->mv_count = nullptr;
  ctx->mv_cap = 0;
  e = cudaMalloc(&ctx->mv_sum, 2 * sizeof(double) * (size_t)npts);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->mv_count, sizeof(int64_t) * (size_t)npts);
  if (e != cudaSuccess) {
    if (ctx->mv_sum) cudaFree(ctx->mv_sum);
    ctx->mv_sum = nullptr;
    ctx->mv_count = nullptr;
    return hfail(ctx, WOS_ENOMEM, std::string("cudaMalloc(accumulators): ") + cudaGetErrorString(e));
  }
  ctx->mv_cap = npts;
  return WOS_OK;
}

int zero_mv(wos_ctx* ctx, int64_t npts, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(ctx->mv_sum, 0, 2 * sizeof(double) * (size_t)npts, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->mv_count, 0, sizeof(int64_t) * (size_t)npts, st);
  return e == cudaSuccess ? WOS_OK : hcuda(ctx, e, "zero accumulators");
}

int merge_mv(wos_ctx* ctx, int64_t npts, double* mean, double* var, int64_t* count, cudaStream_t st) {
  merge_moments_kernel<<<grid_blocks(ctx, npts), 256, 0, st>>>(ctx->mv_sum, ctx->mv_sum + npts, ctx->mv_count,
                                                                npts, mean, var, count);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WOS_OK : hcuda(ctx, e, "merge kernel");
}

int64_t grid_nodes(const DevField<double>& F, int dim) {
  int64_t n = 1;
  for (int d = 0; d < dim; ++d) n *= F.res[d];
  return n;
}

}  // namespace

extern "C" {

int wos_domain_box(wos_ctx* ctx, int32_t dim, const double* lo, const double* hi, wos_domain** out) {
  if (!out) return hfail(ctx, WOS_EINVAL, "null output");
  *out = nullptr;
  if (dim != 2 && dim != 3) return hfail(ctx, WOS_EINVAL, "dim must be 2 or 3");
  if (!lo || !hi || !finite_all(lo, dim) || !finite_all(hi, dim)) return hfail(ctx, WOS_EINVAL, "box corners");
  for (int d = 0; d < dim; ++d)
    if (!(hi[d] > lo[d])) return hfail(ctx, WOS_EINVAL, "box needs hi > lo in every axis");
  wos_domain* D = new wos_domain();
  std::memset(&D->desc, 0, sizeof(D->desc));
  D->dim = dim;
  D->desc.kind = WOS_DOMAIN_BOX;
  for (int d = 0; d < dim; ++d) {
    D->desc.p[d] = lo[d];
    D->desc.p[3 + d] = hi[d];
  }
  *out = D;
  return WOS_OK;
}

int wos_domain_sdf(wos_ctx* ctx, int32_t dim, int32_t kind, const double* params, wos_domain** out) {
  if (!out) return hfail(ctx, WOS_EINVAL, "null output");
  *out = nullptr;
  if (dim != 2 && dim != 3) return hfail(ctx, WOS_EINVAL, "dim must be 2 or 3");
  int np = 0;
  switch (kind) {
    case WOS_DOMAIN_BALL: np = 4; break;
    case WOS_DOMAIN_ANNULUS: np = 5; break;
    case WOS_DOMAIN_ROUNDED_BOX: np = 7; break;
    default: return hfail(ctx, WOS_EINVAL, "kind must be WOS_DOMAIN_BALL, _ANNULUS or _ROUNDED_BOX");
  }
  if (!params || !finite_all(params, np)) return hfail(ctx, WOS_EINVAL, "non-finite or missing parameters");
  const double* p = params;
  bool ok = true;
  if (kind == WOS_DOMAIN_BALL) ok = p[3] > 0;
  if (kind == WOS_DOMAIN_ANNULUS) ok = p[3] >= 0 && p[4] > p[3];
  if (kind == WOS_DOMAIN_ROUNDED_BOX)
    for (int d = 0; d < dim; ++d) ok = ok && p[3 + d] > 0 && p[6] >= 0 && p[6] <= p[3 + d];
  if (!ok) return hfail(ctx, WOS_EINVAL, "invalid radius, extent or corner radius");
  wos_domain* D = new wos_domain();
  std::memset(&D->desc, 0, sizeof(D->desc));
  D->dim = dim;
  D->desc.kind = kind;
  for (int i = 0; i < np; ++i) D->desc.p[i] = p[i];
  *out = D;
  return WOS_OK;
}

int wos_domain_mesh(wos_ctx* ctx, const float* verts, int64_t nverts, const int32_t* tris, int64_t ntris,
                    wos_domain** out) {
  if (!out) return hfail(ctx, WOS_EINVAL, "null output");
  *out = nullptr;
  if (!verts || !tris || nverts < 3 || ntris < 4) return hfail(ctx, WOS_EINVAL, "a closed mesh needs >= 4 triangles");
  if (nverts > (int64_t)INT32_MAX || ntris > (int64_t)INT32_MAX / 3) return hfail(ctx, WOS_EINVAL, "mesh too large");
  HandleDeviceGuard g(ctx ? ctx->device : 0);
  wos_domain* D = new wos_domain();
  D->verts.resize(3 * (size_t)nverts);
  D->tris.resize(3 * (size_t)ntris);
  cudaError_t e = cudaMemcpy(D->verts.data(), verts, D->verts.size() * sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(D->tris.data(), tris, D->tris.size() * sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    delete D;
    return hcuda(ctx, e, "copy mesh arrays to the host");
  }
  for (float v : D->verts)
    if (!std::isfinite(v)) {
      delete D;
      return hfail(ctx, WOS_EINVAL, "mesh: non-finite vertex");
    }
  for (int32_t t : D->tris)
    if (t < 0 || t >= nverts) {
      delete D;
      return hfail(ctx, WOS_EINVAL, "mesh: vertex index out of range");
    }
  if (!mesh_closed(D->tris)) {
    delete D;
    return hfail(ctx, WOS_EINVAL, "mesh: not a closed, consistently oriented surface");
  }
  std::memset(&D->desc, 0, sizeof(D->desc));
  D->dim = 3;
  D->desc.kind = WOS_DOMAIN_MESH;
  D->desc.verts = D->verts.data();
  D->desc.nverts = nverts;
  D->desc.tris = D->tris.data();
  D->desc.ntris = ntris;
  *out = D;
  return WOS_OK;
}

int wos_domain_destroy(wos_domain* dom) {
  if (!dom) return WOS_EINVAL;
  delete dom;
  return WOS_OK;
}

int wos_field_analytic(wos_ctx* ctx, int32_t family_id, const double* params, int32_t nparams, wos_field** out) {
  if (!out) return hfail(ctx, WOS_EINVAL, "null output");
  *out = nullptr;
  if (nparams < 0 || (nparams > 0 && !params)) return hfail(ctx, WOS_EINVAL, "missing parameters");
  if (nparams > 0 && !finite_all(params, nparams)) return hfail(ctx, WOS_EINVAL, "non-finite parameter");
  wos_field* F = new wos_field();
  std::memset(&F->desc, 0, sizeof(F->desc));
  F->family = family_id;
  switch (family_id) {
    case WOS_FIELD_ZERO:
      if (nparams != 0) break;
      F->desc.kind = WOS_FIELD_ZERO;
      *out = F;
      return WOS_OK;
    case WOS_FIELD_CONST:
      if (nparams != 1) break;
      F->desc.kind = WOS_FIELD_CONST;
      F->desc.value = params[0];
      *out = F;
      return WOS_OK;
    case WOS_FIELD_SST:
    case WOS_FIELD_MANUFACTURED: {
      if (nparams % 10 != 0 || nparams / 10 > wos::kMaxTerms) break;
      const int nt = nparams / 10;
      F->terms.resize(nt > 0 ? nt : 1);
      bool ok = true;
      for (int n = 0; n < nt; ++n) {
        const double* q = params + 10 * n;
        wos_term& T = F->terms[n];
        T.c = q[0];
        for (int d = 0; d < 3; ++d) {
          const double ty = q[1 + d];
          ok = ok && ty == std::floor(ty) && ty >= WOS_ATOM_ONE && ty <= WOS_ATOM_QUAD;
          T.type[d] = ok ? (int32_t)ty : 0;
          T.k[d] = q[4 + d];
          T.phi[d] = q[7 + d];
        }
      }
      if (!ok) break;
      // a manufactured source keeps u_m's terms; wos_problem_assemble places them
      F->desc.kind = WOS_FIELD_SST;
      F->desc.nterms = nt;
      F->desc.terms = F->terms.data();
      *out = F;
      return WOS_OK;
    }
    default:
      break;
  }
  delete F;
  return hfail(ctx, WOS_EINVAL, "unknown family or wrong parameter count / atom type");
}

int wos_field_grid(wos_ctx* ctx, int32_t dim, const int32_t* res, const double* lo, const double* hi,
                   const float* data, int32_t interp, wos_field** out) {
  if (!out) return hfail(ctx, WOS_EINVAL, "null output");
  *out = nullptr;
  if (dim != 2 && dim != 3) return hfail(ctx, WOS_EINVAL, "dim must be 2 or 3");
  if (interp != WOS_FIELD_GRID_LINEAR && interp != WOS_FIELD_GRID_BSPLINE)
    return hfail(ctx, WOS_EINVAL, "interp must be WOS_FIELD_GRID_LINEAR or WOS_FIELD_GRID_BSPLINE");
  if (!res || !lo || !hi || !data) return hfail(ctx, WOS_EINVAL, "null grid argument");
  if (!finite_all(lo, dim) || !finite_all(hi, dim)) return hfail(ctx, WOS_EINVAL, "non-finite grid box");
  for (int d = 0; d < dim; ++d)
    if (res[d] < 2 || !(hi[d] > lo[d])) return hfail(ctx, WOS_EINVAL, "grid needs res >= 2 and hi > lo");
  wos_field* F = new wos_field();
  std::memset(&F->desc, 0, sizeof(F->desc));
  F->dim = dim;
  F->family = interp;
  F->desc.kind = interp;
  for (int d = 0; d < 3; ++d) {
    F->desc.res[d] = d < dim ? res[d] : 1;
    F->desc.lo[d] = d < dim ? lo[d] : 0.0;
    F->desc.hi[d] = d < dim ? hi[d] : 1.0;
  }
  F->desc.data = data;
  *out = F;
  return WOS_OK;
}

int wos_field_destroy(wos_field* field) {
  if (!field) return WOS_EINVAL;
  delete field;
  return WOS_OK;
}

int wos_problem_assemble(wos_ctx* ctx, const wos_domain* dom, const wos_field* alpha, const wos_field* sigma,
                         const wos_field* phi, const wos_field* f, const wos_field* g, wos_problem** prob) {
  if (!ctx) return WOS_EINVAL;
  if (!prob) return hfail(ctx, WOS_EINVAL, "null output");
  *prob = nullptr;
  if (!dom || !alpha || !sigma || !f || !g) return hfail(ctx, WOS_EINVAL, "domain, alpha, sigma, f and g are required");
  const wos_field* all[5] = {alpha, sigma, phi, f, g};
  for (const wos_field* F : all)
    if (F && F->dim != 0 && F->dim != dom->dim) return hfail(ctx, WOS_EINVAL, "a grid's dimension differs from the domain's");
  for (const wos_field* F : {alpha, sigma, phi, g})
    if (F && F->family == WOS_FIELD_MANUFACTURED) return hfail(ctx, WOS_EINVAL, "only the source f may be MANUFACTURED");
  wos_problem_desc d;
  std::memset(&d, 0, sizeof(d));
  d.dim = dom->dim;
  d.domain = dom->desc;
  d.alpha = alpha->desc;
  if (phi) d.phi = phi->desc;
  d.sigma = sigma->desc;
  d.g = g->desc;
  if (f->family == WOS_FIELD_MANUFACTURED) {
    d.f.kind = WOS_FIELD_MANUFACTURED;
    d.um = f->desc;  // u_m's terms; the source is derived from it with the problem's fields
  } else {
    d.f = f->desc;
  }
  return wos_problem_create(ctx, &d, prob);
}

int wos_problem_sigma_bar(wos_ctx* ctx, const wos_problem* prob, double* sigma_bar, double* sigma_prime_min,
                          double* sigma_prime_max) {
  if (!ctx) return WOS_EINVAL;
  if (!prob || !sigma_bar) return hfail(ctx, WOS_EINVAL, "null problem or output");
  double mn = 0.0, mx = 0.0;
  int rc = wos_sigma_bar(ctx, prob, prob->dim == 2 ? 256 : 128, sigma_bar, &mn, &mx, nullptr);
  if (rc != WOS_OK) return rc;
  if (sigma_prime_min) *sigma_prime_min = mn;
  if (sigma_prime_max) *sigma_prime_max = mx;
  return WOS_OK;
}

int wos_solve_mean(wos_ctx* ctx, const wos_problem* prob, const float* pts, int64_t npts, const int32_t* walks,
                   int32_t walks_uniform, const wos_params* params, double* mean, double* var, int64_t* count,
                   uint64_t* stats, void* stream) {
  if (!ctx) return WOS_EINVAL;
  if (!prob) return hfail(ctx, WOS_EINVAL, "null problem");
  if (npts < 0) return hfail(ctx, WOS_EINVAL, "negative size");
  if (npts == 0) return WOS_OK;
  if (!mean || !var || !count) return hfail(ctx, WOS_EINVAL, "null mean, var or count");
  HandleDeviceGuard g(ctx->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = ensure_mv(ctx, npts);
  if (rc == WOS_OK) rc = zero_mv(ctx, npts, st);
  if (rc == WOS_OK)
    rc = wos_solve(ctx, prob, pts, npts, walks, walks_uniform, params, ctx->mv_sum, ctx->mv_sum + npts,
                   ctx->mv_count, stats, stream);
  if (rc == WOS_OK) rc = merge_mv(ctx, npts, mean, var, count, st);
  return rc;
}

int wos_solve_batched(wos_ctx* ctx, const wos_problem* const* probs, int32_t nprob, const int64_t* pt_offsets,
                      const double* sigma_bars, const float* pts, const int32_t* walks, int32_t walks_uniform,
                      const wos_params* params, double* mean, double* var, int64_t* count, uint64_t* stats,
                      void* stream) {
  if (!ctx) return WOS_EINVAL;
  if (!probs || nprob < 1 || !pt_offsets) return hfail(ctx, WOS_EINVAL, "null problems or offsets");
  if (!mean || !var || !count) return hfail(ctx, WOS_EINVAL, "null mean, var or count");
  for (int32_t i = 0; i < nprob; ++i)
    if (!probs[i]) return hfail(ctx, WOS_EINVAL, "null problem in the list");
  std::vector<double> sb(nprob);
  for (int32_t i = 0; i < nprob; ++i) {
    if (sigma_bars) {
      sb[i] = sigma_bars[i];
    } else {
      int rc = wos_problem_sigma_bar(ctx, probs[i], &sb[i], nullptr, nullptr);
      if (rc != WOS_OK) return rc;
    }
  }
  const int64_t npts = pt_offsets[nprob];
  wos_batch* b = nullptr;
  int rc = wos_batch_create(ctx, probs, nprob, pt_offsets, sb.data(), &b);
  if (rc != WOS_OK) return rc;
  HandleDeviceGuard g(ctx->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (npts > 0) {
    rc = ensure_mv(ctx, npts);
    if (rc == WOS_OK) rc = zero_mv(ctx, npts, st);
    if (rc == WOS_OK)
      rc = wos_solve_batch(ctx, b, pts, walks, walks_uniform, params, ctx->mv_sum, ctx->mv_sum + npts,
                           ctx->mv_count, stats, stream);
    if (rc == WOS_OK) rc = merge_mv(ctx, npts, mean, var, count, st);
  }
  // the batch's device tables are read by the launch: finish it before freeing them
  cudaError_t e = cudaStreamSynchronize(st);
  if (rc == WOS_OK && e != cudaSuccess) rc = hcuda(ctx, e, "batched solve");
  wos_batch_destroy(b);
  return rc;
}

int wos_adjoint(wos_ctx* ctx, const wos_problem* prob, const float* pts, int64_t npts, int32_t walks_uniform,
                const wos_params* params, const double* grad_u, float* grad_sigma, float* grad_alpha,
                uint64_t* stats, void* stream) {
  if (!ctx) return WOS_EINVAL;
  if (!prob) return hfail(ctx, WOS_EINVAL, "null problem");
  const DevProblem<double>& P = prob->host64;
  int64_t ns = 0, na = 0;
  if (grad_sigma) {
    if (P.sigma.kind != wos::F_GRID_LINEAR)
      return hfail(ctx, WOS_EUNSUPPORTED, "the sigma gradient needs sigma as a multilinear grid");
    ns = grid_nodes(P.sigma, prob->dim);
  }
  if (grad_alpha) {
    if (P.alpha.kind != wos::F_GRID_BSPLINE)
      return hfail(ctx, WOS_EUNSUPPORTED, "the alpha gradient needs alpha as a B-spline grid");
    na = grid_nodes(P.alpha, prob->dim);
  }
  if (ns + na == 0) return WOS_OK;
  HandleDeviceGuard g(ctx->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (ns + na > ctx->adj_cap) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return hcuda(ctx, e, "synchronise before growing the gradient buffer");
    if (ctx->adj_buf) cudaFree(ctx->adj_buf);
    ctx->adj_buf = nullptr;
    ctx->adj_cap = 0;
    e = cudaMalloc(&ctx->adj_buf, sizeof(double) * (size_t)(ns + na));
    if (e != cudaSuccess) return hfail(ctx, WOS_ENOMEM, std::string("cudaMalloc(gradient): ") + cudaGetErrorString(e));
    ctx->adj_cap = ns + na;
  }
  cudaError_t e = cudaMemsetAsync(ctx->adj_buf, 0, sizeof(double) * (size_t)(ns + na), st);
  if (e != cudaSuccess) return hcuda(ctx, e, "zero gradient buffer");
  int rc = WOS_OK;
  if (grad_sigma)
    rc = wos_adjoint_sigma(ctx, prob, pts, npts, walks_uniform, params, grad_u, ctx->adj_buf, stats, stream);
  if (rc == WOS_OK && grad_alpha)
    rc = wos_adjoint_alpha(ctx, prob, pts, npts, walks_uniform, params, grad_u, ctx->adj_buf + ns, stats, stream);
  if (rc != WOS_OK) return rc;
  if (grad_sigma) to_float_kernel<<<grid_blocks(ctx, ns), 256, 0, st>>>(ctx->adj_buf, ns, grad_sigma);
  if (grad_alpha) to_float_kernel<<<grid_blocks(ctx, na), 256, 0, st>>>(ctx->adj_buf + ns, na, grad_alpha);
  e = cudaGetLastError();
  return e == cudaSuccess ? WOS_OK : hcuda(ctx, e, "gradient conversion");
}

}  // extern "C"
