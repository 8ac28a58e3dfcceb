// wos_adjoint_impl.cuh -- gradient of the delta-tracking estimate with respect to
// the node values of a multilinear screening grid sigma, by replaying each walk.
//
// Given sigma_bar, nothing that steers a walk depends on sigma: distances, the
// Green's-function samples, and the null/boundary decision mu <= sigma_bar |G|
// use only the geometry, sigma_bar and the randoms (Sec. 5.1, eq. 11).  sigma
// enters only through the null weights w_j = 1 - sigma'(y_j)/sigma_bar, with
// sigma' = sigma/alpha + (terms of alpha and Phi) (Sec. 4.1), so
//     d sigma'(y) / d sigma_m = N_m(y) / alpha(y),
// N_m the multilinear weight of node m at y.  A walk's estimate is
//     u = e^{-gamma(x_0)} A,   A = sum_k W_k |G_k| f'(y_k) + W_n e^{gamma(x_n)} g(xbar_n),
// W_k the product of the null weights before step k.  The terms up to and
// including step j do not contain w_j; every later term contains it once, so
//     dA / dw_j = (A - P_{j+1}) / w_j,
// P_{j+1} the sum of the terms up to step j.  Each walk therefore runs twice
// on the same Philox stream: a first pass for A, a second that recomputes
// the prefix and, at every null event j, adds
//     c * (A - P_{j+1}) / w_j * (-N_m(y_j) / (alpha(y_j) sigma_bar))
// to the gradient of node m, c = grad_u[p] e^{-gamma(x_0)} / (walks of point p).
// The estimator's paths are not stored (path replay).
//
// ALPHA: the gradient with respect to the control values alpha_m of a cubic
// B-spline alpha grid.  alpha enters through gamma = (ln alpha + Phi)/2, so
// through e^{-gamma(x_0)}, the sources f'(y) = e^{gamma} f / alpha, the null
// weights through sigma' = sigma/alpha + Lap gamma + |grad gamma|^2, and the
// boundary factor e^{gamma(x_n)} (Sec. 4.1, App. A).  With N_m the basis function
// of node m, d gamma / d alpha_m = N_m / (2 alpha) and d ln f' / d alpha_m = -N_m/(2 alpha);
// d sigma'/d alpha_m = cN N_m + cG . grad N_m + cL Lap N_m with
//   cN = -sigma/alpha^2 - Lap alpha/(2 alpha^2) + |grad alpha|^2/alpha^3 - grad gamma . grad alpha/alpha^2,
//   cG = grad gamma/alpha - grad alpha/alpha^2,   cL = 1/(2 alpha).
// So the replay scatters, per step k at y_k, c W_k |G_k| f'_k (-1/(2 alpha)) N_m plus,
// at a null event, c (A - P_{k+1})/w_k (-1/sigma_bar) d sigma'/d alpha_m; at the end
// c W_n e^{gamma(x_n)} g(xbar_n) / (2 alpha(x_n)) N_m(x_n); and once per walk
// -c A / (2 alpha(x_0)) N_m(x_0).  Small grids are accumulated per CTA in shared
// memory in the walk's precision (FP32 shared atomics are native; FP64 ones are not)
// and added to the FP64 gradient once per CTA.
#pragma once

#if !defined(__CUDACC_RTC__)
#include <cuda_runtime.h>
#endif

#include "wos_internal.h"
#include "wos_math.cuh"
#include "wos_problem.cuh"

namespace wos {

constexpr int kAdjBlock = 128;

template <int DIM, typename R>
__device__ __forceinline__ void grid_scatter(const DevField<R>& F, const R* y, R val, double* grad) {
  int i0[3] = {0, 0, 0};
  R t[3] = {R(0), R(0), R(0)};
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    R s = (y[d] - F.lo[d]) * F.inv_h[d];
    s = w_fmin(w_fmax(s, R(0)), R(F.res[d] - 1));
    int i = (int)s;
    if (i > F.res[d] - 2) i = F.res[d] - 2;
    i0[d] = i;
    t[d] = s - R(i);
  }
  const int nc = (DIM == 3) ? 8 : 4;
#pragma unroll
  for (int c = 0; c < nc; ++c) {
    R w = val;
    int64_t idx = 0, stride = 1;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      int o = (c >> d) & 1;
      w *= (o ? t[d] : R(1) - t[d]);
      idx += (int64_t)(i0[d] + o) * stride;
      stride *= F.res[d];
    }
    if (w != R(0)) atomicAdd(&grad[idx], (double)w);
  }
}

// add vN N_m + vG . grad N_m + vL Lap N_m at y to grad[m] over the 4^DIM nodes of
// the cubic B-spline support (indices clamped as in grid_bspline)
// grad is indexed j0 + s1 j1 + s2 j2: the grid's own layout in global memory, a padded one
// (s1 = res0 + 1, s2 = s1 res1 + 1) for the per-CTA copy in shared memory, which spreads the
// rows of one support over different banks.
template <int DIM, typename R, typename A>
__device__ void bspline_scatter(const DevField<R>& F, const R* y, R vN, const R* vG, R vL, A* grad, int64_t s1,
                                int64_t s2) {
  int ib[3] = {0, 0, 0};
  R B[3][4], B1[3][4], B2[3][4];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
#pragma unroll
    for (int a = 0; a < 4; ++a) { B[d][a] = (a == 0) ? R(1) : R(0); B1[d][a] = R(0); B2[d][a] = R(0); }
  }
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    R s = (y[d] - F.lo[d]) * F.inv_h[d];
    R fs = floor(s);
    ib[d] = (int)fs - 1;
    bspline_w(s - fs, B[d], B1[d], B2[d]);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      B1[d][a] *= F.inv_h[d];
      B2[d][a] *= F.inv_h[d] * F.inv_h[d];
    }
  }
  // clamped control indices per axis, once: x offsets and the row / plane offsets (32-bit:
  // grids stay far below 2^31 nodes)
  const int t1 = (int)s1, t2 = (int)s2;
  int o0[4], o1[4], o2[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    o0[a] = min(max(ib[0] + a, 0), F.res[0] - 1);
    o1[a] = t1 * min(max(ib[1] + a, 0), F.res[1] - 1);
    o2[a] = (DIM == 3) ? t2 * min(max(ib[2] + a, 0), F.res[2] - 1) : 0;
  }
  // Rows (c1, c2) of the support are visited in an order rotated by the lane, so lanes
  // whose points share a cell (walks of one point start together) add to different
  // addresses at the same time instead of serialising on one.
  auto sel4 = [](const R* v, int i) { return i == 0 ? v[0] : (i == 1 ? v[1] : (i == 2 ? v[2] : v[3])); };
  auto sel4i = [](const int* v, int i) { return i == 0 ? v[0] : (i == 1 ? v[1] : (i == 2 ? v[2] : v[3])); };
  const int nrows = (DIM == 3) ? 16 : 4;
  const int rot = (int)(threadIdx.x & 31);
  for (int k = 0; k < nrows; ++k) {
    const int r = (k + rot) & (nrows - 1);
    const int c1 = r & 3, c2 = (DIM == 3) ? (r >> 2) : 0;
    const R b1 = sel4(B[1], c1), d1 = sel4(B1[1], c1), e1 = sel4(B2[1], c1);
    const R b2 = (DIM == 3) ? sel4(B[2], c2) : R(1), d2 = (DIM == 3) ? sel4(B1[2], c2) : R(0);
    const R e2 = (DIM == 3) ? sel4(B2[2], c2) : R(0);
    const R b12 = b1 * b2;
    // the tap (c0, c1, c2) is b0 P + B1_0 Q + B2_0 T with the row's P, Q, T: the value,
    // gradient and Laplacian weights factored along x
    R Prow = vN * b12 + vG[1] * d1 * b2 + vL * (e1 * b2 + b1 * e2);
    if (DIM == 3) Prow += vG[2] * b1 * d2;
    const R Qrow = vG[0] * b12, Trow = vL * b12;
    A* row = grad + (sel4i(o1, c1) + sel4i(o2, c2));
#pragma unroll
    for (int c0 = 0; c0 < 4; ++c0) {
      const R val = B[0][c0] * Prow + B1[0][c0] * Qrow + B2[0][c0] * Trow;
      if (val != R(0)) atomicAdd(&row[o0[c0]], A(val));
    }
  }
}

// d sigma' / d alpha_m = cN N_m + cG . grad N_m + cL Lap N_m at y, from the fields coeffs
// evaluated there (in the walk's precision: FP64 arithmetic is a small fraction of FP32's
// rate here)
template <int DIM, typename R>
__device__ void alpha_sensitivity(const FieldsAt<R>& F, R* cN, R* cG, R* cL) {
  const FieldVal<R>& A = F.A;
  const FieldVal<R>& Ph = F.Ph;
  const R Sv = F.S;
  const R ia = R(1) / A.v;
  const R ga[3] = {A.gx, A.gy, A.gz}, gp[3] = {Ph.gx, Ph.gy, Ph.gz};
  R na2 = R(0), gg_ga = R(0), gg[3] = {R(0), R(0), R(0)};
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    gg[d] = R(0.5) * (ga[d] * ia + gp[d]);
    na2 += ga[d] * ga[d];
    gg_ga += gg[d] * ga[d];
  }
  const R ia2 = ia * ia;
  *cN = -Sv * ia2 - R(0.5) * A.lap * ia2 + na2 * ia2 * ia - gg_ga * ia2;
#pragma unroll
  for (int d = 0; d < 3; ++d) cG[d] = (d < DIM) ? gg[d] * ia - ga[d] * ia2 : R(0);
  *cL = R(0.5) * ia;
}

// Compiled at run time for one problem (WOS_JIT_FIELDS, wos_problem_specialize with the
// adjoint variant) the fields are the problem's generated code and the kernel is named
// wos_adjoint_spec_kernel, so that profiles tell the two apart.
#if defined(WOS_JIT_FIELDS)
#define WOS_ADJOINT_KERNEL wos_adjoint_spec_kernel
#else
#define WOS_ADJOINT_KERNEL wos_adjoint_kernel
#endif
// PASS 1 runs every walk's first replay only and stores its total A in L.totals (indexed by
// the walk's place in the launch); PASS 2 starts every walk in the second replay from that
// total and scatters.  The walks of one launch are items L.item_base .. + L.total_items.  Two
// launches instead of one keep the lanes of a warp in one phase: in a single launch, lanes
// whose walks were still in their first replay idled through the others' scatters.
template <int DIM, typename R, bool ALPHA, int PASS>
__global__ void __launch_bounds__(kAdjBlock, 4) WOS_ADJOINT_KERNEL(AdjLaunch L) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  {
    const int4* src = reinterpret_cast<const int4*>(L.problem);
    int4* dst = reinterpret_cast<int4*>(smem_raw);
    for (int i = threadIdx.x; i < L.problem_bytes / 16; i += blockDim.x) dst[i] = src[i];
  }
  // alpha: per-CTA accumulators in the walk's precision (FP32 shared atomics are native)
  R* gpriv = reinterpret_cast<R*>(smem_raw + L.problem_bytes);
  const bool priv = ALPHA && PASS == 2 && L.priv_nodes > 0;
  R* totals = reinterpret_cast<R*>(L.totals);
  const DevProblem<R>& Pg0 = *reinterpret_cast<const DevProblem<R>*>(L.problem);
  const int64_t ares0 = Pg0.alpha.res[0], ares1 = Pg0.alpha.res[1];
  const int64_t ps1 = ares0 + 1, ps2 = ps1 * ares1 + 1;  // padded shared layout
  if (priv)
    for (int i = threadIdx.x; i < L.priv_nodes; i += blockDim.x) gpriv[i] = R(0);
  __syncthreads();
  const DevProblem<R>& P = *reinterpret_cast<const DevProblem<R>*>(smem_raw);
#define WOS_ALPHA_SCATTER(pt, a, b, c)                                                   \
  do {                                                                                   \
    if (priv) bspline_scatter<DIM, R, R>(P.alpha, pt, a, b, c, gpriv, ps1, ps2);         \
    else bspline_scatter<DIM, R, double>(P.alpha, pt, a, b, c, L.grad_alpha, ares0, ares0 * ares1); \
  } while (0)
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  const R eps = R(L.eps), s_root = w_sqrt(R(L.sigma_bar));
  const R inv_sb = R(1) / R(L.sigma_bar);
  const uint32_t max_k = (L.max_steps >= (int64_t)0xffffffffll) ? 0xffffffffu : (uint32_t)L.max_steps;
  const double inv_walks = 1.0 / (double)L.walks_uniform;

  uint64_t chunk_next = 0, chunk_end = 0;
  const uint64_t magic = (L.walks_uniform > 0) ? ~0ull / (uint64_t)L.walks_uniform : 0ull;
  bool exhausted = false, active = false;
  // walk state; pass 1 computes the total A, pass 2 replays and scatters
  R x[3] = {R(0), R(0), R(0)}, W = R(1), acc = R(0), total = R(0);
  R xbp[3] = {R(0), R(0), R(0)};  // previous closest boundary point (bounds the next mesh query)
  uint32_t p = 0, w = 0, k = 0;
  uint64_t slot = 0;  // the walk's place in the launch (index into L.totals)
  bool fresh = false;  // pass 2: the walk's first iteration (at x_0) is next
  R coef = R(0);  // grad_u e^{-gamma(x_0)} / walks of the walk's point (FP64 only when R is)
  unsigned long long st_steps = 0;
  uint32_t st_walks = 0, st_capped = 0;

  for (;;) {
    unsigned need = __ballot_sync(0xffffffffu, !active);
    while (need != 0u && !exhausted) {
      if (chunk_next >= chunk_end) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(L.work_counter, 64ull);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= L.total_items) {
          exhausted = true;
          break;
        }
        chunk_next = base;
        chunk_end = (base + 64 < L.total_items) ? base + 64 : L.total_items;
      }
      unsigned nneed = __popc(need);
      uint64_t avail = chunk_end - chunk_next;
      unsigned take = (avail < nneed) ? (unsigned)avail : nneed;
      unsigned rank = __popc(need & lt_mask);
      if (!active && rank < take) {
        // item / walks_uniform by a multiply-high and one correction (as in the walk kernel)
        const uint64_t item = L.item_base + chunk_next + rank, dw = (uint64_t)L.walks_uniform;
        uint64_t pp = __umul64hi(item, magic), jj = item - pp * dw;
        if (jj >= dw) {
          ++pp;
          jj -= dw;
        }
        p = (uint32_t)pp;
        w = (uint32_t)(L.walk_offset + jj);
#pragma unroll
        for (int d = 0; d < 3; ++d) x[d] = (d < DIM) ? R(__ldg(&L.pts[(int64_t)d * L.npts + (int64_t)p])) : R(0);
        W = R(1);
        acc = R(0);
        k = 0;
        slot = chunk_next + rank;
        if (PASS == 2) {
          total = totals[slot];
          fresh = true;
        }
        active = true;
      }
      chunk_next += take;
      need = __ballot_sync(0xffffffffu, !active);
    }
    if (__ballot_sync(0xffffffffu, active) == 0u) break;
    if (!active) continue;

    // pass 2 gives each walk one iteration of its own at x_0 first: the fields there give
    // e^{-gamma(x_0)} and the alpha term of x_0, which then goes through the same scatter
    // call as the steps' and the boundary's (lanes that start, step or end a walk in one
    // iteration scatter together instead of one after another)
    const bool first = (PASS == 2) && fresh;
    R y[3] = {x[0], x[1], x[2]};
    R xb[3] = {R(0), R(0), R(0)};
    R d = R(0), dd = R(0), mu = R(1), Gn = R(0), PB = R(0);
    R dz[3] = {R(0), R(0), R(0)};
    bool ends = false;
    if (!first) {
      R bound2 = R(INFINITY);
      if (P.domain_kind == D_MESH && k > 0) {
        R e0 = x[0] - xbp[0], e1 = x[1] - xbp[1], e2 = x[2] - xbp[2];
        bound2 = e0 * e0 + e1 * e1 + e2 * e2;
      }
      d = distance<DIM>(P, x, xb, bound2);
#pragma unroll
      for (int i = 0; i < 3; ++i) xbp[i] = xb[i];
      ends = !(d >= eps) || k >= max_k;
      dd = w_fmax(d, R(0));
      U4 r0 = philox4x32_10_rk(U4{p, w, k, 0u}, L.rk);
      R ur;
      R dy[3] = {R(0), R(0), R(0)};
      if (DIM == 2) {
        mu = to_uniform<R>(r0.x);
        ur = to_uniform<R>(r0.y);
        w_sincospi2(to_uniform<R>(r0.z), &dy[1], &dy[0]);
        w_sincospi2(to_uniform<R>(r0.w), &dz[1], &dz[0]);
      } else {
        // the walk kernel's six 21-bit uniforms of one block
        uint32_t f[6];
        split21(r0, f);
        mu = u21<R>(f[0]);
        ur = u21<R>(f[1]);
        R cy = R(1) - R(2) * u21<R>(f[2]);
        R sy = w_sqrt_fast(w_fmax(R(0), R(1) - cy * cy));
        R sp_, cp_;
        w_sincospi2(u21<R>(f[3]), &sp_, &cp_);
        dy[0] = sy * cp_; dy[1] = sy * sp_; dy[2] = cy;
        R cz = R(1) - R(2) * u21<R>(f[4]);
        R sz = w_sqrt_fast(w_fmax(R(0), R(1) - cz * cz));
        w_sincospi2(u21<R>(f[5]), &sp_, &cp_);
        dz[0] = sz * cp_; dz[1] = sz * sp_; dz[2] = cz;
      }
      R a = s_root * dd;
      R q = green_q<DIM, R>(a);
      Gn = dd * dd * q;
      PB = a * a * q;
      R r = sample_radius<DIM, R>(a, ur, nullptr, (sizeof(R) == 4) ? L.radial_tab : nullptr) * dd;
#pragma unroll
      for (int i = 0; i < DIM; ++i) y[i] = ends ? x[i] : x[i] + r * dy[i];
    }
    R spy, fpy, gam, al;
    FieldsAt<R> fat;
    coeffs<DIM, R, false>(P, y, &spy, &fpy, &gam, &al, nullptr, (ALPHA && PASS == 2) ? &fat : nullptr);
    // alpha scatter of this iteration: vN N_m + vG . grad N_m + vL Lap N_m at y
    R vN = R(0), vG[3] = {R(0), R(0), R(0)}, vL = R(0);
    if (first) {
      // grad_u e^{-gamma(x_0)} / walks; alpha: -A N_m(x_0) / (2 alpha(x_0))
      coef = R(__ldg(&L.grad_u[p]) * inv_walks) * w_exp(-gam);
      if (ALPHA) vN = -coef * total * R(0.5) / al;
      fresh = false;
    } else if (ends) {
      bool capped = (d >= eps);
      if (!capped) {
        const R bterm = W * w_exp(gam) * g_at<DIM>(P, xb);
        acc += bterm;
        // boundary factor e^{gamma(x_n)}: d/d alpha_m = N_m(x_n) / (2 alpha(x_n)) times the term
        if (ALPHA && PASS == 2) vN = coef * bterm * R(0.5) / al;
      }
      if (PASS == 1) {
        totals[slot] = acc;  // the walk's total; the second pass replays it
      } else {
        ++st_walks;
        if (capped) ++st_capped;
      }
      active = false;
    } else {
      const R src = W * Gn * fpy;
      acc += src;
      // source f'(y): d/d alpha_m = -N_m(y) / (2 alpha(y)) times the term
      if (ALPHA && PASS == 2) vN = -coef * src * R(0.5) / al;
      if (mu <= PB) {
        const R wj = R(1) - spy * inv_sb;
        if (PASS == 2) {
          // d total / d w_j = (A - P_{j+1}) / w_j
          const R rem = (total - acc) / wj;
          if (ALPHA) {
            // d w_j / d alpha_m = -(1/sigma_bar) d sigma'/d alpha_m
            const R rj = -coef * rem * inv_sb;
            R cN, cG[3], cL;
            alpha_sensitivity<DIM, R>(fat, &cN, cG, &cL);
            if (isfinite(rj)) {
              vN += rj * cN;
#pragma unroll
              for (int i = 0; i < 3; ++i) vG[i] = rj * cG[i];
              vL = rj * cL;
            }
          } else {
            // d w_j / d sigma_m = -N_m(y) / (alpha(y) sigma_bar)
            const R val = -coef * rem * inv_sb / al;
            if (isfinite(val) && val != R(0)) grid_scatter<DIM, R>(P.sigma, y, val, L.grad_sigma);
          }
        }
        W *= wj;
#pragma unroll
        for (int i = 0; i < DIM; ++i) x[i] = y[i];
      } else {
#pragma unroll
        for (int i = 0; i < DIM; ++i) x[i] = x[i] + dd * dz[i];
      }
      if (PASS == 2) ++st_steps;
      ++k;
    }
    if (ALPHA && PASS == 2 && isfinite(vN) && (vN != R(0) || vL != R(0))) WOS_ALPHA_SCATTER(y, vN, vG, vL);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    st_steps += __shfl_down_sync(0xffffffffu, st_steps, off);
    st_walks += __shfl_down_sync(0xffffffffu, st_walks, off);
    st_capped += __shfl_down_sync(0xffffffffu, st_capped, off);
  }
  if (lane == 0 && L.stats != nullptr) {
    atomicAdd(&L.stats[ST_STEPS], st_steps);
    atomicAdd(&L.stats[ST_WALKS], (unsigned long long)st_walks);
    if (st_capped) atomicAdd(&L.stats[ST_CAPPED], (unsigned long long)st_capped);
  }
  if (priv) {
    __syncthreads();
    const int64_t ares2 = (DIM == 3) ? Pg0.alpha.res[2] : 1, nodes = ares0 * ares1 * ares2;
    for (int64_t i = threadIdx.x; i < nodes; i += blockDim.x) {
      const int64_t j0 = i % ares0, j1 = (i / ares0) % ares1, j2 = i / (ares0 * ares1);
      const R v = gpriv[j0 + ps1 * j1 + ps2 * j2];
      if (v != R(0)) atomicAdd(&L.grad_alpha[i], (double)v);
    }
  }
#undef WOS_ALPHA_SCATTER
}

#if !defined(__CUDACC_RTC__)
// one pass (L.pass 1 or 2) of the adjoint; the caller zeroes the work counter before each
template <int DIM, typename R, bool ALPHA, int PASS>
cudaError_t launch_adjoint_m(const AdjLaunch& L, int num_sms, cudaStream_t stream) {
  size_t smem = (size_t)L.problem_bytes + ((ALPHA && PASS == 2) ? (size_t)L.priv_nodes * sizeof(R) : 0);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(wos_adjoint_kernel<DIM, R, ALPHA, PASS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wos_adjoint_kernel<DIM, R, ALPHA, PASS>,
                                                                kAdjBlock, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int grid = per_sm * num_sms;
  uint64_t blocks_needed = (L.total_items + kAdjBlock - 1) / kAdjBlock;
  if ((uint64_t)grid > blocks_needed) grid = (int)(blocks_needed > 0 ? blocks_needed : 1);
  AdjLaunch arg = L;
  philox_round_keys(arg.seed, arg.rk);
  wos_adjoint_kernel<DIM, R, ALPHA, PASS><<<grid, kAdjBlock, smem, stream>>>(arg);
  return cudaGetLastError();
}

template <int DIM, typename R>
cudaError_t launch_adjoint_t(const AdjLaunch& L, int num_sms, cudaStream_t stream) {
  if (L.pass == 1)
    return L.alpha ? launch_adjoint_m<DIM, R, true, 1>(L, num_sms, stream)
                   : launch_adjoint_m<DIM, R, false, 1>(L, num_sms, stream);
  return L.alpha ? launch_adjoint_m<DIM, R, true, 2>(L, num_sms, stream)
                 : launch_adjoint_m<DIM, R, false, 2>(L, num_sms, stream);
}
#endif  // !__CUDACC_RTC__

}  // namespace wos
