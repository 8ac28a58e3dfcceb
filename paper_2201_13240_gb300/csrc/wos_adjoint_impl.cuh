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

#include <cuda_runtime.h>

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
  // Rows (c1, c2) of the support are visited in an order rotated by the lane, so lanes
  // whose points share a cell (walks of one point start together) add to different
  // addresses at the same time instead of serialising on one.
  auto sel4 = [](const R* a, int i) { return i == 0 ? a[0] : (i == 1 ? a[1] : (i == 2 ? a[2] : a[3])); };
  const int nrows = (DIM == 3) ? 16 : 4;
  const int rot = (int)(threadIdx.x & 31);
  for (int k = 0; k < nrows; ++k) {
    const int r = (k + rot) & (nrows - 1);
    const int c1 = r & 3, c2 = (DIM == 3) ? (r >> 2) : 0;
    const int j1 = min(max(ib[1] + c1, 0), F.res[1] - 1);
    const int j2 = (DIM == 3) ? min(max(ib[2] + c2, 0), F.res[2] - 1) : 0;
    const R b1 = sel4(B[1], c1), d1 = sel4(B1[1], c1), e1 = sel4(B2[1], c1);
    const R b2 = (DIM == 3) ? sel4(B[2], c2) : R(1), d2 = (DIM == 3) ? sel4(B1[2], c2) : R(0);
    const R e2 = (DIM == 3) ? sel4(B2[2], c2) : R(0);
    const R b12 = b1 * b2;
    A* row = grad + s1 * j1 + s2 * j2;
#pragma unroll
    for (int c0 = 0; c0 < 4; ++c0) {
      const int j0 = min(max(ib[0] + c0, 0), F.res[0] - 1);
      const R b0 = B[0][c0];
      R val = vN * b0 * b12 + vG[0] * B1[0][c0] * b12 + vG[1] * b0 * d1 * b2 +
              vL * (B2[0][c0] * b12 + b0 * e1 * b2 + b0 * b1 * e2);
      if (DIM == 3) val += vG[2] * b0 * b1 * d2;
      if (val != R(0)) atomicAdd(&row[j0], A(val));
    }
  }
}

// d sigma' / d alpha_m = cN N_m + cG . grad N_m + cL Lap N_m at y
template <int DIM, typename R>
__device__ void alpha_sensitivity(const DevProblem<R>& P, const R* y, R* cN, R* cG, R* cL) {
  // in the walk's precision (FP64 arithmetic is a small fraction of FP32's rate here)
  FieldVal<R> A = field_eval<DIM>(P, P.alpha, y[0], y[1], y[2], true);
  FieldVal<R> Ph = field_eval<DIM>(P, P.phi, y[0], y[1], y[2], true);
  FieldVal<R> S = field_eval<DIM>(P, P.sigma, y[0], y[1], y[2], false);
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
  *cN = -S.v * ia2 - R(0.5) * A.lap * ia2 + na2 * ia2 * ia - gg_ga * ia2;
#pragma unroll
  for (int d = 0; d < 3; ++d) cG[d] = (d < DIM) ? gg[d] * ia - ga[d] * ia2 : R(0);
  *cL = R(0.5) * ia;
}

template <int DIM, typename R, bool ALPHA>
__global__ void __launch_bounds__(kAdjBlock) wos_adjoint_kernel(AdjLaunch L) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  {
    const int4* src = reinterpret_cast<const int4*>(L.problem);
    int4* dst = reinterpret_cast<int4*>(smem_raw);
    for (int i = threadIdx.x; i < L.problem_bytes / 16; i += blockDim.x) dst[i] = src[i];
  }
  // alpha: per-CTA accumulators in the walk's precision (FP32 shared atomics are native)
  R* gpriv = reinterpret_cast<R*>(smem_raw + L.problem_bytes);
  const bool priv = ALPHA && L.priv_nodes > 0;
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
  const uint32_t key0 = (uint32_t)(L.seed & 0xffffffffull), key1 = (uint32_t)(L.seed >> 32);
  const R eps = R(L.eps), s_root = w_sqrt(R(L.sigma_bar));
  const R inv_sb = R(1) / R(L.sigma_bar);
  const uint32_t max_k = (L.max_steps >= (int64_t)0xffffffffll) ? 0xffffffffu : (uint32_t)L.max_steps;
  const double inv_walks = 1.0 / (double)L.walks_uniform;

  uint64_t chunk_next = 0, chunk_end = 0;
  const uint64_t magic = (L.walks_uniform > 0) ? ~0ull / (uint64_t)L.walks_uniform : 0ull;
  bool exhausted = false, active = false;
  // walk state; phase 0 computes the total A, phase 1 replays and scatters
  R x[3] = {R(0), R(0), R(0)}, W = R(1), acc = R(0), total = R(0);
  R xbp[3] = {R(0), R(0), R(0)};  // previous closest boundary point (bounds the next mesh query)
  uint32_t p = 0, w = 0, k = 0, phase = 0;
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
        const uint64_t item = chunk_next + rank, dw = (uint64_t)L.walks_uniform;
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
        phase = 0;
        // e^{-gamma(x_0)} in the walk's precision (an FP64 exp per walk start, run by the one
        // or two lanes that start, occupied the narrow FP64 pipe)
        coef = R(__ldg(&L.grad_u[p]) * inv_walks) * w_exp(-gamma_at<DIM>(P, x));
        active = true;
      }
      chunk_next += take;
      need = __ballot_sync(0xffffffffu, !active);
    }
    if (__ballot_sync(0xffffffffu, active) == 0u) break;
    if (!active) continue;

    R xb[3];
    R bound2 = R(INFINITY);
    if (P.domain_kind == D_MESH && k > 0) {
      R e0 = x[0] - xbp[0], e1 = x[1] - xbp[1], e2 = x[2] - xbp[2];
      bound2 = e0 * e0 + e1 * e1 + e2 * e2;
    }
    R d = distance<DIM>(P, x, xb, bound2);
#pragma unroll
    for (int i = 0; i < 3; ++i) xbp[i] = xb[i];
    const bool ends = !(d >= eps) || k >= max_k;
    const R dd = w_fmax(d, R(0));
    U4 r0 = philox4x32_10(U4{p, w, k, 0u}, key0, key1);
    R mu = to_uniform<R>(r0.x), ur = to_uniform<R>(r0.y);
    R dy[3] = {R(0), R(0), R(0)}, dz[3] = {R(0), R(0), R(0)};
    if (DIM == 2) {
      w_sincospi2(to_uniform<R>(r0.z), &dy[1], &dy[0]);
      w_sincospi2(to_uniform<R>(r0.w), &dz[1], &dz[0]);
    } else {
      U4 r1 = philox4x32_10(U4{p, w, k, 1u}, key0, key1);
      R cy = R(1) - R(2) * to_uniform<R>(r0.z);
      R sy = w_sqrt(w_fmax(R(0), R(1) - cy * cy));
      R sp_, cp_;
      w_sincospi2(to_uniform<R>(r0.w), &sp_, &cp_);
      dy[0] = sy * cp_; dy[1] = sy * sp_; dy[2] = cy;
      R cz = R(1) - R(2) * to_uniform<R>(r1.x);
      R sz = w_sqrt(w_fmax(R(0), R(1) - cz * cz));
      w_sincospi2(to_uniform<R>(r1.y), &sp_, &cp_);
      dz[0] = sz * cp_; dz[1] = sz * sp_; dz[2] = cz;
    }
    R a = s_root * dd;
    R q = green_q<DIM, R>(a);
    R Gn = dd * dd * q, PB = a * a * q;
    R r = sample_radius<DIM, R>(a, ur, nullptr, (sizeof(R) == 4) ? L.radial_tab : nullptr) * dd;
    R y[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) y[i] = (i < DIM) ? (ends ? x[i] : x[i] + r * dy[i]) : R(0);
    R spy, fpy, gam, al;
    coeffs<DIM>(P, y, &spy, &fpy, &gam, &al);

    if (ends) {
      bool capped = (d >= eps);
      R bterm = R(0);
      if (!capped) {
        bterm = W * w_exp(gam) * g_at<DIM>(P, xb);
        acc += bterm;
      }
      if (ALPHA && phase == 1 && !capped) {
        // boundary factor e^{gamma(x_n)}: d/d alpha_m = N_m(x_n) / (2 alpha(x_n)) times the term
        const R vG[3] = {R(0), R(0), R(0)};
        R v = coef * bterm * R(0.5) / al;
        if (isfinite(v) && v != R(0)) WOS_ALPHA_SCATTER(y, v, vG, R(0));
      }
      if (phase == 0) {
        total = acc;
#pragma unroll
        for (int dd2 = 0; dd2 < 3; ++dd2) x[dd2] = (dd2 < DIM) ? R(__ldg(&L.pts[(int64_t)dd2 * L.npts + (int64_t)p])) : R(0);
        if (ALPHA) {
          // e^{-gamma(x_0)}: -A N_m(x_0) / (2 alpha(x_0))
          const R vG[3] = {R(0), R(0), R(0)};
          R a0 = field_eval<DIM>(P, P.alpha, x[0], x[1], x[2], false).v;
          R v = -coef * total * R(0.5) / a0;
          if (isfinite(v) && v != R(0)) WOS_ALPHA_SCATTER(x, v, vG, R(0));
        }
        W = R(1);
        acc = R(0);
        k = 0;
        phase = 1;
      } else {
        ++st_walks;
        if (capped) ++st_capped;
        active = false;
      }
      continue;
    }
    const R src = W * Gn * fpy;
    acc += src;
    if (ALPHA && phase == 1) {
      // source f'(y): d/d alpha_m = -N_m(y) / (2 alpha(y)) times the term; null weight: see above
      R vN = -coef * src * R(0.5) / al, vG[3] = {R(0), R(0), R(0)}, vL = R(0);
      if (mu <= PB) {
        R wj = R(1) - spy * inv_sb;
        R rem = (total - acc) / wj;
        R rj = -coef * rem * inv_sb;
        R cN, cG[3], cL;
        alpha_sensitivity<DIM, R>(P, y, &cN, cG, &cL);
        if (isfinite(rj)) {
          vN += rj * cN;
#pragma unroll
          for (int i = 0; i < 3; ++i) vG[i] = rj * cG[i];
          vL = rj * cL;
        }
      }
      if (isfinite(vN)) WOS_ALPHA_SCATTER(y, vN, vG, vL);
    }
    if (mu <= PB) {
      R wj = R(1) - spy * inv_sb;
      if (!ALPHA && phase == 1) {
        // d total / d w_j = (A - P_{j+1}) / w_j ; d w_j / d sigma_m = -N_m(y) / (alpha(y) sigma_bar)
        R rem = (total - acc) / wj;
        R val = -coef * rem * inv_sb / al;
        if (isfinite(val) && val != R(0)) grid_scatter<DIM, R>(P.sigma, y, val, L.grad_sigma);
      }
      W *= wj;
#pragma unroll
      for (int i = 0; i < DIM; ++i) x[i] = y[i];
    } else {
#pragma unroll
      for (int i = 0; i < DIM; ++i) x[i] = x[i] + dd * dz[i];
    }
    if (phase == 1) ++st_steps;
    ++k;
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

template <int DIM, typename R, bool ALPHA>
cudaError_t launch_adjoint_m(const AdjLaunch& L, int num_sms, cudaStream_t stream) {
  size_t smem = (size_t)L.problem_bytes + (ALPHA ? (size_t)L.priv_nodes * sizeof(R) : 0);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(wos_adjoint_kernel<DIM, R, ALPHA>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wos_adjoint_kernel<DIM, R, ALPHA>, kAdjBlock,
                                                                smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int grid = per_sm * num_sms;
  uint64_t blocks_needed = (L.total_items + kAdjBlock - 1) / kAdjBlock;
  if ((uint64_t)grid > blocks_needed) grid = (int)(blocks_needed > 0 ? blocks_needed : 1);
  wos_adjoint_kernel<DIM, R, ALPHA><<<grid, kAdjBlock, smem, stream>>>(L);
  return cudaGetLastError();
}

template <int DIM, typename R>
cudaError_t launch_adjoint_t(const AdjLaunch& L, int num_sms, cudaStream_t stream) {
  return L.alpha ? launch_adjoint_m<DIM, R, true>(L, num_sms, stream) : launch_adjoint_m<DIM, R, false>(L, num_sms, stream);
}

}  // namespace wos
