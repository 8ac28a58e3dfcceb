// wos_nf_impl.cuh -- persistent next-flight walk-on-spheres kernel (Sec. 5.2,
// Supplemental Algorithm 2).
//
// A walk takes one distance query per ball.  In the ball B(x) of radius R it
// draws one exit point z on the sphere and unrolls the volume recursion into two
// series over uniform in-ball points x^1, x^2, ...:
//   T_tr  = sum_j P(x^j, z) |dB| prod_{l<j} theta_l,
//   T_src = sum_{j>=1} f'(x^j) G(x^{j-1}, x^j) |B| prod_{l<j-1} theta_l,
//   theta_l = G(x^l, x^{l+1}) |B| (sigma_bar - sigma'(x^{l+1})),
// stopping by Russian roulette with probability min(1, |throughput|).  The walk
// then adds W T_src, multiplies its weight W by T_tr and moves to z.  G and P are
// the approximate off-centred forms of Supplemental 1.2 (NfBall), or (SERIES) its
// series truncated at L.nf_series terms (nf_series_ball / nf_series_eval, with the
// ball's coefficient tables in per-lane local memory); the first term of each ball is
// the centred P.
//
// Lanes run a two-phase state machine.  A lane at the start of a ball runs the
// distance query (phase 0, a divergent branch) and then, in the same iteration,
// joins the inner step that every active lane runs (roulette, one in-ball point,
// coefficients, the two kernels).  As in the delta-tracking kernel, walks are
// items claimed per warp in chunks, lanes regenerate when a walk ends, and FP64
// per-lane partial sums are flushed on a change of point with e^{-gamma(x_0)}.
//
// Randoms: ball k of walk (p, w) draws z from Philox block (p, w, k, 0); inner
// iteration j of that ball draws its roulette uniform and its in-ball point from
// block (p, w, k, j + 1).
#pragma once

#include <cuda_runtime.h>

#include "wos_internal.h"
#include "wos_math.cuh"
#include "wos_problem.cuh"

namespace wos {

constexpr int kNfBlock = 128;
constexpr uint64_t kNfChunk = 128;

template <int DIM, typename R, bool MESH, bool SERIES>
__global__ void __launch_bounds__(kNfBlock, (sizeof(R) == 4) ? 4 : 1) wos_nf_kernel(WalkLaunch L) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  {
    const int4* src = reinterpret_cast<const int4*>(L.problem);
    int4* dst = reinterpret_cast<int4*>(smem_raw);
    for (int i = threadIdx.x; i < L.problem_bytes / 16; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
  }
  const DevProblem<R>& P = *reinterpret_cast<const DevProblem<R>*>(smem_raw);
  int* stk_n = nullptr;
  R* stk_d = nullptr;
  const float* mtop = nullptr;  // the tree's top nodes, staged after the stacks
  if (MESH) {  // this thread's column of the BVH traversal stack, after the problem
    stk_n = reinterpret_cast<int*>(smem_raw + L.problem_bytes) + threadIdx.x;
    stk_d = reinterpret_cast<R*>(smem_raw + L.problem_bytes + sizeof(int) * kMeshStack * kNfBlock) + threadIdx.x;
    float* top = reinterpret_cast<float*>(smem_raw + L.problem_bytes + (sizeof(int) + sizeof(R)) * kMeshStack * kNfBlock);
    const int n4 = 8 * min(P.mesh_top, kMeshTopMax);
    const float4* src = reinterpret_cast<const float4*>(P.mesh_nodes);
    for (int i = threadIdx.x; i < n4; i += blockDim.x) reinterpret_cast<float4*>(top)[i] = __ldg(src + i);
    __syncthreads();
    mtop = top;
  }
  const unsigned kAll = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  const R eps = R(L.eps);
  const R sbar = R(L.sigma_bar);
  const R s_root = w_sqrt(sbar);
  const uint32_t max_k = (L.max_steps >= (int64_t)0xffffffffll) ? 0xffffffffu : (uint32_t)L.max_steps;
  const uint32_t max_j = (L.nf_max_inner >= (int64_t)0xffffffffll) ? 0xffffffffu : (uint32_t)L.nf_max_inner;
  const R cvol = (DIM == 2) ? R(3.14159265358979323846) : R(4.18879020478639098462);   // |B| / R^dim
  const R carea = (DIM == 2) ? R(6.28318530717958647692) : R(12.5663706143591729539);  // |dB| / R^(dim-1)

  const uint64_t total = (L.walk_end != nullptr) ? (uint64_t)__ldg(&L.walk_end[L.npts - 1]) : L.total_items;
  const bool accumulate = (L.sum != nullptr);
  uint64_t chunk_next = 0, chunk_end = 0;
  bool exhausted = false, active = false;

  // walk state
  uint32_t p = 0, w = 0, k = 0, j = 0;
  uint64_t item = 0;
  int phase = 0;          // 0: at a ball centre, needs a distance query; 1: inside the ball's series
  bool capped = false;    // the inner series of some ball hit its cap
  R x[3] = {R(0), R(0), R(0)}, xbp[3] = {R(0), R(0), R(0)};
  R vz[3] = {R(0), R(0), R(0)}, uc[3] = {R(0), R(0), R(0)};
  R W = R(1), acc = R(0), T = R(1), Ttr = R(0), Tsrc = R(0), Rb = R(0);
  NfBall<DIM, R> ball;
  ball.init(R(1), R(1));
  // series tables of the current ball: p_n and rho_n(a) (indices < nser)
  const int nser = SERIES ? L.nf_series : 1;
  R ser_p[SERIES ? kNfSeriesMax : 1], ser_ra[SERIES ? kNfSeriesMax : 1];
  int ser_n0 = 0;  // the ball's start index of the downward sweep

  const uint32_t kNoPoint = 0xffffffffu;
  uint32_t acc_p = kNoPoint;
  double s1 = 0.0, s2 = 0.0;
  uint32_t n_acc = 0;
  unsigned long long st_steps = 0, st_inner = 0;
  uint32_t st_walks = 0, st_capped = 0, st_nonfinite = 0, st_outside = 0;

  for (;;) {
    unsigned need = __ballot_sync(kAll, !active);
    while (need != 0u && !exhausted) {
      if (chunk_next >= chunk_end) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(L.work_counter, (unsigned long long)kNfChunk);
        base = __shfl_sync(kAll, base, 0);
        if (base >= total) {
          exhausted = true;
          break;
        }
        chunk_next = base;
        chunk_end = (base + kNfChunk < total) ? base + kNfChunk : total;
      }
      unsigned nneed = __popc(need);
      uint64_t avail = chunk_end - chunk_next;
      unsigned take = (avail < nneed) ? (unsigned)avail : nneed;
      unsigned rank = __popc(need & lt_mask);
      if (!active && rank < take) {
        item = chunk_next + rank;
        uint64_t pp, jj;
        if (L.walk_end == nullptr) {
          pp = item / (uint64_t)L.walks_uniform;
          jj = item - pp * (uint64_t)L.walks_uniform;
        } else {
          int64_t lo = 0, hi = L.npts - 1;
          while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if ((uint64_t)__ldg(&L.walk_end[mid]) > item) hi = mid; else lo = mid + 1;
          }
          pp = (uint64_t)lo;
          jj = item - ((lo > 0) ? (uint64_t)__ldg(&L.walk_end[lo - 1]) : 0ull);
        }
        p = (uint32_t)pp;
        w = (uint32_t)(L.walk_offset + jj);
        k = 0;
#pragma unroll
        for (int d = 0; d < 3; ++d) x[d] = (d < DIM) ? R(__ldg(&L.pts[(int64_t)d * L.npts + (int64_t)p])) : R(0);
        W = R(1);
        acc = R(0);
        phase = 0;
        capped = false;
        active = true;
      }
      chunk_next += take;
      need = __ballot_sync(kAll, !active);
    }
    if (__ballot_sync(kAll, active) == 0u) break;
    if (!active) continue;

    // A lane whose ball's series stops sets up its next ball in the same iteration: with
    // about one inner iteration per ball, every lane then runs the same sequence in an
    // iteration (the roulette that ends a ball, the next ball's query and set-up, its first
    // inner iteration) instead of half the lanes idling through the others' set-ups.  A new
    // ball's first roulette never stops (T = 1), so two passes suffice.
    U4 r1 = U4{0u, 0u, 0u, 0u};
    R pRR = R(1);
    bool ended = false;
    for (int pass = 0; pass < 2; ++pass) {
      if (phase == 0) {
        // ---- a new ball: distance query, exit point, first boundary term ----
        R xb[3];
        R bound2 = R(INFINITY);
        if (MESH && k > 0) {
          // the previous ball's boundary point bounds the query (NaN when none is known)
          R e0 = x[0] - xbp[0], e1 = x[1] - xbp[1], e2 = x[2] - xbp[2];
          R b2 = e0 * e0 + e1 * e1 + e2 * e2;
          if (b2 < R(INFINITY)) bound2 = b2;
        }
        // meshes: the ball takes the problem's certified radius (any ball inside the domain
        // keeps the series' identities), and the exact distance decides the eps-shell test
        const R tau = MESH ? P.mesh_tau : R(1);
        R d = distance<DIM, R, MESH>(P, x, xb, bound2, stk_n, stk_d, kNfBlock, tau,
                                     (bound2 < R(INFINITY)) ? xbp : nullptr, nullptr, mtop);
        if (MESH && tau < R(1) && !(d >= eps)) {
          R e0 = x[0] - xb[0], e1 = x[1] - xb[1], e2 = x[2] - xb[2];
          R b2 = e0 * e0 + e1 * e1 + e2 * e2;
          R xe[3];
          d = distance<DIM, R, MESH>(P, x, xe, (b2 < R(INFINITY)) ? b2 : R(INFINITY), stk_n, stk_d, kNfBlock, R(1),
                                     nullptr, nullptr, mtop);
  #pragma unroll
          for (int i = 0; i < 3; ++i) xb[i] = xe[i];
        }
        if (MESH) {
  #pragma unroll
          for (int i = 0; i < 3; ++i) xbp[i] = xb[i];
        }
        const bool shell = !(d >= eps);
        if (shell || k >= max_k) {
          if (shell) acc += W * w_exp(gamma_at<DIM>(P, x)) * g_at<DIM>(P, xb);
          else capped = true;
          if (k == 0 && !(d > R(0))) ++st_outside;
          double acc_d = (double)acc;
          if (accumulate && p != acc_p) {
            if (acc_p != kNoPoint) {
              R x0[3];
  #pragma unroll
              for (int dd = 0; dd < 3; ++dd)
                x0[dd] = (dd < DIM) ? R(__ldg(&L.pts[(int64_t)dd * L.npts + (int64_t)acc_p])) : R(0);
              double e0 = exp(-(double)gamma_at<DIM>(P, x0));
              atomicAdd(&L.sum[acc_p], s1 * e0);
              atomicAdd(&L.sumsq[acc_p], s2 * e0 * e0);
              atomicAdd(&L.count[acc_p], (unsigned long long)n_acc);
            }
            acc_p = p;
            s1 = 0.0;
            s2 = 0.0;
            n_acc = 0;
          }
          s1 += acc_d;
          s2 += acc_d * acc_d;
          ++n_acc;
          if (L.uhat != nullptr) {
            R x0[3];
  #pragma unroll
            for (int dd = 0; dd < 3; ++dd) x0[dd] = (dd < DIM) ? R(__ldg(&L.pts[(int64_t)dd * L.npts + (int64_t)p])) : R(0);
            L.uhat[item] = acc_d * exp(-(double)gamma_at<DIM>(P, x0));
            L.steps_out[item] = (int64_t)k;
          }
          st_steps += k;
          ++st_walks;
          if (capped) ++st_capped;
          if (!isfinite(acc_d)) ++st_nonfinite;
          active = false;
          ended = true;
          break;
        }
        Rb = d;
        ball.init(s_root, Rb);
        if (SERIES) {
          nf_series_ball<DIM, R>(s_root * Rb, nser, ser_p, ser_ra);
          ser_n0 = nser + 12 + (int)w_fmin(s_root * Rb, R(4096));
        }
        U4 r0 = philox4x32_10_rk(U4{p, w, k, 0u}, L.rk);
        R dz[3] = {R(0), R(0), R(0)};
        if (DIM == 2) {
          w_sincospi2(to_uniform<R>(r0.x), &dz[1], &dz[0]);
        } else {
          R cz = R(1) - R(2) * to_uniform<R>(r0.x);
          R sz = w_sqrt_fast(w_fmax(R(0), R(1) - cz * cz));
          R sp_, cp_;
          w_sincospi2(to_uniform<R>(r0.y), &sp_, &cp_);
          dz[0] = sz * cp_; dz[1] = sz * sp_; dz[2] = cz;
        }
  #pragma unroll
        for (int i = 0; i < 3; ++i) {
          vz[i] = Rb * dz[i];
          uc[i] = R(0);
        }
        T = R(1);
        Ttr = ball.pcentre;  // P(x, z) |dB| at the centre
        Tsrc = R(0);
        j = 0;
        phase = 1;
      }
      // ---- the roulette of the ball's series ----
      r1 = philox4x32_10_rk(U4{p, w, k, j + 1u}, L.rk);
      pRR = w_fmin(R(1), w_fabs(T));
      bool stop = pRR < to_uniform<R>(r1.x);
      if (!stop && j >= max_j) {
        stop = true;
        capped = true;
      }
      if (stop) {
        acc += W * Tsrc;
        W *= Ttr;
#pragma unroll
        for (int i = 0; i < DIM; ++i) x[i] += vz[i];
        ++k;
        phase = 0;
        continue;  // the next pass sets up the next ball
      }
      break;
    }
    if (ended || phase == 0) continue;

    // ---- one inner iteration of the ball's series ----
    T /= pRR;
    // next in-ball point: a uniform direction w (words z, w) and a distance (word y), uniform
    // in the ball (printed approximations) or from the free-space kernel (series)
    R wd[3] = {R(0), R(0), R(0)};
    if (DIM == 2) {
      w_sincospi2(to_uniform<R>(r1.z), &wd[1], &wd[0]);
    } else {
      R cn = R(1) - R(2) * to_uniform<R>(r1.z);
      R sn = w_sqrt_fast(w_fmax(R(0), R(1) - cn * cn));
      R sp_, cp_;
      w_sincospi2(to_uniform<R>(r1.w), &sp_, &cp_);
      wd[0] = sn * cp_; wd[1] = sn * sp_; wd[2] = cn;
    }
    R vn[3] = {R(0), R(0), R(0)};
    R hm = R(0);  // series: h(k r_m)
    if (SERIES) {
      R uw = R(0), uu = R(0);
#pragma unroll
      for (int i = 0; i < DIM; ++i) {
        uw += uc[i] * wd[i];
        uu += uc[i] * uc[i];
      }
      const R rm = -uw + w_sqrt(w_fmax(R(0), uw * uw + Rb * Rb - uu));
      const R rr = nf_free_radius<DIM, R>(s_root, rm, to_uniform<R>(r1.y));
      hm = nf_free_h<DIM, R>(s_root * rm);
#pragma unroll
      for (int i = 0; i < DIM; ++i) vn[i] = uc[i] + rr * wd[i];
    } else {
      const R rr = (DIM == 2) ? Rb * w_sqrt(to_uniform<R>(r1.y)) : Rb * w_cbrt(to_uniform<R>(r1.y));
#pragma unroll
      for (int i = 0; i < DIM; ++i) vn[i] = rr * wd[i];
    }
    R y[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) y[i] = (i < DIM) ? x[i] + vn[i] : R(0);
    R spy, fpy;
    coeffs<DIM>(P, y, &spy, &fpy);
    R vol = cvol * Rb * Rb * ((DIM == 3) ? Rb : R(1));
    R area = carea * Rb * ((DIM == 3) ? Rb : R(1));
    R Gv, Pyz;  // G(x_c, x_n) / p(x_n) and P(x_n, z)
    if (SERIES) {
      // one downward sweep for both; its start index is the largest of the lanes here,
      // so that the sweep's index (and the tables' local-memory rows) agree across the warp
      const int n0w = __reduce_max_sync(__activemask(), ser_n0);
      R Hxy, Phi;
      nf_series_eval<DIM, R>(s_root, s_root * Rb, Rb, nser, n0w, ser_p, ser_ra, uc, vn, vz, &Hxy, &Phi, &Pyz);
      Gv = (R(1) - Hxy / Phi) * hm / sbar;
    } else {
      Gv = ball.G(uc, vn) * vol;
      Pyz = ball.P(vn, vz);
    }
    Tsrc += fpy * Gv * T;
    T *= Gv * (sbar - spy);
#pragma unroll
    for (int i = 0; i < 3; ++i) uc[i] = vn[i];
    Ttr += Pyz * area * T;                // next term of the boundary series
    ++j;
    ++st_inner;
  }

  if (accumulate && acc_p != kNoPoint) {
    R x0[3];
#pragma unroll
    for (int dd = 0; dd < 3; ++dd) x0[dd] = (dd < DIM) ? R(__ldg(&L.pts[(int64_t)dd * L.npts + (int64_t)acc_p])) : R(0);
    double e0 = exp(-(double)gamma_at<DIM>(P, x0));
    atomicAdd(&L.sum[acc_p], s1 * e0);
    atomicAdd(&L.sumsq[acc_p], s2 * e0 * e0);
    atomicAdd(&L.count[acc_p], (unsigned long long)n_acc);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    st_steps += __shfl_down_sync(kAll, st_steps, off);
    st_inner += __shfl_down_sync(kAll, st_inner, off);
    st_walks += __shfl_down_sync(kAll, st_walks, off);
    st_capped += __shfl_down_sync(kAll, st_capped, off);
    st_nonfinite += __shfl_down_sync(kAll, st_nonfinite, off);
    st_outside += __shfl_down_sync(kAll, st_outside, off);
  }
  if (lane == 0) {
    atomicAdd(&L.stats[ST_STEPS], st_steps);
    atomicAdd(&L.stats[ST_INNER], st_inner);
    atomicAdd(&L.stats[ST_WALKS], (unsigned long long)st_walks);
    if (st_capped) atomicAdd(&L.stats[ST_CAPPED], (unsigned long long)st_capped);
    if (st_nonfinite) atomicAdd(&L.stats[ST_NONFINITE], (unsigned long long)st_nonfinite);
    if (st_outside) atomicAdd(&L.stats[ST_OUTSIDE], (unsigned long long)st_outside);
  }
}

template <int DIM, typename R, bool MESH, bool SERIES>
cudaError_t launch_nf_m(const WalkLaunch& L, int num_sms, cudaStream_t stream) {
  size_t smem = (size_t)L.problem_bytes;
  if (MESH) smem += (sizeof(int) + sizeof(R)) * kMeshStack * kNfBlock + 128 * kMeshTopMax;
  if (smem > 48 * 1024) {
    cudaError_t ea = cudaFuncSetAttribute(wos_nf_kernel<DIM, R, MESH, SERIES>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ea != cudaSuccess) return ea;
  }
  int per_sm = 0;
  cudaError_t e =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wos_nf_kernel<DIM, R, MESH, SERIES>, kNfBlock, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int grid = per_sm * num_sms;
  // total_items is ~0 when per-point walk counts give the total on the device: no cap then
  uint64_t warps_needed = L.total_items / 32 + 1;
  uint64_t blocks_needed = warps_needed / (kNfBlock / 32) + 1;
  if ((uint64_t)grid > blocks_needed) grid = (int)(blocks_needed > 0 ? blocks_needed : 1);
  WalkLaunch arg = L;
  philox_round_keys(arg.seed, arg.rk);
  wos_nf_kernel<DIM, R, MESH, SERIES><<<grid, kNfBlock, smem, stream>>>(arg);
  return cudaGetLastError();
}

template <int DIM, typename R>
cudaError_t launch_nf_t(const WalkLaunch& L, int num_sms, cudaStream_t stream) {
  const bool series = L.nf_series > 0;
  if (DIM == 3 && L.mesh)
    return series ? launch_nf_m<DIM, R, true, true>(L, num_sms, stream)
                  : launch_nf_m<DIM, R, true, false>(L, num_sms, stream);
  return series ? launch_nf_m<DIM, R, false, true>(L, num_sms, stream)
                : launch_nf_m<DIM, R, false, false>(L, num_sms, stream);
}

}  // namespace wos
