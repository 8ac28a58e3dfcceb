// wos_walk_impl.cuh -- persistent delta-tracking walk-on-spheres kernel.
//
// One lane runs one walk of Supplemental Algorithm 1 (Sec. 5.1, eq. 11),
// unrolled into a loop over steps: distance query, epsilon-shell test, a
// Philox block keyed by (point, walk, step), the centred Green's-function
// sample y, the source term W |G| f'(y), and either a null event at y (weight
// 1 - sigma'(y)/sigma_bar) or a jump to the sphere.  The sqrt(alpha) ratios of
// Alg. 1 telescope into e^{gamma(x_n) - gamma(x_0)}, applied once per walk.
//
// Scheduling: the grid is persistent (resident blocks x SMs).  Walks are items
// of a point-major index space claimed in chunks by one atomic per warp; a lane
// whose walk ends takes the next item at the top of the step loop, so warps
// stay full while walk lengths vary.  Each lane keeps partial sums of its current
// point, shifted by the first estimate it saw for that point (sums of u - c and
// (u - c)^2 in the walk's precision: no FP64 arithmetic per walk, and no
// cancellation when the estimates agree), and flushes them to the FP64
// accumulators with atomics when its point changes.
//
// SIMT uniformity: in almost every iteration some lane of a warp ends its walk,
// so the end of a walk must not run a separate instruction stream.  A lane that
// ends still draws its randoms and samples its ball (and discards them), and it
// evaluates the coefficients at its own point x_n instead of at y, which gives
// gamma(x_n) for the boundary term from the same call; only g(xbar) is extra.
// Starting a walk only loads its point: the factor e^{-gamma(x_0)}, common to
// all walks of a point, multiplies the partial sums when they are flushed.
#pragma once

#if !defined(__CUDACC_RTC__)
#include <cuda_runtime.h>
#endif

#include "wos_internal.h"
#include "wos_math.cuh"
#include "wos_problem.cuh"

namespace wos {

constexpr int kWalkBlock = 128;
constexpr unsigned kFull = 0xffffffffu;
// Walks a warp claims at a time: total / (warps x kChunksPerWarp), a multiple of 32,
// within [kChunkMin, kChunkMax].  Items are point-major, so a lane keeps one point (and
// its partial sums) for about chunk/32 walks: with 128-walk chunks a lane changed point
// every ~4 walks and the flushes (FP64 arithmetic and atomics, run by one or two lanes
// of the warp) took a third of the FP64 pipe.  The cap keeps the tail balanced.
constexpr uint64_t kChunkMin = 128, kChunkMax = 2048, kChunksPerWarp = 64;

template <int DIM, typename R>
struct WalkState {
  R x[3];
  R xbp[3];  // closest boundary point of the previous step (bounds the next mesh query)
  R W, acc;
  uint32_t p, w, k;
  uint32_t prob;  // batched launches: the walk's problem
  uint64_t item;
  // weight window: current branch id, next id, branch ended by roulette, steps of the walk
  uint32_t bid, next_bid, steps_walk;
  bool dead;
  // spatial gradient: grad U of the walk = acc * gb + gc, set on the first step
  R gb[3], gc[3];
};

constexpr int kWWDepth = 8;  // most split copies a lane keeps waiting
#if !defined(WOS_WALK_DEFER_LANES)
#define WOS_WALK_DEFER_LANES 4
#endif
constexpr int kDeferLanes = WOS_WALK_DEFER_LANES;  // ended walks a warp gathers before finishing them
static_assert(kDeferLanes >= 1 && kDeferLanes <= 32, "kDeferLanes must be 1..32");

// e^{-gamma(x_0)} of point p (applied once per flush), in the walk's precision: the
// FP32 walk's gamma carries FP32 rounding already, and an FP64 exp costs dozens of
// instructions on the narrow FP64 pipe
template <int DIM, typename R>
__device__ __forceinline__ double point_factor(const WalkLaunch& L, const DevProblem<R>& P, uint32_t p) {
  R x0[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) x0[d] = (d < DIM) ? R(__ldg(&L.pts[(int64_t)d * L.npts + (int64_t)p])) : R(0);
  return (double)w_exp(-gamma_at<DIM>(P, x0));
}

template <int DIM, typename R, bool BATCHED>
__device__ __forceinline__ void start_walk(const WalkLaunch& L, uint64_t item, uint64_t magic,
                                           WalkState<DIM, R>& s) {
  uint64_t p, j;
  if (L.walk_end == nullptr) {
    // item / walks_uniform by a multiply-high with magic = floor((2^64 - 1) / walks_uniform):
    // the product's high word is the quotient or one less, and one correction makes it exact
    const uint64_t d = (uint64_t)L.walks_uniform;
    p = __umul64hi(item, magic);
    j = item - p * d;
    if (j >= d) {
      ++p;
      j -= d;
    }
  } else {
    // first point whose inclusive walk prefix exceeds item
    int64_t lo = 0, hi = L.npts - 1;
    while (lo < hi) {
      int64_t mid = (lo + hi) >> 1;
      if ((uint64_t)__ldg(&L.walk_end[mid]) > item) hi = mid; else lo = mid + 1;
    }
    p = (uint64_t)lo;
    uint64_t begin = (lo > 0) ? (uint64_t)__ldg(&L.walk_end[lo - 1]) : 0ull;
    j = item - begin;
  }
  s.item = item;
  s.p = (uint32_t)p;
  s.prob = 0;
  if (BATCHED) {
    // the problem whose point range holds p: last offset <= p
    int lo = 0, hi = L.nprob - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if ((uint64_t)__ldg(&L.prob_offsets[mid]) <= p) lo = mid; else hi = mid - 1;
    }
    s.prob = (uint32_t)lo;
  }
  s.w = (uint32_t)(L.walk_offset + j);
  s.k = 0;
#pragma unroll
  for (int d = 0; d < 3; ++d) s.x[d] = (d < DIM) ? R(__ldg(&L.pts[(int64_t)d * L.npts + (int64_t)p])) : R(0);
  s.W = R(1);
  s.acc = R(0);
  s.bid = 0;
  s.next_bid = 1;
  s.steps_walk = 0;
  s.dead = false;
}

// FP32: at most 96 registers, so five 128-thread blocks (20 warps) fit an SM.  Left
// alone the compiler takes 168 (12 warps).  Measured on the 3D workload: 128 registers
// (16 warps) 22% faster than 168, 96 registers another 3.5% -- the extra warps hide the
// step's dependency chains better than the spilled bytes cost.
// MESH: the domain is a triangle mesh; the walk then keeps its previous closest
// point to bound the next BVH search (analytic domains carry none of this).
// BATCHED: the launch walks many problems (each walk's problem description is
// read from global memory through L1 instead of being staged in shared memory).
// WW: the Sec. 6 weight window (Russian roulette below ww_lo, expected-value
// splitting above ww_hi); split copies wait on a per-lane stack and run after the
// branch that made them, so a walk's estimate stays in one lane.
// GRAD: also estimate grad u at the walk's start (Supplemental Sec. 2).  The first
// ball weights its source sample by grad G / G at y_0 and the rest of the walk by
// grad G / G (null event) or grad P / P at z_0 (boundary step): with S_0 the first
// source term and A the walk's total, grad U = S_0 gG + (A - S_0) gB = A gB + gc.
// Then grad u = e^{-gamma(x_0)} (grad U - U grad gamma(x_0)); e^{-gamma(x_0)} joins
// the flush like the value's, grad gamma(x_0) is cached per lane and point.  The
// extra FP64 partial sums take registers: this variant runs 20 warps per SM (96 registers,
// a few spilled bytes; measured 6% faster than 16 warps with 112 registers).
// DRIFT: the problem has an extra drift omega (not alpha times a gradient): coeffs adds
// b . grad gamma + div b to sigma', and a null event also carries
// |G'(r)/G(r)| (dir_y . b(y)) / sigma_bar (the drift term moved onto G by parts).
// Compiled at run time for one problem (WOS_JIT_FIELDS) the kernel is named
// wos_walk_spec_kernel, so that profiles tell the two apart.  WOS_WALK_MIN_BLOCKS is the
// FP32 value kernel's resident-block target (the register cap): the generated source of a
// 3D problem asks for six (80 registers, no spills; five measured 7% slower than seven,
// seven 0.6% slower than six).
#if !defined(WOS_WALK_MIN_BLOCKS)
#define WOS_WALK_MIN_BLOCKS 5
#endif
#if defined(WOS_JIT_FIELDS)
#define WOS_WALK_KERNEL wos_walk_spec_kernel
#else
#define WOS_WALK_KERNEL wos_walk_kernel
#endif
// MINB > 0 overrides the resident-block target (the batched launches' high-occupancy
// variant, chosen by the schedule).
template <int DIM, typename R, bool MESH, bool BATCHED, bool WW, bool GRAD, bool DRIFT = false, int MINB = 0>
__global__ void __launch_bounds__(kWalkBlock,
                                  (sizeof(R) == 4) ? (GRAD ? 5 : (MESH ? 5 : (MINB > 0 ? MINB : WOS_WALK_MIN_BLOCKS))) : 1)
    WOS_WALK_KERNEL(WalkLaunch L) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // stage the problem description (a few KB, read by every lane every step) in shared memory
  if (!BATCHED) {
    const int4* src = reinterpret_cast<const int4*>(L.problem);
    int4* dst = reinterpret_cast<int4*>(smem_raw);
    for (int i = threadIdx.x; i < L.problem_bytes / 16; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
  }
  const DevProblem<R>* Pshared = reinterpret_cast<const DevProblem<R>*>(smem_raw);
  const DevProblem<R>* Pall = reinterpret_cast<const DevProblem<R>*>(L.probs);
  // MESH: this thread's column of the BVH traversal stack, after the problem
  int* stk_n = nullptr;
  R* stk_d = nullptr;
  // and the tree's top nodes (every query starts at the root), staged after the stacks
  const float* mtop = nullptr;
  if (MESH) {
    stk_n = reinterpret_cast<int*>(smem_raw + L.problem_bytes) + threadIdx.x;
    stk_d = reinterpret_cast<R*>(smem_raw + L.problem_bytes + sizeof(int) * kMeshStack * kWalkBlock) + threadIdx.x;
    float* top = reinterpret_cast<float*>(smem_raw + L.problem_bytes + (sizeof(int) + sizeof(R)) * kMeshStack * kWalkBlock);
    const int n4 = 8 * min(Pshared->mesh_top, kMeshTopMax);  // 8 x 16 bytes per node
    const float4* src = reinterpret_cast<const float4*>(Pshared->mesh_nodes);
    for (int i = threadIdx.x; i < n4; i += blockDim.x) reinterpret_cast<float4*>(top)[i] = __ldg(src + i);
    __syncthreads();
    mtop = top;
  }

  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  const R eps = R(L.eps);
  const R s_root0 = w_sqrt(R(L.sigma_bar)), inv_sb0 = R(1) / R(L.sigma_bar);
  const uint32_t max_k = (L.max_steps >= (int64_t)0xffffffffll) ? 0xffffffffu : (uint32_t)L.max_steps;

  // with per-point walk counts the total is the last inclusive prefix sum
  const uint64_t total = (L.walk_end != nullptr) ? (uint64_t)__ldg(&L.walk_end[L.npts - 1]) : L.total_items;
  const bool accumulate = (L.sum != nullptr);
  uint64_t chunk = total / ((uint64_t)gridDim.x * (kWalkBlock / 32) * kChunksPerWarp);
  chunk = (chunk < kChunkMin) ? kChunkMin : (chunk > kChunkMax ? kChunkMax : chunk & ~31ull);
  if (L.chunk != 0u) chunk = L.chunk;  // a schedule's choice (a multiple of 32, checked by the host)
  uint64_t chunk_next = 0, chunk_end = 0;
  const uint64_t magic = (L.walks_uniform > 0) ? ~0ull / (uint64_t)L.walks_uniform : 0ull;
  bool exhausted = false;
  bool active = false;
  WalkState<DIM, R> s;
  s.p = 0;

  // per-lane partial sums of the current point (points are < 2^32 per launch)
  const uint32_t kNoPoint = 0xffffffffu;
  uint32_t acc_p = kNoPoint, acc_prob = 0;
  double s1 = 0.0, s2 = 0.0;
  uint32_t n_acc = 0;
  R sh = R(0), d1 = R(0), d2 = R(0);  // FP32 partial sums shifted by the point's first value
  // spatial gradient: per-lane partial sums of (grad U - U grad gamma) and grad gamma(x_0)
  double gs1[3] = {0.0, 0.0, 0.0}, gs2[3] = {0.0, 0.0, 0.0};
  R ggam[3] = {R(0), R(0), R(0)};
  uint32_t gg_p = kNoPoint;
  // per-lane statistics: a lane finishes far fewer than 2^32 walks in one launch
  unsigned long long st_steps = 0;
  uint32_t st_walks = 0, st_capped = 0, st_nonfinite = 0, st_outside = 0;
  MeshVisits mvis = {0ull, 0ull, 0u};  // mesh queries: nodes, triangles, exhausted searches
  // weight window: copies waiting to run (position, weight, step, branch id)
  R stk_x[WW ? kWWDepth : 1][3], stk_W[WW ? kWWDepth : 1];
  uint32_t stk_k[WW ? kWWDepth : 1], stk_id[WW ? kWWDepth : 1];
  int sp = 0;
  const int ww_depth = WW ? (L.ww_depth < kWWDepth ? L.ww_depth : kWWDepth) : 0;
  const R ww_lo = R(L.ww_lo), ww_hi = R(L.ww_hi);

  // a walk's end once g is added: the spatial gradient, the per-point partial sums (flushed
  // when the lane moves to another point), the per-walk outputs and the statistics
  auto finish_walk = [&](const DevProblem<R>& Pw, bool capped) {
    // no FP64 arithmetic here unless a branch needs it: this block runs whenever a lane ends
    R gv[3] = {R(0), R(0), R(0)};
    if (GRAD) {
      if (s.p != gg_p) {
        gg_p = s.p;
        R x0[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) x0[d] = (d < DIM) ? R(__ldg(&L.pts[(int64_t)d * L.npts + (int64_t)s.p])) : R(0);
        grad_gamma_at<DIM>(Pw, x0, ggam);
      }
      // a walk that ends on its first step (start in the eps-shell) has no first ball
#pragma unroll
      for (int i = 0; i < DIM; ++i) gv[i] = (s.k == 0) ? R(NAN) : s.acc * (s.gb[i] - ggam[i]) + s.gc[i];
    }
    if (accumulate && s.p != acc_p) {
      if (acc_p != kNoPoint) {
        double e0 = point_factor<DIM, R>(L, BATCHED ? Pall[acc_prob] : *Pshared, acc_p);
        if (!GRAD) {
          double c = (double)sh, n = (double)n_acc;
          s1 = n * c + (double)d1;
          s2 = n * c * c + 2.0 * c * (double)d1 + (double)d2;
        }
        atomicAdd(&L.sum[acc_p], s1 * e0);
        atomicAdd(&L.sumsq[acc_p], s2 * e0 * e0);
        atomicAdd(&L.count[acc_p], (unsigned long long)n_acc);
        if (GRAD) {
#pragma unroll
          for (int i = 0; i < DIM; ++i) {
            atomicAdd(&L.gsum[(int64_t)i * L.npts + acc_p], gs1[i] * e0);
            atomicAdd(&L.gsumsq[(int64_t)i * L.npts + acc_p], gs2[i] * e0 * e0);
            gs1[i] = 0.0;
            gs2[i] = 0.0;
          }
        }
      }
      acc_p = s.p;
      acc_prob = s.prob;
      s1 = 0.0;
      s2 = 0.0;
      n_acc = 0;
      sh = s.acc;
      d1 = R(0);
      d2 = R(0);
    }
    if (GRAD) {
      const double acc_d = (double)s.acc;
      s1 += acc_d;
      s2 += acc_d * acc_d;
    } else {
      R dv = s.acc - sh;
      d1 += dv;
      d2 += dv * dv;
    }
    ++n_acc;
    if (GRAD) {
#pragma unroll
      for (int i = 0; i < DIM; ++i) {
        gs1[i] += (double)gv[i];
        gs2[i] += (double)gv[i] * (double)gv[i];
      }
    }
    if (L.uhat != nullptr) {
      double e0 = point_factor<DIM, R>(L, Pw, s.p);
      L.uhat[s.item] = (double)s.acc * e0;
      L.steps_out[s.item] = WW ? (int64_t)s.steps_walk : (int64_t)s.k;
      if (GRAD && L.ghat != nullptr) {
#pragma unroll
        for (int i = 0; i < DIM; ++i) L.ghat[(uint64_t)i * L.total_items + s.item] = (double)gv[i] * e0;
      }
    }
    if (!WW) st_steps += s.k;
    ++st_walks;
    if (capped) ++st_capped;
    if (!isfinite(s.acc)) ++st_nonfinite;
    active = false;
  };
  // Plain, drift and batched walks: a lane whose walk ended waits (with its closest point,
  // gamma and capped flag) until kDeferLanes lanes of the warp have ended, or the work is
  // exhausted; they then add g, finish their walks and claim new ones together.  The two
  // divergent blocks (end and regeneration, run by one or two lanes) then run about once per
  // kDeferLanes walk ends instead of in most iterations, while the waiting lanes sit out a
  // few steps.
  constexpr bool DEFER = !WW && !GRAD && !MESH;
  bool pend = false, pcap = false;
  R pgam = R(0), pxb[3] = {R(0), R(0), R(0)};

  for (;;) {
    // ---- regeneration: lanes without a walk claim the next items ----
    unsigned need = __ballot_sync(kFull, !active);
    if (!DEFER || exhausted || __popc(need) >= kDeferLanes) {
      if (DEFER && pend) {
        const DevProblem<R>& Pe = BATCHED ? Pall[s.prob] : *Pshared;
        if (!pcap) s.acc += s.W * w_exp(pgam) * g_at<DIM>(Pe, pxb);   // Alg. 1: g at the closest point
        finish_walk(Pe, pcap);
        pend = false;
      }
      while (need != 0u && !exhausted) {
        if (chunk_next >= chunk_end) {
          unsigned long long base = 0;
          if (lane == 0) base = atomicAdd(L.work_counter, (unsigned long long)chunk);
          base = __shfl_sync(kFull, base, 0);
          if (base >= total) {
            exhausted = true;
            break;
          }
          chunk_next = base;
          chunk_end = (base + chunk < total) ? base + chunk : total;
        }
        unsigned nneed = __popc(need);
        uint64_t avail = chunk_end - chunk_next;
        unsigned take = (avail < nneed) ? (unsigned)avail : nneed;
        unsigned rank = __popc(need & lt_mask);
        if (!active && rank < take) {
          start_walk<DIM, R, BATCHED>(L, chunk_next + rank, magic, s);
          active = true;
        }
        chunk_next += take;
        need = __ballot_sync(kFull, !active);
      }
    }
    if (__ballot_sync(kFull, active) == 0u) break;
    if (!active) continue;
    const DevProblem<R>& P = BATCHED ? Pall[s.prob] : *Pshared;
    R s_root = s_root0, inv_sb = inv_sb0;
    if (BATCHED) {
      double sbp = __ldg(&L.sigma_bars[s.prob]);
      s_root = w_sqrt(R(sbp));
      inv_sb = R(1) / R(sbp);
    }

    // ---- one step of the walk ----
    R xb[3];
    R d;
    if (MESH) {
      // the previous step's boundary point bounds the query (NaN when none is known)
      R bound2 = R(INFINITY);
      if (s.k > 0) {
        R e0 = s.x[0] - s.xbp[0], e1 = s.x[1] - s.xbp[1], e2 = s.x[2] - s.xbp[2];
        R b2 = e0 * e0 + e1 * e1 + e2 * e2;
        if (b2 < R(INFINITY)) bound2 = b2;
      }
      const R tau = P.mesh_tau;
      d = distance<DIM, R, MESH>(P, s.x, xb, bound2, stk_n, stk_d, kWalkBlock, tau,
                                 (bound2 < R(INFINITY)) ? s.xbp : nullptr, &mvis, mtop);
      if (tau < R(1) && !(d >= eps)) {
        // a certified radius below eps: the exact distance decides the eps-shell test and
        // gives the closest point for g (a step or two per walk, near the boundary)
        R e0 = s.x[0] - xb[0], e1 = s.x[1] - xb[1], e2 = s.x[2] - xb[2];
        R b2 = e0 * e0 + e1 * e1 + e2 * e2;
        R xe[3];
        d = distance<DIM, R, MESH>(P, s.x, xe, (b2 < R(INFINITY)) ? b2 : R(INFINITY), stk_n, stk_d, kWalkBlock,
                                   R(1), nullptr, &mvis, mtop);
#pragma unroll
        for (int i = 0; i < 3; ++i) xb[i] = xe[i];
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) s.xbp[i] = xb[i];
    } else {
      d = distance<DIM, R, MESH>(P, s.x, xb);
    }
    // eps-shell (or outside, or NaN), the step cap, or (weight window) a branch lost at roulette
    const bool ends = !(d >= eps) || s.k >= max_k || (WW && s.dead);
    const R dd = w_fmax(d, R(0));
    const uint32_t blk0 = WW ? (s.bid << 2) : 0u;  // branch b of a split walk: block word (b << 2) | block

    U4 r0 = philox4x32_10_rk(U4{s.p, s.w, s.k, blk0}, L.rk);
    R mu, ur;
    R dy[3] = {R(0), R(0), R(0)}, dz[3] = {R(0), R(0), R(0)};
    if (DIM == 2) {
      mu = to_uniform<R>(r0.x);
      ur = to_uniform<R>(r0.y);
      w_sincospi2(to_uniform<R>(r0.z), &dy[1], &dy[0]);
      w_sincospi2(to_uniform<R>(r0.w), &dz[1], &dz[0]);
    } else {
      // six 21-bit uniforms of the one block: mu, ur, the two directions
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
    // DRIFT: the ball's own bound max(sigma_bar, 10 B / d) with B the problem's drift bound
    // (any positive bound per ball keeps the ball's identity; this one keeps the drift
    // weight of small balls near the boundary bounded)
    if (DRIFT && P.drift_bound > R(0)) {
      const R sb_ball = (R(10) * P.drift_bound) / dd;
      if (sb_ball > R(L.sigma_bar)) {
        s_root = w_sqrt(sb_ball);
        inv_sb = R(1) / sb_ball;
      }
    }
    R a = s_root * dd;
    R q = green_q<DIM, R>(a);
    R Gn = dd * dd * q;        // |G| on the ball of radius d
    R PB = a * a * q;          // sigma_bar |G|, probability of the volume term
    // DRIFT (every ball, G/|G| weight 0.97: the weight ratios multiply along the walk) and
    // GRAD (the first ball only, weight 1/2) draw the mixture sample whose weight mixw
    // bounds the |G'/G| and grad G / G factors; the others draw from G/|G|
    // (one radius solve for every lane, its argument chosen per lane: a mixture lane whose
    // uniform falls in the uniform-radius part solves a dummy and discards it)
    R mixw = R(1);
    const float* tab = (sizeof(R) == 4) ? L.radial_tab : nullptr;
    const bool mix = DRIFT || (GRAD && s.k == 0);
    const R lam = DRIFT ? R(0.97) : R(0.5);
    R rho = sample_radius<DIM, R>(a, mix ? ((ur < lam) ? ur / lam : R(0.5)) : ur, nullptr, tab);
    if (mix) rho = mix_radius_weight<DIM, R>(a, ur, rho, lam, &mixw);
    R r = rho * dd;
    // coefficient point: y for a step; the walk's own point when it ends (gamma(x_n))
    R y[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) y[i] = (i < DIM) ? (ends ? s.x[i] : s.x[i] + r * dy[i]) : R(0);
    R spy, fpy, gam;
    R bvec[3] = {R(0), R(0), R(0)};
    coeffs<DIM, R, DRIFT>(P, y, &spy, &fpy, &gam, nullptr, DRIFT ? bvec : nullptr);

    if (ends) {
      const bool lost = WW && s.dead;
      bool capped = (d >= eps) && !lost;
      if (s.k == 0 && !(d > R(0))) ++st_outside;
      if (DEFER) {
        // the walk's end (g and the accumulation) waits for the loop's head
        pend = true;
        pcap = capped;
        pgam = gam;
#pragma unroll
        for (int i = 0; i < 3; ++i) pxb[i] = xb[i];
        active = false;
        continue;
      }
      if (!capped && !lost) s.acc += s.W * w_exp(gam) * g_at<DIM>(P, xb);   // Alg. 1: g at the closest point
      if (WW) {
        if (capped) ++st_capped;
        if (sp > 0) {  // the walk goes on with its last split copy
          --sp;
#pragma unroll
          for (int i = 0; i < 3; ++i) s.x[i] = stk_x[sp][i];
          s.W = stk_W[sp];
          s.k = stk_k[sp];
          s.bid = stk_id[sp];
          s.dead = false;
          continue;
        }
        capped = false;  // already counted per branch
      }
      finish_walk(P, capped);
      continue;
    }

    s.acc += s.W * Gn * fpy * mixw;   // source term, every step
    if (GRAD && s.k == 0) {    // first ball: gradient weights (W = 1 here)
      R gGR, gPR;
      grad_ratios<DIM, R>(a, rho, &gGR, &gPR);
      const R inv_d = R(1) / dd, S0 = Gn * fpy * mixw;
      const bool nul = mu <= PB;
#pragma unroll
      for (int i = 0; i < DIM; ++i) {
        R vg = gGR * inv_d * dy[i];
        R vb = nul ? vg : gPR * inv_d * dz[i];
        s.gb[i] = vb;
        s.gc[i] = S0 * (vg - vb);
      }
    }
    if (WW) {
      ++st_steps;
      ++s.steps_walk;
    }
    if (mu <= PB) {            // volume term: null event at y
      R wn = R(1) - spy * inv_sb;
      if (DRIFT) {
        R db = R(0);
#pragma unroll
        for (int i = 0; i < DIM; ++i) db += dy[i] * bvec[i];
        wn += green_dlog_r<DIM, R>(a, rho) / dd * db * inv_sb;
      }
      s.W *= wn * mixw;
#pragma unroll
      for (int i = 0; i < DIM; ++i) s.x[i] = y[i];
      if (WW) {
        R aw = w_fabs(s.W);
        if (aw < ww_lo || aw > ww_hi) {
          // the window's own uniform: block 1, word 0 (2D) or word 2 (3D)
          const U4 r1 = philox4x32_10_rk(U4{s.p, s.w, s.k, blk0 | 1u}, L.rk);
          R uww = to_uniform<R>((DIM == 3) ? r1.z : r1.x);
          if (aw < ww_lo) {  // Russian roulette: survive with |W| / lo, at weight lo
            if (uww < aw / ww_lo) s.W = (s.W < R(0)) ? -ww_lo : ww_lo;
            else s.dead = true;
          } else {           // expected-value splitting into floor(m) or floor(m)+1 copies of W/m
            R m = aw / ww_hi;
            R room = R(ww_depth - sp);
            if (m > room + R(1)) m = room + R(1);
            R fl = floor(m);
            int n = (int)fl + ((uww < fl + R(1) - m) ? 0 : 1);
            s.W = s.W / m;
            for (int c = 1; c < n; ++c) {
#pragma unroll
              for (int i = 0; i < 3; ++i) stk_x[sp][i] = s.x[i];
              stk_W[sp] = s.W;
              stk_k[sp] = s.k + 1;
              stk_id[sp] = s.next_bid++;
              ++sp;
            }
          }
        }
      }
    } else {                   // boundary term: uniform point on the sphere
#pragma unroll
      for (int i = 0; i < DIM; ++i) s.x[i] = s.x[i] + dd * dz[i];
    }
    ++s.k;
  }

  if (accumulate && acc_p != kNoPoint) {
    double e0 = point_factor<DIM, R>(L, BATCHED ? Pall[acc_prob] : *Pshared, acc_p);
    if (!GRAD) {
      double c = (double)sh, n = (double)n_acc;
      s1 = n * c + (double)d1;
      s2 = n * c * c + 2.0 * c * (double)d1 + (double)d2;
    }
    atomicAdd(&L.sum[acc_p], s1 * e0);
    atomicAdd(&L.sumsq[acc_p], s2 * e0 * e0);
    atomicAdd(&L.count[acc_p], (unsigned long long)n_acc);
    if (GRAD) {
#pragma unroll
      for (int i = 0; i < DIM; ++i) {
        atomicAdd(&L.gsum[(int64_t)i * L.npts + acc_p], gs1[i] * e0);
        atomicAdd(&L.gsumsq[(int64_t)i * L.npts + acc_p], gs2[i] * e0 * e0);
      }
    }
  }
  // warp-reduce the statistics, one atomic per warp and word
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    st_steps += __shfl_down_sync(kFull, st_steps, off);
    st_walks += __shfl_down_sync(kFull, st_walks, off);
    st_capped += __shfl_down_sync(kFull, st_capped, off);
    st_nonfinite += __shfl_down_sync(kFull, st_nonfinite, off);
    st_outside += __shfl_down_sync(kFull, st_outside, off);
    if (MESH) {
      mvis.nodes += __shfl_down_sync(kFull, mvis.nodes, off);
      mvis.tris += __shfl_down_sync(kFull, mvis.tris, off);
      mvis.exhausted += __shfl_down_sync(kFull, mvis.exhausted, off);
    }
  }
  if (lane == 0) {
    atomicAdd(&L.stats[ST_STEPS], st_steps);
    atomicAdd(&L.stats[ST_WALKS], (unsigned long long)st_walks);
    if (st_capped) atomicAdd(&L.stats[ST_CAPPED], (unsigned long long)st_capped);
    if (st_nonfinite) atomicAdd(&L.stats[ST_NONFINITE], (unsigned long long)st_nonfinite);
    if (st_outside) atomicAdd(&L.stats[ST_OUTSIDE], (unsigned long long)st_outside);
    if (MESH) {
      atomicAdd(&L.stats[ST_MESH_NODES], mvis.nodes);
      atomicAdd(&L.stats[ST_MESH_TRIS], mvis.tris);
      if (mvis.exhausted) atomicAdd(&L.stats[ST_EXHAUSTED], (unsigned long long)mvis.exhausted);
    }
  }
}

#if !defined(__CUDACC_RTC__)
template <int DIM, typename R, bool MESH, bool BATCHED, bool WW, bool GRAD = false, bool DRIFT = false,
          int MINB = 0>
cudaError_t launch_walks_m(const WalkLaunch& L, int num_sms, cudaStream_t stream) {
  size_t smem = BATCHED ? 0 : (size_t)L.problem_bytes;
  if (MESH) smem += (sizeof(int) + sizeof(R)) * kMeshStack * kWalkBlock + 128 * kMeshTopMax;
  if (smem > 48 * 1024) {
    cudaError_t ea = cudaFuncSetAttribute(wos_walk_kernel<DIM, R, MESH, BATCHED, WW, GRAD, DRIFT, MINB>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ea != cudaSuccess) return ea;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, wos_walk_kernel<DIM, R, MESH, BATCHED, WW, GRAD, DRIFT, MINB>, kWalkBlock, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  if (L.blocks_per_sm > 0 && L.blocks_per_sm < per_sm) per_sm = L.blocks_per_sm;
  int grid = per_sm * num_sms;
  // total_items is ~0 when per-point walk counts give the total on the device: no cap then
  uint64_t warps_needed = L.total_items / 32 + 1;
  uint64_t blocks_needed = warps_needed / (kWalkBlock / 32) + 1;
  if ((uint64_t)grid > blocks_needed) grid = (int)(blocks_needed > 0 ? blocks_needed : 1);
  WalkLaunch arg = L;
  philox_round_keys(arg.seed, arg.rk);
  wos_walk_kernel<DIM, R, MESH, BATCHED, WW, GRAD, DRIFT, MINB><<<grid, kWalkBlock, smem, stream>>>(arg);
  return cudaGetLastError();
}

template <int DIM, typename R>
cudaError_t launch_walks_t(const WalkLaunch& L, int num_sms, cudaStream_t stream) {
  if (L.probs != nullptr)
    return (L.regs_variant == 1) ? launch_walks_m<DIM, R, false, true, false, false, false, 8>(L, num_sms, stream)
                                 : launch_walks_m<DIM, R, false, true, false>(L, num_sms, stream);
  if (L.drift) return launch_walks_m<DIM, R, false, false, false, false, true>(L, num_sms, stream);
  if (L.gsum != nullptr || L.ghat != nullptr)  // spatial gradient (no weight window)
    return (DIM == 3 && L.mesh) ? launch_walks_m<DIM, R, true, false, false, true>(L, num_sms, stream)
                                : launch_walks_m<DIM, R, false, false, false, true>(L, num_sms, stream);
  const bool ww = L.ww_lo > 0.0;
  if (DIM == 3 && L.mesh)
    return ww ? launch_walks_m<DIM, R, true, false, true>(L, num_sms, stream)
              : launch_walks_m<DIM, R, true, false, false>(L, num_sms, stream);
  return ww ? launch_walks_m<DIM, R, false, false, true>(L, num_sms, stream)
            : launch_walks_m<DIM, R, false, false, false>(L, num_sms, stream);
}

template <int DIM, typename R>
int blocks_per_sm_t() {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wos_walk_kernel<DIM, R, false, false, false, false>, kWalkBlock,
                                                sizeof(DevProblem<R>));
  return per_sm;
}
#endif  // !__CUDACC_RTC__

}  // namespace wos
