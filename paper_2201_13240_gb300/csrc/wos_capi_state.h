// wos_capi_state.h -- the library-owned handle objects behind include/wos.h
// (host code only; not part of the public interface).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "wos.h"
#include "wos_jit.h"
#include "wos_problem.cuh"

using wos::DevField;
using wos::DevProblem;
using wos::DevTerm;

struct wos_ctx {
  int device = 0;
  int num_sms = 0;
  std::string err;
  // scratch: [0] work counter, [8..8+ST_WORDS) default stats, [24..29) sigma-bar reduction
  unsigned long long* scratch = nullptr;
  // walks-per-point prefix sums
  int64_t* walk_end = nullptr;
  int64_t walk_end_cap = 0;
  // FP32 inverse radial CDF start tables for 2D and 3D (wos::kTabSize floats each)
  float* radial_tab[2] = {nullptr, nullptr};
  // buffers of wos_solve_host
  float* h_pts = nullptr;
  double* h_acc = nullptr;  // sum, sumsq, mean, var, se: 5 * cap doubles
  int64_t* h_count = nullptr;
  int64_t host_cap = 0;
  // FP64 accumulators of wos_solve_mean / wos_solve_batched (sum, sumsq, count per point)
  double* mv_sum = nullptr;   // 2 * mv_cap doubles: sum, then sumsq
  int64_t* mv_count = nullptr;
  int64_t mv_cap = 0;
  // FP64 gradient buffer of wos_adjoint (sigma nodes + alpha nodes)
  double* adj_buf = nullptr;
  int64_t adj_cap = 0;
  // per-walk totals between the two passes of the path-replay adjoint
  void* adj_totals = nullptr;
  size_t adj_totals_bytes = 0;
};

struct wos_batch {
  wos_ctx* ctx = nullptr;
  int device = 0;                     // kept here: destroy must not read a destroyed context
  int dim = 0;
  int32_t nprob = 0;
  int64_t npts = 0;
  DevProblem<float>* d32 = nullptr;   // [nprob]
  DevProblem<double>* d64 = nullptr;  // [nprob]
  int64_t* offsets = nullptr;         // [nprob + 1]
  double* sigma_bars = nullptr;       // [nprob]
  int64_t* walk_end = nullptr;        // [npts] prefix sums for per-point walk counts
  wos_schedule sched = {0, 0, 0, 0};  // launch schedule (wos_batch_set_schedule / autotune)
  wos::BatchJitInfo jit_info;         // fields shared by every problem (wos_batch_specialize)
  wos::JitState jit;                  // batched kernels compiled for them: [fp64][regs variant]
};

struct wos_problem {
  wos_ctx* ctx = nullptr;
  int device = 0;  // kept here: destroy must not read a destroyed context
  int dim = 0;
  DevProblem<float>* d32 = nullptr;
  DevProblem<double>* d64 = nullptr;
  DevProblem<double> host64;  // host copy for the sigma_bar lattice bounds
  DevProblem<float> host32;   // host copy for batches
  float* mesh_nodes = nullptr;  // device BVH of a mesh boundary
  float* mesh_tris = nullptr;
  float* mgrid32 = nullptr;     // mesh distance grid (FP32 walks)
  double* mgrid64 = nullptr;    // the same grid in FP64 (replay walks)
  double mesh_lo[3] = {0, 0, 0}, mesh_hi[3] = {0, 0, 0};
  int mesh_depth = 0;
  wos::JitState jit;  // walk kernels compiled for this problem (wos_problem_specialize)
};

