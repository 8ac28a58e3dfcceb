// wos_internal.h -- launch descriptors shared by the C-ABI layer and the
// walk-kernel translation units (not part of the public interface).
#pragma once

#if defined(__CUDACC_RTC__)
#include "wos_math.cuh"  // fixed-width integer types of runtime compilation
#else
#include <cuda_runtime.h>
#include <stdint.h>
#endif

namespace wos {

// statistics words written by the walk kernel (added atomically)
enum {
  ST_STEPS = 0, ST_WALKS = 1, ST_CAPPED = 2, ST_NONFINITE = 3, ST_OUTSIDE = 4, ST_INNER = 5,
  ST_MESH_NODES = 6, ST_MESH_TRIS = 7, ST_EXHAUSTED = 8, ST_WORDS = 9
};

struct WalkLaunch {
  const void* problem;            // DevProblem<R> in device memory
  int problem_bytes;              // sizeof(DevProblem<R>), multiple of 16
  int dim;
  const float* pts;               // SoA [dim][npts], device
  int64_t npts;
  const int64_t* walk_end;        // inclusive prefix sums of walks per point, or null
  int64_t walks_uniform;
  uint64_t total_items;           // total walks of the launch
  uint64_t seed;
  uint64_t walk_offset;
  double eps;
  double sigma_bar;
  int64_t max_steps;
  double* sum;                    // [npts], accumulated
  double* sumsq;                  // [npts], accumulated
  unsigned long long* count;      // [npts], accumulated
  unsigned long long* stats;      // [ST_WORDS], accumulated
  unsigned long long* work_counter;  // zeroed before the launch
  double* uhat;                   // optional per-walk estimates [total_items]
  int64_t* steps_out;             // optional per-walk step counts [total_items]
  const float* radial_tab;        // FP32 Newton start table of the launch's dimension
  int mesh;                       // the domain is a triangle mesh
  // batched launches: many problems, points of problem i are prob_offsets[i] .. prob_offsets[i+1]-1
  const void* probs;              // contiguous DevProblem<R>[nprob], device
  const int64_t* prob_offsets;    // [nprob + 1], device
  const double* sigma_bars;       // [nprob], device
  int32_t nprob;
  // weight window (ww_lo > 0 enables it)
  double ww_lo, ww_hi;
  int32_t ww_depth;
  // spatial gradient (Supplemental Sec. 2): either pointer non-null enables it
  double* gsum;                   // SoA [dim][npts], accumulated
  double* gsumsq;                 // SoA [dim][npts], accumulated
  double* ghat;                   // optional per-walk gradients SoA [dim][total_items]
  // next-flight launches: cap on the inner iterations of one ball, and the kernels: 0 the
  // printed approximations, N > 0 the series with N terms
  int64_t nf_max_inner;
  int32_t nf_series;
  int drift;                      // the problem has an extra drift (omega fields)
  // launch schedule (0 = the kernel's own rule): walks claimed per warp at a time, resident
  // blocks launched per SM, and the register-cap variant of batched launches (1: 8 blocks/SM)
  uint32_t chunk;
  int32_t blocks_per_sm;
  int32_t regs_variant;
  // Philox round keys of `seed`, set by the launch functions (philox_round_keys): in the
  // kernel's parameter space each round's key is a constant operand of the XOR
  uint32_t rk[20];
};

// adjoint launch: d(sum_p grad_u[p] mean_u[p]) / d(sigma grid nodes), added to grad_sigma
struct AdjLaunch {
  const void* problem;
  int problem_bytes;
  int dim;
  const float* pts;
  int64_t npts;
  int64_t walks_uniform;
  uint64_t total_items;           // walks of this launch: items item_base .. item_base + total_items - 1
  uint64_t item_base;             // item = point * walks_uniform + walk
  uint64_t seed;
  uint64_t walk_offset;
  double eps;
  double sigma_bar;
  int64_t max_steps;
  const double* grad_u;           // [npts]
  double* grad_sigma;             // [sigma grid nodes], accumulated (sigma launches)
  double* grad_alpha;             // [alpha grid nodes], accumulated (alpha launches)
  int alpha;                      // 1: gradient with respect to the alpha B-spline grid
  int priv_nodes;                 // > 0: accumulate per CTA in shared memory over this many nodes
  unsigned long long* stats;      // optional
  unsigned long long* work_counter;
  const float* radial_tab;
  void* totals;                   // [total_items] walk totals in the walk's precision (pass 1 writes them)
  int pass;                       // 1: the walks' totals, 2: the replay that scatters
  uint32_t rk[20];                // Philox round keys of `seed`, set by the launch (philox_round_keys)
};

#if !defined(__CUDACC_RTC__)
cudaError_t launch_adjoint_f32(const AdjLaunch& L, int num_sms, cudaStream_t stream);
cudaError_t launch_adjoint_f64(const AdjLaunch& L, int num_sms, cudaStream_t stream);
// an adjoint kernel compiled at run time for one problem (same parameter block and launch shape)
cudaError_t launch_adjoint_kernel(const AdjLaunch& L, cudaKernel_t kernel, int real_bytes, int num_sms,
                                  cudaStream_t stream);

// launch the persistent walk kernel; returns a cudaError_t
cudaError_t launch_walks_f32(const WalkLaunch& L, int num_sms, cudaStream_t stream);
cudaError_t launch_walks_f64(const WalkLaunch& L, int num_sms, cudaStream_t stream);

// a walk kernel compiled at run time for one problem (same parameter block and launch
// shape as wos_walk_kernel); real_bytes = sizeof the walk's real type
cudaError_t launch_walks_kernel(const WalkLaunch& L, cudaKernel_t kernel, int real_bytes, int num_sms,
                                cudaStream_t stream);

// next-flight walks (Sec. 5.2)
cudaError_t launch_nf_f32(const WalkLaunch& L, int num_sms, cudaStream_t stream);
cudaError_t launch_nf_f64(const WalkLaunch& L, int num_sms, cudaStream_t stream);

// per-SM resident blocks of the walk kernel (for reporting)
int walk_blocks_per_sm_f32(int dim);
int walk_blocks_per_sm_f64(int dim);
#endif

}  // namespace wos
