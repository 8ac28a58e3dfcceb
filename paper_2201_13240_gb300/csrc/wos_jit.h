// wos_jit.h -- problem-specialised walk kernels (runtime compilation); internal.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "wos_problem.cuh"

namespace wos {

// kernel variants of one problem and precision (the domain fixes MESH, the problem DRIFT);
// bit kJitAdjoint of a variant mask asks for the path-replay adjoint kernels (sigma and alpha,
// each as its two passes); kJitExprs counts the kernels one program can hold
enum { kJitPlain = 0, kJitWindow = 1, kJitGrad = 2, kJitVariants = 3, kJitAdjoint = 3, kJitExprs = 7 };

struct JitState {
  cudaKernel_t kernel[2][kJitVariants] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};  // [fp64]
  cudaKernel_t adjoint[2][2][2] = {};  // [fp64][alpha][pass - 1]
  std::vector<cudaLibrary_t> libs;
};

// the generated program: field code for P, after the walk kernel's headers
std::string jit_source(const DevProblem<double>& P);

// NVRTC compile of the variants in variant_mask (bit v = variant v) for sm_103a; no device needed
int jit_compile(const DevProblem<double>& P, bool fp64, int variant_mask, std::vector<char>* cubin,
                std::vector<std::string>* lowered, std::string* log);

// compile and load the variants not yet loaded; the current device must be the problem's
int jit_specialise(JitState* js, const DevProblem<double>& P, bool fp64, int variant_mask, std::string* why);

void jit_release(JitState* js);

// ---- batches of problems: one kernel for every problem of a batch ----
// Field f (FieldId order: alpha, phi, sigma, f, g, u_m) is "uniform" when every problem of
// the batch has the same kind and, for CONST and SST, the same value or terms: its code is
// generated from the representative problem (grids read the walk's own problem descriptor).
// Other fields call the generic interpreter on the walk's problem.
struct BatchJitInfo {
  DevProblem<double> rep;   // the first problem (the representative)
  uint32_t uniform = 0;     // bit FieldId: uniform across the batch
  bool f_kind_uniform = true;
};

// true when field F of A and field G of B generate the same code
bool same_field(const DevProblem<double>& A, const DevField<double>& F, const DevProblem<double>& B,
                const DevField<double>& G);

std::string jit_source_batch(const BatchJitInfo& info);

// the shared fields of a batch whose problems are probs[0..n)
void batch_jit_info(const DevProblem<double>* probs, int n, BatchJitInfo* info);

// NVRTC compile (no device, no load) of a batch's kernels of one precision
int jit_compile_batch(const BatchJitInfo& info, bool fp64, std::vector<char>* cubin, std::vector<std::string>* lowered,
                      std::string* log);

// compile and load the batched kernels of one precision, both register caps (index 0: the
// default, 1: eight blocks per SM) into js->kernel[fp64][0..1]
int jit_specialise_batch(JitState* js, const BatchJitInfo& info, bool fp64, std::string* why);

}  // namespace wos
