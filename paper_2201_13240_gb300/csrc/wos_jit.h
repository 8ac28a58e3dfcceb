// wos_jit.h -- problem-specialised walk kernels (runtime compilation); internal.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "wos_problem.cuh"

namespace wos {

// kernel variants of one problem and precision (the domain fixes MESH, the problem DRIFT)
enum { kJitPlain = 0, kJitWindow = 1, kJitGrad = 2, kJitVariants = 3 };

struct JitState {
  cudaKernel_t kernel[2][kJitVariants] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};  // [fp64]
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

}  // namespace wos
