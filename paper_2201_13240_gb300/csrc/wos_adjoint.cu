// wos_adjoint.cu -- instantiations of the path-replay adjoint kernel.
#include "wos_adjoint_impl.cuh"

namespace wos {

cudaError_t launch_adjoint_f32(const AdjLaunch& L, int num_sms, cudaStream_t stream) {
  return (L.dim == 2) ? launch_adjoint_t<2, float>(L, num_sms, stream) : launch_adjoint_t<3, float>(L, num_sms, stream);
}

// an adjoint kernel compiled at run time for one problem: the launch shape of launch_adjoint_m
cudaError_t launch_adjoint_kernel(const AdjLaunch& L, cudaKernel_t kernel, int real_bytes, int num_sms,
                                  cudaStream_t stream) {
  const void* fn = reinterpret_cast<const void*>(kernel);
  size_t smem = (size_t)L.problem_bytes + ((L.alpha && L.pass == 2) ? (size_t)L.priv_nodes * (size_t)real_bytes : 0);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kAdjBlock, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int grid = per_sm * num_sms;
  uint64_t blocks_needed = (L.total_items + kAdjBlock - 1) / kAdjBlock;
  if ((uint64_t)grid > blocks_needed) grid = (int)(blocks_needed > 0 ? blocks_needed : 1);
  AdjLaunch arg = L;
  philox_round_keys(arg.seed, arg.rk);
  void* args[] = {&arg};
  return cudaLaunchKernel(fn, dim3(grid), dim3(kAdjBlock), args, smem, stream);
}

cudaError_t launch_adjoint_f64(const AdjLaunch& L, int num_sms, cudaStream_t stream) {
  return (L.dim == 2) ? launch_adjoint_t<2, double>(L, num_sms, stream)
                      : launch_adjoint_t<3, double>(L, num_sms, stream);
}

}  // namespace wos
