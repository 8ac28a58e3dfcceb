// wos_walk_f32.cu -- FP32 walk kernels (2D and 3D): the production path.
#include "wos_walk_impl.cuh"

namespace wos {

cudaError_t launch_walks_f32(const WalkLaunch& L, int num_sms, cudaStream_t stream) {
  return (L.dim == 2) ? launch_walks_t<2, float>(L, num_sms, stream)
                      : launch_walks_t<3, float>(L, num_sms, stream);
}

cudaError_t launch_walks_kernel(const WalkLaunch& L, cudaKernel_t kernel, int real_bytes, int num_sms,
                                cudaStream_t stream) {
  const void* fn = reinterpret_cast<const void*>(kernel);
  size_t smem = (size_t)L.problem_bytes;
  if (L.mesh) smem += (sizeof(int) + (size_t)real_bytes) * kMeshStack * kWalkBlock + 128 * kMeshTopMax;
  if (smem > 48 * 1024) {
    cudaError_t ea = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ea != cudaSuccess) return ea;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kWalkBlock, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  if (L.blocks_per_sm > 0 && L.blocks_per_sm < per_sm) per_sm = L.blocks_per_sm;
  int grid = per_sm * num_sms;
  uint64_t warps_needed = L.total_items / 32 + 1;
  uint64_t blocks_needed = warps_needed / (kWalkBlock / 32) + 1;
  if ((uint64_t)grid > blocks_needed) grid = (int)(blocks_needed > 0 ? blocks_needed : 1);
  WalkLaunch arg = L;
  philox_round_keys(arg.seed, arg.rk);
  void* args[] = {&arg};
  return cudaLaunchKernel(fn, dim3(grid), dim3(kWalkBlock), args, smem, stream);
}

int walk_blocks_per_sm_f32(int dim) {
  return dim == 2 ? blocks_per_sm_t<2, float>() : blocks_per_sm_t<3, float>();
}

}  // namespace wos
