// wos_walk_f32.cu -- FP32 walk kernels (2D and 3D): the production path.
#include "wos_walk_impl.cuh"

namespace wos {

cudaError_t launch_walks_f32(const WalkLaunch& L, int num_sms, cudaStream_t stream) {
  return (L.dim == 2) ? launch_walks_t<2, float>(L, num_sms, stream)
                      : launch_walks_t<3, float>(L, num_sms, stream);
}

int walk_blocks_per_sm_f32(int dim) {
  return dim == 2 ? blocks_per_sm_t<2, float>() : blocks_per_sm_t<3, float>();
}

}  // namespace wos
