// wos_walk_f64.cu -- FP64 walk kernels (2D and 3D): the replay path that
// reproduces the FP64 oracle's walks from the same Philox streams.
#include "wos_walk_impl.cuh"

namespace wos {

cudaError_t launch_walks_f64(const WalkLaunch& L, int num_sms, cudaStream_t stream) {
  return (L.dim == 2) ? launch_walks_t<2, double>(L, num_sms, stream)
                      : launch_walks_t<3, double>(L, num_sms, stream);
}

int walk_blocks_per_sm_f64(int dim) {
  return dim == 2 ? blocks_per_sm_t<2, double>() : blocks_per_sm_t<3, double>();
}

}  // namespace wos
