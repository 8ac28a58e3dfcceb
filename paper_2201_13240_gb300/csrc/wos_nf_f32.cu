// wos_nf_f32.cu -- FP32 next-flight walk kernels (2D and 3D).
#include "wos_nf_impl.cuh"

namespace wos {

cudaError_t launch_nf_f32(const WalkLaunch& L, int num_sms, cudaStream_t stream) {
  return (L.dim == 2) ? launch_nf_t<2, float>(L, num_sms, stream) : launch_nf_t<3, float>(L, num_sms, stream);
}

}  // namespace wos
