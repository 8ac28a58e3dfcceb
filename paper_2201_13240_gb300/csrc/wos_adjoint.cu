// wos_adjoint.cu -- instantiations of the path-replay adjoint kernel.
#include "wos_adjoint_impl.cuh"

namespace wos {

cudaError_t launch_adjoint_f32(const AdjLaunch& L, int num_sms, cudaStream_t stream) {
  return (L.dim == 2) ? launch_adjoint_t<2, float>(L, num_sms, stream) : launch_adjoint_t<3, float>(L, num_sms, stream);
}

cudaError_t launch_adjoint_f64(const AdjLaunch& L, int num_sms, cudaStream_t stream) {
  return (L.dim == 2) ? launch_adjoint_t<2, double>(L, num_sms, stream)
                      : launch_adjoint_t<3, double>(L, num_sms, stream);
}

}  // namespace wos
