// wos_nf_f64.cu -- FP64 next-flight walk kernels: per-walk replay of the oracle.
#include "wos_nf_impl.cuh"

namespace wos {

cudaError_t launch_nf_f64(const WalkLaunch& L, int num_sms, cudaStream_t stream) {
  return (L.dim == 2) ? launch_nf_t<2, double>(L, num_sms, stream) : launch_nf_t<3, double>(L, num_sms, stream);
}

}  // namespace wos
