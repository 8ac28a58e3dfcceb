// wos_peaks.cu -- measurement utilities (not part of the method): sustained rates of
// the units the walk kernels run on, measured on the device the context uses, so that
// roofline fractions divide by measured peaks rather than nominal ones.
//   FP32 lanes: independent chains of fused multiply-adds (one lane operation each; the
//               FP32/INT32 lanes also bound the issue rate of every other instruction);
//   MUFU:       independent chains of approximate reciprocal square roots (the
//               special-function unit that evaluates the walk's exp, log, sin, sqrt);
//   L2 read:    repeated 16-byte loads of a buffer small enough to stay in L2, with the
//               L1 bypassed (cache-global loads).
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "wos_capi_state.h"

namespace {

constexpr int kPeakBlock = 256;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kPeakBlock) peak_ffma_kernel(float* sink, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 1e-3f * (float)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = fmaf(x[k], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == -1.0f) sink[threadIdx.x & 63] = s;  // never true for these inputs; keeps the chains live
}

__device__ __forceinline__ float rsqrt_approx(float v) {
  float r;
  asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}

__global__ void __launch_bounds__(kPeakBlock) peak_mufu_kernel(float* sink, int iters) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 1.5f + 1e-3f * (float)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int k = 0; k < kChains; ++k) x[k] = rsqrt_approx(x[k]);  // stays in (0.5, 2): no denormals
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == -1.0f) sink[threadIdx.x & 63] = s;
}

// every thread reads 16-byte words of the buffer, grid-strided, `reps` times
__global__ void __launch_bounds__(kPeakBlock) peak_l2_kernel(const float4* buf, int64_t nvec, int reps, float* sink) {
  float acc = 0.0f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int r = 0; r < reps; ++r) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nvec; i += stride) {
      float4 v = __ldcg(buf + i);
      acc += v.x + v.y + v.z + v.w;
    }
  }
  if (acc == -1.0f) sink[threadIdx.x & 63] = acc;
}

int pfail(wos_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

}  // namespace

extern "C" int wos_measure_peak(wos_ctx* ctx, int32_t which, void* buf, int64_t bytes, double* rate, double* ms_out,
                                void* stream) {
  if (!ctx) return WOS_EINVAL;
  if (!rate) return pfail(ctx, WOS_EINVAL, "null output");
  if (which < WOS_PEAK_FP32_LANES || which > WOS_PEAK_L2_READ) return pfail(ctx, WOS_EINVAL, "unknown unit");
  if (which == WOS_PEAK_L2_READ && (!buf || bytes < (1 << 20) || (reinterpret_cast<uintptr_t>(buf) & 15) != 0))
    return pfail(ctx, WOS_EINVAL, "the L2 measurement needs a 16-byte aligned device buffer of at least 1 MiB");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != ctx->device)
    return pfail(ctx, WOS_EINVAL, "make the context's device current");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the sink is never written (the kernels' conditions are false for these inputs and a
  // zero-filled buffer); the first 256 bytes of the context's scratch stand in for it
  float* sink = reinterpret_cast<float*>(ctx->scratch);
  const int blocks = ctx->num_sms * 4;  // 32 warps per SM
  const int64_t threads = (int64_t)blocks * kPeakBlock;
  const int reps = 5;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  double work = 0.0;  // operations or bytes per launch
  for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {  // pass 0 warms up
    if (pass == 1) e = cudaEventRecord(e0, st);
    for (int r = 0; r < (pass == 0 ? 1 : reps) && e == cudaSuccess; ++r) {
      if (which == WOS_PEAK_FP32_LANES) {
        const int iters = 16384;
        peak_ffma_kernel<<<blocks, kPeakBlock, 0, st>>>(sink, iters, 0.999999f, 1e-7f);
        work = (double)threads * iters * 16 * kChains;
      } else if (which == WOS_PEAK_MUFU) {
        const int iters = 2048;
        peak_mufu_kernel<<<blocks, kPeakBlock, 0, st>>>(sink, iters);
        work = (double)threads * iters * 16 * kChains;
      } else {
        const int64_t nvec = bytes / 16;
        const int l2reps = (int)(4e10 / (double)bytes) + 1;  // about 40 GB per launch
        peak_l2_kernel<<<blocks, kPeakBlock, 0, st>>>(static_cast<const float4*>(buf), nvec, l2reps, sink);
        work = (double)nvec * 16.0 * l2reps;
      }
      e = cudaGetLastError();
    }
  }
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return pfail(ctx, WOS_ECUDA, std::string("peak measurement: ") + cudaGetErrorString(e));
  const double per_launch_ms = (double)ms / reps;
  *rate = work / (per_launch_ms * 1e-3);
  if (ms_out) *ms_out = per_launch_ms;
  return WOS_OK;
}
