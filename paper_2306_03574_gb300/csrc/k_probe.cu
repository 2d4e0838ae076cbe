// Arithmetic-rate probes (statistics for the roofline, not part of the method): a
// kernel of independent fused multiply-add chains on every SM, timed with CUDA events.
// The FP64 probe measures the rate of GB300's FP64 pipe, which bounds every FP64 kernel
// of the path; the FP32 probe the FP32 pipes, which bound the double-word kernels.
#include <cuda_runtime.h>

#include "aao_internal.cuh"

namespace {

constexpr int PROBE_NT = 256;
constexpr int PROBE_CHAINS = 8;

template <typename T>
__global__ void __launch_bounds__(PROBE_NT) k_fma_probe(T* out, int iters, T a, T b) {
  T x[PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = T(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = fma(x[c], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) s += x[c];
  if (s == T(12345.678)) out[0] = s;  // keeps the chains live; practically never taken
}

template <typename T>
aao_status probe(int iters, double* tflops, double* ms) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return AAO_ECUDA;
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return AAO_ENOMEM;
  }
  const int blocks = sms * 8;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  aao_status st = AAO_OK;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    st = AAO_ECUDA;
  } else {
    const T a = T(0.999999), b = T(1e-7);
    k_fma_probe<T><<<blocks, PROBE_NT, 0, s>>>(out, iters / 16, a, b);  // warm-up
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0, s);
      k_fma_probe<T><<<blocks, PROBE_NT, 0, s>>>(out, iters, a, b);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        st = AAO_ECUDA;
        break;
      }
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      best = t < best ? t : best;
    }
    if (st == AAO_OK && cudaGetLastError() != cudaSuccess) st = AAO_ECUDA;
    const double flops = 2.0 * PROBE_CHAINS * (double)iters * PROBE_NT * blocks;
    if (ms) *ms = best;
    if (tflops) *tflops = flops / (best * 1e-3) / 1e12;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaFree(out);
  return st;
}

}  // namespace

extern "C" aao_status aao_alu_peak(int precision, int iters, double* tflops, double* ms) {
  if (iters < 16 || (precision != AAO_PREC_FP64 && precision != AAO_PREC_FP32_IR)) return AAO_EINVAL;
  return precision == AAO_PREC_FP64 ? probe<double>(iters, tflops, ms) : probe<float>(iters, tflops, ms);
}
