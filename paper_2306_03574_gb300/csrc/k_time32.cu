// FP32 instantiations of the time-pipeline kernel (kernels in k_time.cuh): FP32
// vectors, and FP32 arithmetic on FP64 vectors (converted on load and store).
#include "k_time.cuh"

namespace aao {

template cudaError_t launch_time<float>(const Plan&, const float*, float*, int, cudaStream_t,
                                        uint64_t*);

cudaError_t launch_time_mixed(const Plan& P, const double* in, double* out, int nrhs, cudaStream_t s,
                              uint64_t* nl) {
  if (nl) ++*nl;
  return time_dispatch<float, double>(P, in, out, nrhs, s);
}

}  // namespace aao
