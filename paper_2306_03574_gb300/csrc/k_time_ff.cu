// Double-float instantiations of the time-pipeline kernel (kernels in k_time.cuh):
// FP64 vectors in and out, every operation of the pipeline in double-word arithmetic
// on the FP32 pipes (dfloat.cuh).
#include "k_time.cuh"

namespace aao {

cudaError_t launch_time_ff(const Plan& P, const double* in, double* out, int nrhs, cudaStream_t s,
                           uint64_t* nl) {
  if (nl) ++*nl;
  return time_dispatch<dfl, double>(P, in, out, nrhs, s);
}

}  // namespace aao
