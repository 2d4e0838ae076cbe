// FP64 instantiations of the time-pipeline kernel (kernels in k_time.cuh).
#include "k_time.cuh"

namespace aao {

template cudaError_t launch_time<double>(const Plan&, const double*, double*, int, cudaStream_t,
                                         uint64_t*);

}  // namespace aao
