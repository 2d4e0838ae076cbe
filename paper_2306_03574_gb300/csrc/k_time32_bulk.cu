// Bulk-staged FP32 time pipeline on FP64 vectors (kernels in k_time_bulk.cuh), and the
// counter of bounded waits that gave up.
#include "k_time_bulk.cuh"

namespace aao {

cudaError_t time_bulk_launch(int v, const Plan& P, const double* in, double* out, int nrhs, cudaStream_t s) {
  return time_bulk_dispatch(v, P, in, out, nrhs, s);
}

}  // namespace aao

// Bounded waits of the library's kernels that gave up (statistics; 0 in a healthy run).
extern "C" unsigned int aao_wait_timeouts(void) {
  unsigned int v = 0;
  if (cudaMemcpyFromSymbol(&v, aao::g_wait_timeouts, sizeof(v)) != cudaSuccess) {
    cudaGetLastError();
    return 0xFFFFFFFFu;
  }
  return v;
}
