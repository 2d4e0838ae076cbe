// FP32 instantiations of the time-pipeline kernel (kernels in k_time.cuh): FP32
// vectors, and FP32 arithmetic on FP64 vectors (converted on load and store).  The
// bulk-staged variants of the latter are instantiated in k_time32_bulk.cu.
#include <cstdint>

#include "k_time.cuh"

namespace aao {

template cudaError_t launch_time<float>(const Plan&, const float*, float*, int, cudaStream_t,
                                        uint64_t*);

cudaError_t time_bulk_launch(int v, const Plan& P, const double* in, double* out, int nrhs, cudaStream_t s);

// Variants 0..7 are those of k_time.cuh, 16 and 17 its variants 5 and 7 with integer
// conversions, 18..21 variants 5 and 7 with the tile's loads batched ahead of their
// conversion (8 or 16 tasks per batch); 8..15 the bulk-staged kernel (bits of v - 8:
// tile, staged table slice, integer conversions), which needs 16-byte aligned vectors (a
// vector that is only 8-byte aligned takes the batched-load kernel of the same tile).
cudaError_t launch_time_mixed(const Plan& P, const double* in, double* out, int nrhs, cudaStream_t s,
                              uint64_t* nl) {
  if (nl) ++*nl;
  const int v = P.time_variant32;
  const bool aligned = (((uintptr_t)in | (uintptr_t)out) & 15) == 0;
  if (v >= 8 && v < 16) {
    if (aligned) return time_bulk_launch(v & 7, P, in, out, nrhs, s);
    Plan Q = P;
    Q.time_variant32 = (v & 1) ? 19 : 18;
    return time_dispatch<float, double>(Q, in, out, nrhs, s);
  }
  return time_dispatch<float, double>(P, in, out, nrhs, s);
}

}  // namespace aao
