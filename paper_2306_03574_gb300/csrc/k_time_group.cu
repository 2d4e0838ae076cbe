// Grouped launch of the time pipeline (serving): one launch maps the modes of every
// problem in a (precision, n) bucket.  Block b belongs to problem r with
// tile[r] <= b < tile[r+1] and runs the problem's tile b - tile[r] with the same
// device code, variant and tile shape as the problem's solo launch (k_time.cuh), so
// its output is bit for bit that of the solo launch.  Problems already converged
// (scalars done) are skipped.  FP64 and double-float arithmetic on FP64 vectors.
#include "k_time.cuh"

namespace aao {

namespace {

template <typename R, int L, int NS, int NT, int FFTV, int LAY, int STG, int PRE>
__global__ void __launch_bounds__(NT) k_g_time(const TimeGroup<R>* __restrict__ g) {
  const int r = group_find(g->tile, g->count, blockIdx.x);
  const TimeGroupEntry<R>& e = g->e[r];
  if (e.sc->done) return;
  TimeArgs a;
  a.m = e.m;
  a.n = L;
  a.npairs = e.npairs;
  time_body<R, double, L, NS, NT, FFTV, LAY, STG, 0, PRE>(e.in, e.out, a, e.tb, blockIdx.x - g->tile[r]);
}

// The variant of each precision that has a grouped form -- the precision's default --
// and its configuration, which must equal the solo launch's (k_time.cuh,
// time_launch_L): FP64 variant 3 (radix-16 stage plan, 2048/L mode pairs x 128 threads,
// sequence-major layout); double-float variant 12 (radix-16, 4096/L x 256, interleaved
// layout without the staged table slice, loads batched 8 tasks at a time).  A problem
// whose handle runs another variant takes its solo launch instead.
template <typename R> struct GroupTimeCfg;
template <> struct GroupTimeCfg<double> {
  static constexpr int V = 3, PAIRS = 2048, NT = 128, FFTV = 1, LAY = 0, STG = -1, PRE = 0;
};
template <> struct GroupTimeCfg<dfl> {
  static constexpr int V = 12, PAIRS = 4096, NT = 256, FFTV = 1, LAY = 1, STG = 0, PRE = 8;
};

template <typename R, int L>
cudaError_t g_time_L(const TimeGroup<R>* d, int total, cudaStream_t s) {
  using G = GroupTimeCfg<R>;
  using C = typename Cplx<R>::T;
  constexpr int NS = G::PAIRS / L;
  constexpr bool STAGED = G::STG < 0 ? G::LAY == 1 : G::STG == 1;
  const size_t smem = sizeof(C) * (SLay<L, NS, G::LAY>::size + (STAGED ? 2 * NS * (L / 2 + 1) : 0) + L) +
                      2 * sizeof(R) * L;
  auto kern = k_g_time<R, L, NS, G::NT, G::FFTV, G::LAY, G::STG, G::PRE>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  kern<<<total, G::NT, smem, s>>>(d);
  return cudaGetLastError();
}

}  // namespace

template <typename R>
int group_time_tiles(int L, int m) {
  const int ns = GroupTimeCfg<R>::PAIRS / L;
  return (m + 2 * ns - 1) / (2 * ns);
}
template int group_time_tiles<double>(int, int);
template int group_time_tiles<dfl>(int, int);

template <typename R>
int group_time_variant() { return GroupTimeCfg<R>::V; }
template int group_time_variant<double>();
template int group_time_variant<dfl>();

template <typename R>
cudaError_t launch_group_time(int L, int variant, const TimeGroup<R>* d_group, int total_tiles, cudaStream_t s) {
  if (variant != group_time_variant<R>()) return cudaErrorInvalidValue;
  switch (L) {
    case 64: return g_time_L<R, 64>(d_group, total_tiles, s);
    case 128: return g_time_L<R, 128>(d_group, total_tiles, s);
    case 256: return g_time_L<R, 256>(d_group, total_tiles, s);
    case 512: return g_time_L<R, 512>(d_group, total_tiles, s);
    case 1024: return g_time_L<R, 1024>(d_group, total_tiles, s);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_group_time<double>(int, int, const TimeGroup<double>*, int, cudaStream_t);
template cudaError_t launch_group_time<dfl>(int, int, const TimeGroup<dfl>*, int, cudaStream_t);

}  // namespace aao
