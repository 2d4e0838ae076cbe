// Allocation-free relative residual ||b - Y T x|| / ||b|| (no handle, no cudaMalloc).
//
// Why it exists: some callers of this library cannot allocate device memory at the
// point where they need a residual check -- for example a host framework whose
// pool allocator owns all device memory and forbids outside allocations (plugin
// code that is only handed device pointers), or a latency-critical loop where the
// implicit device synchronisation of cudaMalloc/cudaFree is not acceptable.
// aao_residual_norm needs a handle, and creating a handle allocates; this entry
// point needs neither.
//
// Its only scratch is the file-scope device array g_noalloc_scratch below (256 KiB).
// Host code cannot pass the array's name to a kernel (in host code the name is a
// host stand-in, not a device address), so the device address is looked up once per
// device with cudaGetSymbolAddress, with that device current, on the first call.
// With CUDA's lazy module loading (the default) that first lookup is also what loads
// this file's module -- the array and the kernels -- onto the device: a driver-side
// allocation of about 256 KiB plus code, held from then until the process exits (or
// until the device is reset).  Callers that cannot allocate at all later on make the
// first call at initialisation time; every call after it allocates nothing.  The
// cached address does not survive cudaDeviceReset (the module is unloaded with the
// context): a process that resets the device must not call this entry point again.
#include <mutex>
#include <string>

#include "aao_internal.cuh"

namespace {

constexpr int NA_NT = 256;              // threads per block
constexpr int NA_NB = 256;              // blocks (partial sums) per right-hand side
constexpr int NA_CH = 32;               // time levels per thread run
constexpr int NA_SCRATCH = 32768;       // doubles in the static scratch (256 KiB)
constexpr int NA_MAX_RHS = NA_SCRATCH / (2 * NA_NB);  // = 64
constexpr int NA_MAX_DEVICES = 64;

// Partial sums: [rhs][0: sum (b - YTx)^2 | 1: sum b^2][block].  Every slot that the
// final reduction reads is rewritten by the first kernel of the same call, so
// nothing has to be cleared between calls; contents persist between calls.
static __device__ __align__(256) double g_noalloc_scratch[NA_SCRATCH];

struct NaArgs {
  int d, N, n, m;
  double coef, diag;
};

__device__ __forceinline__ double na_apply_L(const double* __restrict__ v, int s, int ix, int iy, int iz,
                                             const NaArgs& a) {
  const int N = a.N;
  double sum = (ix > 0 ? v[s - 1] : 0.0) + (ix < N - 1 ? v[s + 1] : 0.0);
  if (a.d >= 2) sum += (iy > 0 ? v[s - N] : 0.0) + (iy < N - 1 ? v[s + N] : 0.0);
  if (a.d >= 3) sum += (iz > 0 ? v[s - N * N] : 0.0) + (iz < N - 1 ? v[s + N * N] : 0.0);
  return fma(-a.coef, sum, a.diag * v[s]);
}

__device__ __forceinline__ double na_block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = (l < NA_NT / 32) ? red[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;  // valid in thread 0
}

// Grid-stride form of the residual stencil: a fixed NA_NB blocks per rhs walk the
// (spatial tile, time run) work items, so the partial-sum count does not grow with size.
__global__ void __launch_bounds__(NA_NT) k_na_residual(const double* __restrict__ b,
                                                       const double* __restrict__ x,
                                                       double* __restrict__ part, NaArgs a) {
  __shared__ double red[NA_NT / 32];
  const int n = a.n, m = a.m, N = a.N;
  const long long rb = (long long)blockIdx.y * n * m;
  const int stiles = (m + NA_NT - 1) / NA_NT;
  const int runs = (n + NA_CH - 1) / NA_CH;
  const long long items = (long long)stiles * runs;
  double racc = 0.0, bacc = 0.0;
  for (long long it = blockIdx.x; it < items; it += gridDim.x) {
    const int s = (int)(it % stiles) * NA_NT + threadIdx.x;
    const int i0 = (int)(it / stiles) * NA_CH;
    const int i1 = min(n, i0 + NA_CH);
    if (s >= m) continue;
    const int ix = s % N;
    const int iy = (a.d >= 2) ? (s / N) % N : 0;
    const int iz = (a.d >= 3) ? s / (N * N) : 0;
    const double* xr = x + rb;
    double Lv1 = 0.0, Lv2 = 0.0, v1 = 0.0;
    for (int i = max(0, i0 - 2); i < i1; ++i) {
      const double* vi = xr + (long long)i * m;
      const double Lv = na_apply_L(vi, s, ix, iy, iz, a);
      if (i >= i0) {
        const double o = fma(-2.0, v1, Lv + Lv2);
        const double bb = b[rb + (long long)(n - 1 - i) * m + s];
        const double r = bb - o;
        racc = fma(r, r, racc);
        bacc = fma(bb, bb, bacc);
      }
      Lv2 = Lv1;
      Lv1 = Lv;
      v1 = vi[s];
    }
  }
  const double tr = na_block_sum(racc, red);
  const double tb = na_block_sum(bacc, red);
  if (threadIdx.x == 0) {
    double* p = part + (long long)blockIdx.y * 2 * NA_NB;
    p[blockIdx.x] = tr;
    p[NA_NB + blockIdx.x] = tb;
  }
}

__global__ void k_na_final(const double* __restrict__ part, double* __restrict__ relres) {
  const double* p = part + (long long)blockIdx.x * 2 * NA_NB;
  double s1 = 0.0, s2 = 0.0;
  for (int i = threadIdx.x; i < NA_NB; i += 32) {
    s1 += p[i];
    s2 += p[NA_NB + i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if (threadIdx.x == 0) relres[blockIdx.x] = (s2 > 0.0) ? sqrt(s1 / s2) : sqrt(s1);
}

std::mutex g_na_mu;
double* g_na_ptr[NA_MAX_DEVICES] = {nullptr};

thread_local std::string g_na_err;

aao_status na_fail(aao_status st, const std::string& msg) {
  g_na_err = msg;
  return st;
}

}  // namespace

extern "C" const char* aao_noalloc_last_error(void) { return g_na_err.c_str(); }

extern "C" aao_status aao_residual_norm_noalloc(const aao_grid* grid, int nt, double tau,
                                                const double* b, const double* x, double* relres,
                                                int nrhs, void* stream) {
  g_na_err.clear();
  if (!grid || !b || !x || !relres) return na_fail(AAO_EINVAL, "null pointer");
  if (grid->dim < 1 || grid->dim > 3) return na_fail(AAO_EINVAL, "dim must be 1, 2 or 3");
  if (grid->N < 1 || nt < 1) return na_fail(AAO_EINVAL, "N and nt must be >= 1");
  if (!(tau > 0.0) || !(grid->c2 > 0.0)) return na_fail(AAO_EINVAL, "tau and c2 must be > 0");
  if (nrhs < 1 || nrhs > NA_MAX_RHS)
    return na_fail(AAO_EINVAL, "nrhs must be in [1, " + std::to_string(NA_MAX_RHS) +
                                   "]: the static scratch holds " + std::to_string(NA_SCRATCH) +
                                   " partial sums (" + std::to_string(2 * NA_NB) + " per right-hand side)");
  long long m = 1;
  for (int i = 0; i < grid->dim; ++i) m *= grid->N;
  if (m > (1LL << 31) - 1 || (long long)nt * m > (1LL << 40))
    return na_fail(AAO_EINVAL, "problem too large");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(AAO_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= NA_MAX_DEVICES) return na_fail(AAO_EINVAL, "device index out of range");
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
      // once per device, with that device current: device address of the static array
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess)
        return na_fail(AAO_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_na_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_na_ptr[dev];
  }
  NaArgs a;
  a.d = grid->dim;
  a.N = grid->N;
  a.n = nt;
  a.m = (int)m;
  const double h = 1.0 / (grid->N + 1.0);
  a.coef = grid->c2 * tau * tau / (2.0 * h * h);
  a.diag = 1.0 + 2.0 * a.d * a.coef;
  cudaStream_t s = (cudaStream_t)stream;
  k_na_residual<<<dim3(NA_NB, nrhs), NA_NT, 0, s>>>(b, x, scratch, a);
  k_na_final<<<nrhs, 32, 0, s>>>(scratch, relres);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(AAO_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  return AAO_OK;
}
