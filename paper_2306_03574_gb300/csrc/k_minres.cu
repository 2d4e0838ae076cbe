// Preconditioned MINRES vector kernels and scalar recurrences on the device
// (Section 3 uses MINRES with P_alpha; the recurrences are the standard
// Lanczos + Givens form of preconditioned MINRES: with P = L L^T it is MINRES on
// L^{-1} A L^{-T} written so that only P^{-1} is applied).
//
// Per iteration j (z~_j = P^{-1} v_j unnormalised, gamma_j = sqrt(<z~_j, v_j>)):
//   delta_j  = <A z~_j, z~_j> / gamma_j^2
//   v_{j+1}  = A z~_j / gamma_j - (delta_j/gamma_j) v_j - (gamma_j/gamma_{j-1}) v_{j-1}
//   z~_{j+1} = P^{-1} v_{j+1},  gamma_{j+1} = sqrt(<z~_{j+1}, v_{j+1}>)
//   a0 = c_j delta_j - c_{j-1} s_j gamma_j,  a1 = sqrt(a0^2 + gamma_{j+1}^2),
//   a2 = s_j delta_j + c_{j-1} c_j gamma_j,  a3 = s_{j-1} gamma_j,
//   c_{j+1} = a0/a1, s_{j+1} = gamma_{j+1}/a1,
//   w_{j+1} = (z~_j/gamma_j - a3 w_{j-1} - a2 w_j)/a1,  x += c_{j+1} eta w_{j+1},  eta <- -s_{j+1} eta.
// Every reduction is two-level and deterministic: fixed blocks write partial
// sums, one warp per right-hand side adds them in a fixed order.
#include "aao_internal.cuh"
#include "minres_scalars.cuh"

namespace aao {

namespace {
constexpr int VNT = 256;
constexpr int DOT_BLOCKS = 608;  // most partial sums per right-hand side (4 per SM)
constexpr int DOT_PER_BLOCK = 4 * VNT;  // fewest elements per block: small vectors take fewer blocks

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block bx of nbx blocks: the partial sum of a_i c_i over i = bx*VNT + t + k*nbx*VNT
// (fixed assignment, so the partials do not depend on anything but nbx).
__device__ __forceinline__ void dot_body(const double* __restrict__ a, const double* __restrict__ c,
                                         double* __restrict__ out, long long len, int bx, int nbx) {
  double acc = 0.0;
#pragma unroll 4
  for (long long i = (long long)bx * VNT + threadIdx.x; i < len; i += (long long)nbx * VNT)
    acc = fma(a[i], c[i], acc);
  __shared__ double red[VNT / 32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = (threadIdx.x < VNT / 32) ? red[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) *out = t;
  }
}

__global__ void __launch_bounds__(VNT) k_dot(const double* __restrict__ a, const double* __restrict__ c,
                                             double* __restrict__ partial, long long len) {
  const long long rb = (long long)blockIdx.y * len;
  dot_body(a + rb, c + rb, partial + (long long)blockIdx.y * gridDim.x + blockIdx.x, len, blockIdx.x, gridDim.x);
}

// Three dot products in one pass (the initialisation's <z, v>, <b, b>, <v, v>): each
// running sum takes the same elements in the same order as dot_body, and each block
// reduction is dot_body's, so every partial is bit for bit that of a separate k_dot.
__global__ void __launch_bounds__(VNT) k_dot3(const double* __restrict__ a1, const double* __restrict__ c1,
                                              const double* __restrict__ a2, const double* __restrict__ c2,
                                              const double* __restrict__ a3, const double* __restrict__ c3,
                                              double* __restrict__ p1, double* __restrict__ p2,
                                              double* __restrict__ p3, long long len) {
  const long long rb = (long long)blockIdx.y * len;
  const int bx = blockIdx.x, nbx = gridDim.x;
  double s1 = 0.0, s2 = 0.0, s3 = 0.0;
#pragma unroll 4
  for (long long i = rb + (long long)bx * VNT + threadIdx.x; i < rb + len; i += (long long)nbx * VNT) {
    s1 = fma(a1[i], c1[i], s1);
    s2 = fma(a2[i], c2[i], s2);
    s3 = fma(a3[i], c3[i], s3);
  }
  __shared__ double red[3][VNT / 32];
  s1 = warp_sum(s1);
  s2 = warp_sum(s2);
  s3 = warp_sum(s3);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = s1;
    red[1][threadIdx.x >> 5] = s2;
    red[2][threadIdx.x >> 5] = s3;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const long long o = (long long)blockIdx.y * nbx + bx;
    double* outs[3] = {p1, p2, p3};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double t = (threadIdx.x < VNT / 32) ? red[k][threadIdx.x] : 0.0;
      t = warp_sum(t);
      if (threadIdx.x == 0) outs[k][o] = t;
    }
  }
}

// with a MINRES scalar step on the partials in the tail (minres_scalars.cuh); 8 resident
// blocks per SM, the register budget of k_dot
__global__ void __launch_bounds__(VNT, 8) k_dot_tail(const double* __restrict__ a, const double* __restrict__ c,
                                                  double* __restrict__ partial, long long len, ScalarTail tl) {
  const long long rb = (long long)blockIdx.y * len;
  double* pr = partial + (long long)blockIdx.y * gridDim.x;
  dot_body(a + rb, c + rb, pr + blockIdx.x, len, blockIdx.x, gridDim.x);
  scalar_tail(tl, blockIdx.y, pr, gridDim.x, gridDim.x);
}

__device__ __forceinline__ void vupdate_body(const double* __restrict__ T, const double* __restrict__ v,
                                             double* __restrict__ vprev, const MinresScalars& S, long long len,
                                             int bx, int nbx) {
  const bool dn = S.done != 0;
  const double c0 = S.cv[0], c1 = S.cv[1], c2 = S.cv[2];
#pragma unroll 4
  for (long long k = (long long)bx * VNT + threadIdx.x; k < len; k += (long long)nbx * VNT)
    vprev[k] = dn ? 0.0 : fma(c0, T[k], fma(c1, v[k], c2 * vprev[k]));
}

__global__ void __launch_bounds__(VNT) k_vupdate(const double* __restrict__ T, const double* __restrict__ v,
                                                 double* __restrict__ vprev, const MinresScalars* __restrict__ sc,
                                                 long long len) {
  const long long rb = (long long)blockIdx.y * len;
  vupdate_body(T + rb, v + rb, vprev + rb, sc[blockIdx.y], len, blockIdx.x, gridDim.x);
}

__device__ __forceinline__ void wxupdate_run(const double* __restrict__ z, double* __restrict__ wprev,
                                             const double* __restrict__ w, double* __restrict__ x,
                                             const MinresScalars* __restrict__ sc, long long len) {
  const MinresScalars& S = sc[blockIdx.y];
  if (!S.done) {
    const long long rb = (long long)blockIdx.y * len;
    const double c0 = S.cw[0], c1 = S.cw[1], c2 = S.cw[2], c3 = S.cw[3];
#pragma unroll 4
    for (long long i = (long long)blockIdx.x * VNT + threadIdx.x; i < len; i += (long long)gridDim.x * VNT) {
      const long long k = rb + i;
      const double wn = fma(c0, z[k], fma(c1, wprev[k], c2 * w[k]));
      wprev[k] = wn;
      x[k] = fma(c3, wn, x[k]);
    }
  }
}

__global__ void __launch_bounds__(VNT) k_wxupdate(const double* __restrict__ z, double* __restrict__ wprev,
                                                  const double* __restrict__ w, double* __restrict__ x,
                                                  const MinresScalars* __restrict__ sc, long long len) {
  wxupdate_run(z, wprev, w, x, sc, len);
}

// with step 4 (the recurrence-estimate stop test, no partial sums) in the tail
__global__ void __launch_bounds__(VNT, 8) k_wxupdate_tail(const double* __restrict__ z, double* __restrict__ wprev,
                                                       const double* __restrict__ w, double* __restrict__ x,
                                                       const MinresScalars* __restrict__ sc, long long len,
                                                       ScalarTail tl) {
  wxupdate_run(z, wprev, w, x, sc, len);
  scalar_tail(tl, blockIdx.y, nullptr, 0, gridDim.x);
}

__global__ void k_set_params(double* prm, double rtol, int maxit) {
  prm[0] = rtol;
  prm[1] = (double)maxit;
}

__global__ void __launch_bounds__(VNT) k_sub(const double* __restrict__ a, const double* __restrict__ b,
                                             double* __restrict__ y, long long len) {
  for (long long i = (long long)blockIdx.x * VNT + threadIdx.x; i < len; i += (long long)gridDim.x * VNT)
    y[i] = a[i] - b[i];
}

__global__ void __launch_bounds__(VNT) k_cast(const double* __restrict__ in, float* __restrict__ out,
                                              long long len) {
  for (long long i = (long long)blockIdx.x * VNT + threadIdx.x; i < len; i += (long long)gridDim.x * VNT)
    out[i] = (float)in[i];
}

__global__ void __launch_bounds__(VNT) k_uncast(const float* __restrict__ in, double* __restrict__ out,
                                                long long len) {
  for (long long i = (long long)blockIdx.x * VNT + threadIdx.x; i < len; i += (long long)gridDim.x * VNT)
    out[i] = (double)in[i];
}

__global__ void __launch_bounds__(VNT) k_axpy(double a, const double* __restrict__ x,
                                              double* __restrict__ y, long long len) {
  for (long long i = (long long)blockIdx.x * VNT + threadIdx.x; i < len; i += (long long)gridDim.x * VNT)
    y[i] = fma(a, x[i], y[i]);
}

__global__ void k_scalars(int step, MinresScalars* sc, const double* __restrict__ p1, int nb1,
                          const double* __restrict__ p2, int nb2, const double* __restrict__ p3,
                          int nb3, double rtol, int maxit, const double* __restrict__ prm) {
  const int r = blockIdx.x;
  scalars_body<false>(step, sc[r], p1 + (long long)r * nb1, nb1, p2 + (long long)r * nb2, nb2,
               p3 + (long long)r * nb3, nb3, rtol, maxit, prm);
}

// relres[r] = sqrt(sum r^2 / sum b^2) (absolute norm if b = 0)
__global__ void k_relres(const double* __restrict__ p1, int nb1, const double* __restrict__ p2, int nb2,
                         double* __restrict__ relres) {
  const int r = blockIdx.x;
  const double s1 = sum_partials<false>(p1 + (long long)r * nb1, nb1);
  const double s2 = sum_partials<false>(p2 + (long long)r * nb2, nb2);
  if (threadIdx.x == 0) relres[r] = (s2 > 0.0) ? sqrt(s1 / s2) : sqrt(s1);
}

// Device-side loop control for the graph-captured solve (loop_cond_body).
__global__ void k_loop_cond(cudaGraphConditionalHandle hw, const MinresScalars* __restrict__ sc, int nrhs,
                            int* trips, int trip_limit, int count, const double* __restrict__ prm) {
  if (threadIdx.x != 0) return;
  loop_cond_body<false>(hw, sc, nrhs, trips, trip_limit, count, prm);
}

// ---- grouped launches (serving): see GroupRound ----
__global__ void __launch_bounds__(VNT) k_g_vupdate(const GroupRound* __restrict__ g) {
  const int r = group_find(g->vu, g->count, blockIdx.x);
  const GroupProblem& P = g->p[r];
  if (P.sc->done) return;
  vupdate_body(P.T, P.v, P.vp, *P.sc, (long long)P.n * P.m, blockIdx.x - g->vu[r], P.nb_vu);
}

// <z~_{j+1}, v_{j+1}> of every problem
__global__ void __launch_bounds__(VNT) k_g_dot(const GroupRound* __restrict__ g) {
  const int r = group_find(g->dot, g->count, blockIdx.x);
  const GroupProblem& P = g->p[r];
  if (P.sc->done) return;
  const int lb = blockIdx.x - g->dot[r];
  dot_body(P.zn, P.vp, P.partial + lb, (long long)P.n * P.m, lb, P.nb_dot);
}

// steps 1 (delta; the operator's partials), 2 (gamma + Givens; the dot's partials) and
// 3 (true-residual stop test; the w/x update's partials), one warp per problem; step 3
// also publishes each problem's done flag
__global__ void k_g_scalars(int step, const GroupRound* __restrict__ g) {
  const int r = blockIdx.x;
  const GroupProblem& P = g->p[r];
  const int nb = step == 1 ? g->yt[r + 1] - g->yt[r] : step == 2 ? P.nb_dot : g->wx[r + 1] - g->wx[r];
  scalars_body<false>(step, *P.sc, P.partial, nb, nullptr, 0, nullptr, 0, 0.0, 0, nullptr);
  if (step == 3 && threadIdx.x == 0) g->flags[r] = P.sc->done;
}

inline dim3 vgrid(const Plan& P, int nrhs) {
  const long long len = (long long)P.n * P.m;
  long long b = (len + VNT - 1) / VNT;
  if (b > 152 * 8) b = 152 * 8;
  return dim3((unsigned)b, nrhs);
}

}  // namespace

int dot_blocks_for(long long len) {
  const long long b = (len + DOT_PER_BLOCK - 1) / DOT_PER_BLOCK;
  return (int)(b < 1 ? 1 : (b > DOT_BLOCKS ? DOT_BLOCKS : b));
}

int dot_blocks_per_rhs(const Plan& P) { return dot_blocks_for((long long)P.n * P.m); }

int group_vu_blocks(int n, int m) {
  const long long b = ((long long)n * m + 4 * VNT - 1) / (4 * VNT);
  return (int)(b < 1 ? 1 : (b > 152 * 8 ? 152 * 8 : b));
}

cudaError_t launch_group_vupdate(const GroupRound* d_round, int total_blocks, cudaStream_t s) {
  k_g_vupdate<<<total_blocks, VNT, 0, s>>>(d_round);
  return cudaGetLastError();
}

cudaError_t launch_group_dot(const GroupRound* d_round, int total_blocks, cudaStream_t s) {
  k_g_dot<<<total_blocks, VNT, 0, s>>>(d_round);
  return cudaGetLastError();
}

cudaError_t launch_group_scalars(int step, const GroupRound* d_round, int count, cudaStream_t s) {
  k_g_scalars<<<count, 32, 0, s>>>(step, d_round);
  return cudaGetLastError();
}

cudaError_t launch_dot(const Plan& P, const double* a, const double* c, double* partial, int nrhs,
                       cudaStream_t s, uint64_t* nl, const ScalarTail* tail) {
  if (nl) ++*nl;
  const dim3 g(dot_blocks_per_rhs(P), nrhs);
  if (tail) k_dot_tail<<<g, VNT, 0, s>>>(a, c, partial, (long long)P.n * P.m, *tail);
  else k_dot<<<g, VNT, 0, s>>>(a, c, partial, (long long)P.n * P.m);
  return cudaGetLastError();
}

cudaError_t launch_dot3(const Plan& P, const double* a1, const double* c1, const double* a2, const double* c2,
                        const double* a3, const double* c3, double* p1, double* p2, double* p3, int nrhs,
                        cudaStream_t s, uint64_t* nl) {
  if (nl) ++*nl;
  k_dot3<<<dim3(dot_blocks_per_rhs(P), nrhs), VNT, 0, s>>>(a1, c1, a2, c2, a3, c3, p1, p2, p3,
                                                           (long long)P.n * P.m);
  return cudaGetLastError();
}

// y[i] = a deterministic pseudo-random value in (-1, 1) (an integer hash of i): timing
// input for the autotuner, whose kernels take shortcuts on zeros (the integer
// conversions of the FP32 and double-float kernels return early for them).
__global__ void __launch_bounds__(VNT) k_fill_test(double* __restrict__ y, long long len) {
  for (long long i = (long long)blockIdx.x * VNT + threadIdx.x; i < len; i += (long long)gridDim.x * VNT) {
    unsigned long long z = (unsigned long long)i * 0x9E3779B97F4A7C15ull;
    z ^= z >> 29;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 32;
    y[i] = (double)(long long)(z >> 11) * 0x1.0p-52 - 1.0;
  }
}

cudaError_t launch_fill_test(double* y, size_t count, cudaStream_t s) {
  long long nb = ((long long)count + VNT - 1) / VNT;
  if (nb > 152 * 8) nb = 152 * 8;
  if (nb < 1) nb = 1;
  k_fill_test<<<(unsigned)nb, VNT, 0, s>>>(y, (long long)count);
  return cudaGetLastError();
}

cudaError_t launch_vupdate(const Plan& P, const double* T, const double* v, double* vprev_out,
                           const MinresScalars* sc, int nrhs, cudaStream_t s, uint64_t* nl) {
  if (nl) ++*nl;
  k_vupdate<<<vgrid(P, nrhs), VNT, 0, s>>>(T, v, vprev_out, sc, (long long)P.n * P.m);
  return cudaGetLastError();
}

cudaError_t launch_wxupdate(const Plan& P, const double* z, double* wprev_out, const double* w,
                            double* x, const MinresScalars* sc, int nrhs, cudaStream_t s,
                            uint64_t* nl, const ScalarTail* tail) {
  if (nl) ++*nl;
  if (tail) k_wxupdate_tail<<<vgrid(P, nrhs), VNT, 0, s>>>(z, wprev_out, w, x, sc, (long long)P.n * P.m, *tail);
  else k_wxupdate<<<vgrid(P, nrhs), VNT, 0, s>>>(z, wprev_out, w, x, sc, (long long)P.n * P.m);
  return cudaGetLastError();
}

cudaError_t launch_sub(const Plan& P, const double* a, const double* b, double* y, int nrhs,
                       cudaStream_t s, uint64_t* nl) {
  if (nl) ++*nl;
  const long long len = (long long)nrhs * P.n * P.m;
  long long nb = (len + VNT - 1) / VNT;
  if (nb > 152 * 8) nb = 152 * 8;
  k_sub<<<(unsigned)nb, VNT, 0, s>>>(a, b, y, len);
  return cudaGetLastError();
}

cudaError_t launch_loop_cond(cudaGraphConditionalHandle hw, const MinresScalars* sc, int nrhs, int* trips,
                             int trip_limit, int count, cudaStream_t s, uint64_t* nl, const double* prm) {
  if (nl) ++*nl;
  k_loop_cond<<<1, 32, 0, s>>>(hw, sc, nrhs, trips, trip_limit, count, prm);
  return cudaGetLastError();
}

cudaError_t launch_set_params(double* prm, double rtol, int maxit, cudaStream_t s, uint64_t* nl) {
  if (nl) ++*nl;
  k_set_params<<<1, 1, 0, s>>>(prm, rtol, maxit);
  return cudaGetLastError();
}

cudaError_t launch_relres(const double* p1, int nb1, const double* p2, int nb2, double* relres,
                          int nrhs, cudaStream_t s, uint64_t* nl) {
  if (nl) ++*nl;
  k_relres<<<nrhs, 32, 0, s>>>(p1, nb1, p2, nb2, relres);
  return cudaGetLastError();
}

cudaError_t launch_cast(const double* in, float* out, size_t count, cudaStream_t s, uint64_t* nl) {
  if (nl) ++*nl;
  long long nb = ((long long)count + VNT - 1) / VNT;
  if (nb > 152 * 8) nb = 152 * 8;
  if (nb < 1) nb = 1;
  k_cast<<<(unsigned)nb, VNT, 0, s>>>(in, out, (long long)count);
  return cudaGetLastError();
}

cudaError_t launch_uncast(const float* in, double* out, size_t count, cudaStream_t s, uint64_t* nl) {
  if (nl) ++*nl;
  long long nb = ((long long)count + VNT - 1) / VNT;
  if (nb > 152 * 8) nb = 152 * 8;
  if (nb < 1) nb = 1;
  k_uncast<<<(unsigned)nb, VNT, 0, s>>>(in, out, (long long)count);
  return cudaGetLastError();
}

cudaError_t launch_axpy(double a, const double* x, double* y, size_t count, cudaStream_t s,
                        uint64_t* nl) {
  if (nl) ++*nl;
  long long nb = ((long long)count + VNT - 1) / VNT;
  if (nb > 152 * 8) nb = 152 * 8;
  if (nb < 1) nb = 1;
  k_axpy<<<(unsigned)nb, VNT, 0, s>>>(a, x, y, (long long)count);
  return cudaGetLastError();
}

cudaError_t launch_scalars(int step, MinresScalars* sc, const double* partial, int nb,
                           const double* partial2, int nb2, const double* partial3, int nb3,
                           int nrhs, double rtol, int maxit, cudaStream_t s, uint64_t* nl,
                           const double* prm) {
  if (nl) ++*nl;
  k_scalars<<<nrhs, 32, 0, s>>>(step, sc, partial, nb, partial2, nb2, partial3, nb3, rtol, maxit, prm);
  return cudaGetLastError();
}

}  // namespace aao
