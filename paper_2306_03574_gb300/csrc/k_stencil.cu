// Y T v as a stencil x time-band kernel (Section 2.3, first paragraph: T is
// sparse, Y only reverses the time levels), and the right-hand side b = Y f of
// eq. (main_matrix).
//
// (T v)_i = L v_i - 2 v_{i-1} + L v_{i-2}, v_{-1} = v_{-2} = 0, L = I - coef*(-h^2 Delta_h),
// L w(s) = (1 + 2d coef) w(s) - coef * sum_{neighbours s'} w(s'), Dirichlet zeros outside.
// One thread owns one spatial point s and a run of CH time levels; it keeps
// L v_{i-1}, L v_{i-2} and v_{i-1} in registers (two extra halo levels at the
// start of its run) and writes (Y T v) at time slot n-1-i.  Optional fused
// reductions: sum (YTv)*w  (the MINRES delta), or sum (w - YTv)^2 (the true
// residual, with w = b).
#include "aao_internal.cuh"
#include "minres_scalars.cuh"

namespace aao {

namespace {

constexpr int YT_NT = YT_THREADS;
constexpr int YT_CH = YT_CH_STD;  // the grouped (serving) launches
// Resident blocks per SM of the stencil kernels with a fused scalar step in their tail
// (minres_scalars.cuh): the register budgets of the same kernels without it, so that the
// step's registers (spilled if need be; it runs once per right-hand side) do not lower
// the main loop's occupancy.
constexpr int yt_min_blocks(int D, int MODE) { return MODE == 2 && D < 3 ? 6 : 8; }
constexpr int ytv_min_blocks(int D, int MODE) {
  return D == 1 ? (MODE == 2 ? 6 : 8) : D == 2 ? (MODE == 2 ? 4 : 6) : 5;
}

struct YtArgs {
  int N, n, m;
  int ch;  // time levels per thread run (Plan::yt_ch)
  double coef, diag;
};

template <int D>
__device__ __forceinline__ double apply_L(const double* __restrict__ v, int s, int ix, int iy, int iz,
                                          const YtArgs& a) {
  const int N = a.N;
  double sum = (ix > 0 ? v[s - 1] : 0.0) + (ix < N - 1 ? v[s + 1] : 0.0);
  if (D >= 2) sum += (iy > 0 ? v[s - N] : 0.0) + (iy < N - 1 ? v[s + N] : 0.0);
  if (D >= 3) sum += (iz > 0 ? v[s - N * N] : 0.0) + (iz < N - 1 ? v[s + N * N] : 0.0);
  return fma(-a.coef, sum, a.diag * v[s]);
}

template <int NT = YT_NT>
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[NT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = (l < NT / 32) ? red[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;  // valid in thread 0
}

template <int D, int MODE>
__device__ __forceinline__ void yt_run(const double* __restrict__ x, double* __restrict__ y,
                                       const double* __restrict__ w, double* __restrict__ partial,
                                       const YtArgs& a) {
  const int s = blockIdx.x * YT_NT + threadIdx.x;
  const int n = a.n, m = a.m, N = a.N;
  const int i0 = blockIdx.y * a.ch;
  const int i1 = min(n, i0 + a.ch);
  const long long rb = (long long)blockIdx.z * n * m;
  double acc = 0.0;
  if (s < m) {
    const int ix = s % N;
    const int iy = (D >= 2) ? (s / N) % N : 0;
    const int iz = (D >= 3) ? s / (N * N) : 0;
    const double* xr = x + rb;
    double Lv1 = 0.0, Lv2 = 0.0, v1 = 0.0;  // L v_{i-1}, L v_{i-2}, v_{i-1}
    for (int i = max(0, i0 - 2); i < i1; ++i) {
      const double* vi = xr + (long long)i * m;
      const double Lv = apply_L<D>(vi, s, ix, iy, iz, a);
      if (i >= i0) {
        const double o = fma(-2.0, v1, Lv + Lv2);
        const long long idx = rb + (long long)(n - 1 - i) * m + s;
        if (MODE != 2) y[idx] = o;
        if (MODE == 1) acc = fma(o, w[idx], acc);
        if (MODE == 2) {
          const double r = w[idx] - o;
          acc = fma(r, r, acc);
        }
      }
      Lv2 = Lv1;
      Lv1 = Lv;
      v1 = vi[s];
    }
  }
  if (MODE != 0) {
    const double t = block_sum(acc);
    const int nb = gridDim.x * gridDim.y;
    if (threadIdx.x == 0) partial[(long long)blockIdx.z * nb + (long long)blockIdx.y * gridDim.x + blockIdx.x] = t;
  }
}

template <int D, int MODE>
__global__ void __launch_bounds__(YT_NT) k_yt(const double* __restrict__ x, double* __restrict__ y,
                                              const double* __restrict__ w, double* __restrict__ partial,
                                              YtArgs a) {
  yt_run<D, MODE>(x, y, w, partial, a);
}

// The same with a MINRES scalar step on the partials in the tail (modes 1, 2).  A kernel
// of its own so that the step's registers do not change the budget of k_yt.
template <int D, int MODE>
__global__ void __launch_bounds__(YT_NT, yt_min_blocks(D, MODE))
    k_yt_tail(const double* __restrict__ x, double* __restrict__ y, const double* __restrict__ w,
              double* __restrict__ partial, YtArgs a, ScalarTail tl) {
  yt_run<D, MODE>(x, y, w, partial, a);
  const int nb = gridDim.x * gridDim.y;
  scalar_tail(tl, blockIdx.z, partial + (long long)blockIdx.z * nb, nb, nb);
}

// The same operator in the DST basis: with U = S (x)..(x) S orthogonal and symmetric,
// (I (x) U) Y T (I (x) U) is Y T with L replaced by diag(Lambda), so
// (Y T^ v)_{n-1-i} = Lambda_s (v_i + v_{i-2}) - 2 v_{i-1} pointwise in s.  Modes as k_yt,
// plus mode 3: the residual vector y = w - Y T^ v written out with the sum of its squares
// (the refinement loop's r = b - A x and ||r||^2 in one pass).
// Block (bx, by) of one right-hand side (x, y, w point at it): spatial tile bx, time run
// by; its partial sum (modes 1-3) goes to *part.
template <int MODE>
__device__ __forceinline__ void ythat_body(const double* __restrict__ x, double* __restrict__ y,
                                           const double* __restrict__ w, double* __restrict__ part,
                                           const double* __restrict__ lam, int n, int m, int bx, int by,
                                           int ch) {
  const int s = bx * YT_NT + threadIdx.x;
  const int i0 = by * ch;
  const int i1 = min(n, i0 + ch);
  double acc = 0.0;
  if (s < m) {
    const double ls = lam[s];
    const double* xr = x + s;
    double x1 = 0.0, x2 = 0.0;  // v_{i-1}, v_{i-2}
    for (int i = max(0, i0 - 2); i < i1; ++i) {
      const double xi = xr[(long long)i * m];
      if (i >= i0) {
        const double o = fma(-2.0, x1, ls * (xi + x2));
        const long long idx = (long long)(n - 1 - i) * m + s;
        if (MODE == 0 || MODE == 1) y[idx] = o;
        if (MODE == 1) acc = fma(o, w[idx], acc);
        if (MODE >= 2) {
          const double r = w[idx] - o;
          if (MODE == 3) y[idx] = r;
          acc = fma(r, r, acc);
        }
      }
      x2 = x1;
      x1 = xi;
    }
  }
  if (MODE != 0) {
    const double t = block_sum(acc);
    if (threadIdx.x == 0) *part = t;
  }
}

template <int MODE>
__device__ __forceinline__ void ythat_run(const double* __restrict__ x, double* __restrict__ y,
                                          const double* __restrict__ w, double* __restrict__ partial,
                                          const double* __restrict__ lam, const YtArgs& a) {
  const long long rb = (long long)blockIdx.z * a.n * a.m;
  const int nb = gridDim.x * gridDim.y;
  double* part = MODE != 0 ? partial + (long long)blockIdx.z * nb + (long long)blockIdx.y * gridDim.x + blockIdx.x
                           : nullptr;
  ythat_body<MODE>(x + rb, y ? y + rb : nullptr, w ? w + rb : nullptr, part, lam, a.n, a.m, blockIdx.x,
                   blockIdx.y, a.ch);
}

template <int MODE>
__global__ void __launch_bounds__(YT_NT) k_ythat(const double* __restrict__ x, double* __restrict__ y,
                                                 const double* __restrict__ w,
                                                 double* __restrict__ partial,
                                                 const double* __restrict__ lam, YtArgs a) {
  ythat_run<MODE>(x, y, w, partial, lam, a);
}

// with a MINRES scalar step on the partials in the tail (modes 1..3)
template <int MODE>
__global__ void __launch_bounds__(YT_NT, 8)
    k_ythat_tail(const double* __restrict__ x, double* __restrict__ y, const double* __restrict__ w,
                 double* __restrict__ partial, const double* __restrict__ lam, YtArgs a, ScalarTail tl) {
  ythat_run<MODE>(x, y, w, partial, lam, a);
  const int nb = gridDim.x * gridDim.y;
  scalar_tail(tl, blockIdx.z, partial + (long long)blockIdx.z * nb, nb, nb);
}

// One MINRES step's direction and iterate update fused with the true residual, in the
// DST basis (Section 3's stopping test on the system whose operator is pointwise in s):
//   w_{j+1} = c0 z + c1 w_{j-1} + c2 w_j (written over w_{j-1}),   x += c3 w_{j+1},
//   r_{n-1-i} = b_{n-1-i} - (Lambda_s (x_i + x_{i-2}) - 2 x_{i-1}),  partial = sum r^2,
// with (c0..c3) = sc[rhs].cw.  A block owns S consecutive spatial modes and all n time
// levels of them, split into C runs of n/C levels, one thread per mode and run.  A run
// needs the updated x at the two levels before it, which the thread of the previous
// run overwrites in place; every thread therefore recomputes those two values (the
// same operations on the same inputs, so bit for bit the same) before a barrier, and
// only then starts writing.  Converged right-hand sides (sc.done) are left untouched
// and their partial is not written.  Standard shape S = 32, C = 4; small problems
// (fewer blocks than SMs) S = 8, C = 16: more blocks and shorter serial runs.
constexpr int WXR_S = 32;
constexpr int WXR_C = 4;
constexpr int WXR_NT = WXR_S * WXR_C;
constexpr int WXR_S_SMALL = 8;
constexpr int WXR_C_SMALL = 16;

// Block bx of one right-hand side (vectors point at it); partial sum to *part.
template <int WS = WXR_S, int WC = WXR_C>
__device__ __forceinline__ void wx_res_body(const double* __restrict__ z, double* __restrict__ wprev,
                                            const double* __restrict__ w, double* __restrict__ x,
                                            const double* __restrict__ b, const double* __restrict__ lam,
                                            const MinresScalars& S, double* __restrict__ part, int n, int m,
                                            int bx) {
  if (S.done) return;  // uniform over the block
  const int s = bx * WS + (int)(threadIdx.x % WS);
  const int len = n / WC;
  const int i0 = (int)(threadIdx.x / WS) * len;
  const bool on = s < m;
  const double c0 = S.cw[0], c1 = S.cw[1], c2 = S.cw[2], c3 = S.cw[3];
  const long long rb = s;
  const double* zp = z + rb;
  double* wpp = wprev + rb;
  const double* wq = w + rb;
  double* xp = x + rb;
  const double* bp = b + rb + (long long)(n - 1) * m;  // b at time slot n-1-i is bp[-i m]
  double x1 = 0.0, x2 = 0.0;                           // updated x_{i-1}, x_{i-2}
  if (on && i0 > 0) {
    const long long o2 = (long long)(i0 - 2) * m, o1 = o2 + m;
    x2 = fma(c3, fma(c0, zp[o2], fma(c1, wpp[o2], c2 * wq[o2])), xp[o2]);
    x1 = fma(c3, fma(c0, zp[o1], fma(c1, wpp[o1], c2 * wq[o1])), xp[o1]);
  }
  __syncthreads();
  double acc = 0.0;
  if (on) {
    const double ls = lam[s];
#pragma unroll 4
    for (int i = i0; i < i0 + len; ++i) {
      const long long o = (long long)i * m;
      const double wn = fma(c0, zp[o], fma(c1, wpp[o], c2 * wq[o]));
      wpp[o] = wn;
      const double xi = fma(c3, wn, xp[o]);
      xp[o] = xi;
      const double r = fma(-ls, xi + x2, fma(2.0, x1, bp[-o]));
      acc = fma(r, r, acc);
      x2 = x1;
      x1 = xi;
    }
  }
  const double t = block_sum<WS * WC>(acc);
  if (threadIdx.x == 0) *part = t;
}

template <int WS, int WC>
__global__ void __launch_bounds__(WS * WC) k_wx_res(const double* __restrict__ z, double* __restrict__ wprev,
                                                   const double* __restrict__ w, double* __restrict__ x,
                                                   const double* __restrict__ b, const double* __restrict__ lam,
                                                   const MinresScalars* __restrict__ sc,
                                                   double* __restrict__ partial, int n, int m) {
  const long long rb = (long long)blockIdx.y * n * m;
  double* pr = partial + (long long)blockIdx.y * gridDim.x;
  wx_res_body<WS, WC>(z + rb, wprev + rb, w + rb, x + rb, b + rb, lam, sc[blockIdx.y], pr + blockIdx.x, n, m,
                      blockIdx.x);
}

// with the stop test (MINRES scalar step 3) in the tail
template <int WS, int WC>
__global__ void __launch_bounds__(WS * WC, 12) k_wx_res_tail(const double* __restrict__ z, double* __restrict__ wprev,
                                                   const double* __restrict__ w, double* __restrict__ x,
                                                   const double* __restrict__ b, const double* __restrict__ lam,
                                                   const MinresScalars* __restrict__ sc,
                                                   double* __restrict__ partial, int n, int m, ScalarTail tl) {
  const long long rb = (long long)blockIdx.y * n * m;
  double* pr = partial + (long long)blockIdx.y * gridDim.x;
  wx_res_body<WS, WC>(z + rb, wprev + rb, w + rb, x + rb, b + rb, lam, sc[blockIdx.y], pr + blockIdx.x, n, m,
                      blockIdx.x);
  scalar_tail(tl, blockIdx.y, pr, gridDim.x, gridDim.x);
}

// ---- grouped launches (serving): see GroupRound ----
// Y T^ z~_j and its partial dot with z~_j (mode 1) for every problem
__global__ void __launch_bounds__(YT_NT) k_g_ythat(const GroupRound* __restrict__ g) {
  const int r = group_find(g->yt, g->count, blockIdx.x);
  const GroupProblem& P = g->p[r];
  if (P.sc->done) return;
  const int lb = blockIdx.x - g->yt[r];
  const int bx = lb % P.yt_gx, by = lb / P.yt_gx;
  ythat_body<1>(P.z, P.T, P.z, P.partial + lb, P.lam, P.n, P.m, bx, by, YT_CH);
}

// the w/x update fused with the true residual for every problem
__global__ void __launch_bounds__(WXR_NT) k_g_wx_res(const GroupRound* __restrict__ g) {
  const int r = group_find(g->wx, g->count, blockIdx.x);
  const GroupProblem& P = g->p[r];
  const int lb = blockIdx.x - g->wx[r];
  wx_res_body(P.z, P.wp, P.w, P.x, P.b, P.lam, *P.sc, P.partial + lb, P.n, P.m, lb);
}

// Variable coefficient: L_a w(s) = w(s) + cv sum_axes [aR (w(s) - w(s+e)) + aL (w(s) - w(s-e))],
// cv = tau^2/(2h^2), aR/aL the coefficients on the faces right/left of s along the axis
// (face arrays concatenated by axis; axis ax has N+1 faces along ax, N along the others).
struct VarArgs {
  int N, n, m, d;
  int ch;  // time levels per thread run (Plan::yt_ch)
  double cv;
  const double* face;  // d * (N+1) * N^(d-1)
};

// The coefficients on the faces left/right of point s along each axis (constant in time,
// so a thread loads them once for its whole run of time levels).
struct Faces {
  double xl, xr, yl, yr, zl, zr;
};

template <int D>
__device__ __forceinline__ Faces load_faces(int ix, int iy, int iz, const VarArgs& a) {
  const int N = a.N;
  const long long fsz = (long long)(N + 1) * (D == 1 ? 1 : (D == 2 ? N : N * N));
  Faces f{};
  {  // x faces: index (iz*N + iy)*(N+1) + f
    const long long base = ((long long)iz * N + iy) * (N + 1);
    f.xl = a.face[base + ix];
    f.xr = a.face[base + ix + 1];
  }
  if (D >= 2) {  // y faces: index (iz*(N+1) + f)*N + ix
    const double* F = a.face + fsz;
    const long long base = (long long)iz * (N + 1);
    f.yl = F[(base + iy) * N + ix];
    f.yr = F[(base + iy + 1) * N + ix];
  }
  if (D >= 3) {  // z faces: index (f*N + iy)*N + ix
    const double* F = a.face + 2 * fsz;
    f.zl = F[((long long)iz * N + iy) * N + ix];
    f.zr = F[((long long)(iz + 1) * N + iy) * N + ix];
  }
  return f;
}

// L_a w(s) = w(s) + sum_faces g (w(s) - w(neighbour)) with g = cv a per face, the
// neighbour outside the grid 0.  The g are constant in time, so a thread forms them once
// for its run: each application is one difference and one multiply-add per face (the
// FP64 pipe bounds this kernel).  The differences are kept rather than expanding to
// (1 + sum g) w(s) - sum g w(neighbour): with a ~ 10^3 that form cancels three digits.
struct VarStencil {
  double xl, xr, yl, yr, zl, zr;
};

template <int D>
__device__ __forceinline__ VarStencil var_stencil(const Faces& f, double cv) {
  VarStencil g{};
  g.xl = cv * f.xl;
  g.xr = cv * f.xr;
  if (D >= 2) { g.yl = cv * f.yl; g.yr = cv * f.yr; }
  if (D >= 3) { g.zl = cv * f.zl; g.zr = cv * f.zr; }
  return g;
}

template <int D>
__device__ __forceinline__ double apply_La_f(const double* __restrict__ v, int s, int ix, int iy, int iz, int N,
                                             const VarStencil& g) {
  const double c = v[s];
  double acc = c;
  acc = fma(g.xl, c - (ix > 0 ? v[s - 1] : 0.0), acc);
  acc = fma(g.xr, c - (ix < N - 1 ? v[s + 1] : 0.0), acc);
  if (D >= 2) {
    acc = fma(g.yl, c - (iy > 0 ? v[s - N] : 0.0), acc);
    acc = fma(g.yr, c - (iy < N - 1 ? v[s + N] : 0.0), acc);
  }
  if (D >= 3) {
    acc = fma(g.zl, c - (iz > 0 ? v[s - N * N] : 0.0), acc);
    acc = fma(g.zr, c - (iz < N - 1 ? v[s + N * N] : 0.0), acc);
  }
  return acc;
}

template <int D>
__device__ __forceinline__ double apply_La(const double* __restrict__ v, int s, int ix, int iy, int iz,
                                           const VarArgs& a) {
  return apply_La_f<D>(v, s, ix, iy, iz, a.N, var_stencil<D>(load_faces<D>(ix, iy, iz, a), a.cv));
}

template <int D, int MODE>
__device__ __forceinline__ void yt_var_run(const double* __restrict__ x, double* __restrict__ y,
                                           const double* __restrict__ w, double* __restrict__ partial,
                                           const VarArgs& a) {
  const int s = blockIdx.x * YT_NT + threadIdx.x;
  const int n = a.n, m = a.m, N = a.N;
  const int i0 = blockIdx.y * a.ch;
  const int i1 = min(n, i0 + a.ch);
  const long long rb = (long long)blockIdx.z * n * m;
  double acc = 0.0;
  if (s < m) {
    const int ix = s % N;
    const int iy = (D >= 2) ? (s / N) % N : 0;
    const int iz = (D >= 3) ? s / (N * N) : 0;
    const double* xr = x + rb;
    const VarStencil g = var_stencil<D>(load_faces<D>(ix, iy, iz, a), a.cv);
    double Lv1 = 0.0, Lv2 = 0.0, v1 = 0.0;
    for (int i = max(0, i0 - 2); i < i1; ++i) {
      const double* vi = xr + (long long)i * m;
      const double Lv = apply_La_f<D>(vi, s, ix, iy, iz, N, g);
      if (i >= i0) {
        const double o = fma(-2.0, v1, Lv + Lv2);
        const long long idx = rb + (long long)(n - 1 - i) * m + s;
        if (MODE != 2) y[idx] = o;
        if (MODE == 1) acc = fma(o, w[idx], acc);
        if (MODE == 2) {
          const double r = w[idx] - o;
          acc = fma(r, r, acc);
        }
      }
      Lv2 = Lv1;
      Lv1 = Lv;
      v1 = vi[s];
    }
  }
  if (MODE != 0) {
    const double t = block_sum(acc);
    const int nb = gridDim.x * gridDim.y;
    if (threadIdx.x == 0) partial[(long long)blockIdx.z * nb + (long long)blockIdx.y * gridDim.x + blockIdx.x] = t;
  }
}

template <int D, int MODE>
__global__ void __launch_bounds__(YT_NT) k_yt_var(const double* __restrict__ x, double* __restrict__ y,
                                                  const double* __restrict__ w, double* __restrict__ partial,
                                                  VarArgs a) {
  yt_var_run<D, MODE>(x, y, w, partial, a);
}

// with a MINRES scalar step on the partials in the tail (modes 1, 2)
template <int D, int MODE>
__global__ void __launch_bounds__(YT_NT, ytv_min_blocks(D, MODE))
    k_yt_var_tail(const double* __restrict__ x, double* __restrict__ y, const double* __restrict__ w,
                  double* __restrict__ partial, VarArgs a, ScalarTail tl) {
  yt_var_run<D, MODE>(x, y, w, partial, a);
  const int nb = gridDim.x * gridDim.y;
  scalar_tail(tl, blockIdx.z, partial + (long long)blockIdx.z * nb, nb, nb);
}

template <int D>
__global__ void __launch_bounds__(YT_NT) k_rhs_var(const double* __restrict__ f,
                                                   const double* __restrict__ psi0,
                                                   const double* __restrict__ psi1,
                                                   double* __restrict__ b, VarArgs a, double tau) {
  const int s = blockIdx.x * YT_NT + threadIdx.x;
  const int k = blockIdx.y;
  const int n = a.n, m = a.m, N = a.N;
  if (s >= m) return;
  const long long rb = (long long)blockIdx.z * n * m;
  const long long ib = (long long)blockIdx.z * m;
  const double t2 = tau * tau;
  const double fk = f[rb + (long long)k * m + s];
  double v;
  if (k == 0) {
    v = fma(0.5 * t2, fk, fma(tau, psi1[ib + s], psi0[ib + s]));
  } else if (k == 1) {
    const int ix = s % N;
    const int iy = (D >= 2) ? (s / N) % N : 0;
    const int iz = (D >= 3) ? s / (N * N) : 0;
    v = fma(t2, fk, -apply_La<D>(psi0 + ib, s, ix, iy, iz, a));
  } else {
    v = t2 * fk;
  }
  b[rb + (long long)(n - 1 - k) * m + s] = v;
}

// b[n-1-k] = tau^2 f^k for k >= 2; tau^2 f^1 - L psi0; tau^2 f^0/2 + tau psi1 + psi0.
// (levels k0 .. k0 + gridDim.y - 1 of every right-hand side)
template <int D>
__global__ void __launch_bounds__(YT_NT) k_rhs(const double* __restrict__ f,
                                               const double* __restrict__ psi0,
                                               const double* __restrict__ psi1,
                                               double* __restrict__ b, YtArgs a, double tau, int k0) {
  const int s = blockIdx.x * YT_NT + threadIdx.x;
  const int k = k0 + blockIdx.y;
  const int n = a.n, m = a.m, N = a.N;
  if (s >= m) return;
  const long long rb = (long long)blockIdx.z * n * m;
  const long long ib = (long long)blockIdx.z * m;
  const double t2 = tau * tau;
  const double fk = f[rb + (long long)k * m + s];
  double v;
  if (k == 0) {
    v = fma(0.5 * t2, fk, fma(tau, psi1[ib + s], psi0[ib + s]));
  } else if (k == 1) {
    const int ix = s % N;
    const int iy = (D >= 2) ? (s / N) % N : 0;
    const int iz = (D >= 3) ? s / (N * N) : 0;
    v = fma(t2, fk, -apply_L<D>(psi0 + ib, s, ix, iy, iz, a));
  } else {
    v = t2 * fk;
  }
  b[rb + (long long)(n - 1 - k) * m + s] = v;
}

YtArgs make_args(const Plan& P) {
  YtArgs a;
  a.N = P.N;
  a.n = P.n;
  a.m = P.m;
  a.ch = P.yt_ch;
  a.coef = P.coef;
  a.diag = 1.0 + 2.0 * P.d * P.coef;
  return a;
}

}  // namespace

int wxres_blocks_per_rhs(const Plan& P) {
  const int S = P.wx_small ? WXR_S_SMALL : WXR_S;
  return (P.m + S - 1) / S;
}

int group_yt_tiles(int m) { return (m + YT_NT - 1) / YT_NT; }
int group_yt_blocks(int n, int m) { return group_yt_tiles(m) * ((n + YT_CH - 1) / YT_CH); }
int group_wx_blocks(int m) { return (m + WXR_S - 1) / WXR_S; }

cudaError_t launch_group_ythat(const GroupRound* d_round, int total_blocks, cudaStream_t s) {
  k_g_ythat<<<total_blocks, YT_NT, 0, s>>>(d_round);
  return cudaGetLastError();
}

cudaError_t launch_group_wx_res(const GroupRound* d_round, int total_blocks, cudaStream_t s) {
  k_g_wx_res<<<total_blocks, WXR_NT, 0, s>>>(d_round);
  return cudaGetLastError();
}

cudaError_t launch_wx_res(const Plan& P, const double* lam, const double* z, double* wprev_out,
                          const double* w, double* x, const double* b, const MinresScalars* sc,
                          double* partial, int nrhs, cudaStream_t s, uint64_t* nl, int* nb,
                          const ScalarTail* tail) {
  if (nl) ++*nl;
  const dim3 g(wxres_blocks_per_rhs(P), nrhs);
  if (nb) *nb = (int)g.x;
  constexpr int SS = WXR_S_SMALL, CS = WXR_C_SMALL;
  if (P.wx_small && tail)
    k_wx_res_tail<SS, CS><<<g, SS * CS, 0, s>>>(z, wprev_out, w, x, b, lam, sc, partial, P.n, P.m, *tail);
  else if (P.wx_small) k_wx_res<SS, CS><<<g, SS * CS, 0, s>>>(z, wprev_out, w, x, b, lam, sc, partial, P.n, P.m);
  else if (tail) k_wx_res_tail<WXR_S, WXR_C><<<g, WXR_NT, 0, s>>>(z, wprev_out, w, x, b, lam, sc, partial, P.n, P.m,
                                                                 *tail);
  else k_wx_res<WXR_S, WXR_C><<<g, WXR_NT, 0, s>>>(z, wprev_out, w, x, b, lam, sc, partial, P.n, P.m);
  return cudaGetLastError();
}

int yt_blocks_per_rhs(const Plan& P) {
  return ((P.m + YT_NT - 1) / YT_NT) * ((P.n + P.yt_ch - 1) / P.yt_ch);
}

template <int D>
static void yt_dispatch(int mode, dim3 g, cudaStream_t s, const double* x, double* y,
                        const double* w, double* partial, const YtArgs& a, const ScalarTail& tl) {
  if (mode == 0) k_yt<D, 0><<<g, YT_NT, 0, s>>>(x, y, w, partial, a);
  else if (tl.sc && mode == 1) k_yt_tail<D, 1><<<g, YT_NT, 0, s>>>(x, y, w, partial, a, tl);
  else if (tl.sc) k_yt_tail<D, 2><<<g, YT_NT, 0, s>>>(x, y, w, partial, a, tl);
  else if (mode == 1) k_yt<D, 1><<<g, YT_NT, 0, s>>>(x, y, w, partial, a);
  else k_yt<D, 2><<<g, YT_NT, 0, s>>>(x, y, w, partial, a);
}

cudaError_t launch_yt(const Plan& P, const double* x, double* y, const double* w, double* partial,
                      int mode, int nrhs, cudaStream_t s, uint64_t* nl, int* nb, const ScalarTail* tail) {
  if (nl) ++*nl;
  const YtArgs a = make_args(P);
  dim3 g((P.m + YT_NT - 1) / YT_NT, (P.n + P.yt_ch - 1) / P.yt_ch, nrhs);
  if (nb) *nb = (int)(g.x * g.y);
  const ScalarTail tl = tail ? *tail : ScalarTail{};
  switch (P.d) {
    case 1: yt_dispatch<1>(mode, g, s, x, y, w, partial, a, tl); break;
    case 2: yt_dispatch<2>(mode, g, s, x, y, w, partial, a, tl); break;
    case 3: yt_dispatch<3>(mode, g, s, x, y, w, partial, a, tl); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_ythat(const Plan& P, const double* lam, const double* x, double* y, const double* w,
                        double* partial, int mode, int nrhs, cudaStream_t s, uint64_t* nl, int* nb,
                        const ScalarTail* tail) {
  if (nl) ++*nl;
  const YtArgs a = make_args(P);
  dim3 g((P.m + YT_NT - 1) / YT_NT, (P.n + P.yt_ch - 1) / P.yt_ch, nrhs);
  if (nb) *nb = (int)(g.x * g.y);
  const ScalarTail tl = tail ? *tail : ScalarTail{};
  if (mode == 0) k_ythat<0><<<g, YT_NT, 0, s>>>(x, y, w, partial, lam, a);
  else if (tl.sc && mode == 1) k_ythat_tail<1><<<g, YT_NT, 0, s>>>(x, y, w, partial, lam, a, tl);
  else if (tl.sc && mode == 2) k_ythat_tail<2><<<g, YT_NT, 0, s>>>(x, y, w, partial, lam, a, tl);
  else if (tl.sc) k_ythat_tail<3><<<g, YT_NT, 0, s>>>(x, y, w, partial, lam, a, tl);
  else if (mode == 1) k_ythat<1><<<g, YT_NT, 0, s>>>(x, y, w, partial, lam, a);
  else if (mode == 2) k_ythat<2><<<g, YT_NT, 0, s>>>(x, y, w, partial, lam, a);
  else k_ythat<3><<<g, YT_NT, 0, s>>>(x, y, w, partial, lam, a);
  return cudaGetLastError();
}

static VarArgs make_var(const Plan& P, const double* face) {
  VarArgs a;
  a.N = P.N;
  a.n = P.n;
  a.m = P.m;
  a.d = P.d;
  a.ch = P.yt_ch;
  a.cv = P.tau * P.tau / (2.0 * P.h * P.h);
  a.face = face;
  return a;
}

template <int D>
static void ytv_dispatch(int mode, dim3 g, cudaStream_t s, const double* x, double* y,
                         const double* w, double* partial, const VarArgs& a, const ScalarTail& tl) {
  if (mode == 0) k_yt_var<D, 0><<<g, YT_NT, 0, s>>>(x, y, w, partial, a);
  else if (tl.sc && mode == 1) k_yt_var_tail<D, 1><<<g, YT_NT, 0, s>>>(x, y, w, partial, a, tl);
  else if (tl.sc) k_yt_var_tail<D, 2><<<g, YT_NT, 0, s>>>(x, y, w, partial, a, tl);
  else if (mode == 1) k_yt_var<D, 1><<<g, YT_NT, 0, s>>>(x, y, w, partial, a);
  else k_yt_var<D, 2><<<g, YT_NT, 0, s>>>(x, y, w, partial, a);
}

cudaError_t launch_yt_var(const Plan& P, const double* face, const double* x, double* y, const double* w,
                          double* partial, int mode, int nrhs, cudaStream_t s, uint64_t* nl, int* nb,
                          const ScalarTail* tail) {
  if (nl) ++*nl;
  const VarArgs a = make_var(P, face);
  dim3 g((P.m + YT_NT - 1) / YT_NT, (P.n + P.yt_ch - 1) / P.yt_ch, nrhs);
  if (nb) *nb = (int)(g.x * g.y);
  const ScalarTail tl = tail ? *tail : ScalarTail{};
  switch (P.d) {
    case 1: ytv_dispatch<1>(mode, g, s, x, y, w, partial, a, tl); break;
    case 2: ytv_dispatch<2>(mode, g, s, x, y, w, partial, a, tl); break;
    case 3: ytv_dispatch<3>(mode, g, s, x, y, w, partial, a, tl); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_build_rhs_var(const Plan& P, const double* face, const double* f, const double* psi0,
                                 const double* psi1, double* b, int nrhs, cudaStream_t s, uint64_t* nl) {
  if (nl) ++*nl;
  const VarArgs a = make_var(P, face);
  dim3 g((P.m + YT_NT - 1) / YT_NT, P.n, nrhs);
  switch (P.d) {
    case 1: k_rhs_var<1><<<g, YT_NT, 0, s>>>(f, psi0, psi1, b, a, P.tau); break;
    case 2: k_rhs_var<2><<<g, YT_NT, 0, s>>>(f, psi0, psi1, b, a, P.tau); break;
    case 3: k_rhs_var<3><<<g, YT_NT, 0, s>>>(f, psi0, psi1, b, a, P.tau); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_build_rhs(const Plan& P, const double* f, const double* psi0, const double* psi1,
                             double* b, int nrhs, cudaStream_t s, uint64_t* nl) {
  if (nl) ++*nl;
  const YtArgs a = make_args(P);
  dim3 g((P.m + YT_NT - 1) / YT_NT, P.n, nrhs);
  switch (P.d) {
    case 1: k_rhs<1><<<g, YT_NT, 0, s>>>(f, psi0, psi1, b, a, P.tau, 0); break;
    case 2: k_rhs<2><<<g, YT_NT, 0, s>>>(f, psi0, psi1, b, a, P.tau, 0); break;
    case 3: k_rhs<3><<<g, YT_NT, 0, s>>>(f, psi0, psi1, b, a, P.tau, 0); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_build_rhs_levels(const Plan& P, const double* f, const double* psi0, const double* psi1,
                                    double* b, int k0, int cnt, cudaStream_t s, uint64_t* nl) {
  if (nl) ++*nl;
  if (k0 < 0 || cnt < 1 || k0 + cnt > P.n) return cudaErrorInvalidValue;
  const YtArgs a = make_args(P);
  dim3 g((P.m + YT_NT - 1) / YT_NT, cnt, 1);
  switch (P.d) {
    case 1: k_rhs<1><<<g, YT_NT, 0, s>>>(f, psi0, psi1, b, a, P.tau, k0); break;
    case 2: k_rhs<2><<<g, YT_NT, 0, s>>>(f, psi0, psi1, b, a, P.tau, k0); break;
    case 3: k_rhs<3><<<g, YT_NT, 0, s>>>(f, psi0, psi1, b, a, P.tau, k0); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace aao
