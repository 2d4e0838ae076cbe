// Spectral factors of the preconditioner (built once by aao_create).
//
// For spatial mode s with L-eigenvalue Lambda_s = 1 + e_s, e_s = (c2 tau^2/2) sum_axes mu(i_axis),
// mu(i) = (4/h^2) sin^2((i+1) pi h/2), and time frequency k:
//   Sigma_{k,s} = Lambda_s lambda_{1,k} + lambda_{2,k}
//              = Lambda_s (1 + a^2 theta^{2k}) - 2 a theta^k,  a = alpha^{1/n}, theta = exp(2 pi i/n)
// (eq. (calphaprediagform); Section 2.3), G_{k,s} = Sigma^{-1/2} on the principal
// branch (eq. (calphasqrtdiagform)); Lemma calphanonsinglm keeps Sigma off (-inf, 0].
// Sigma is evaluated as (1 - a theta^k)^2 + e_s (1 + a^2 theta^{2k}) (the same value
// expanded): the literal form cancels when Lambda_s ~ 1 and a ~ 1 (low modes, large n)
// and would lose up to ~1e-11 relative accuracy.  The per-k terms
// w2_k = (1 - a theta^k)^2 and q_k = 1 + a^2 theta^{2k} come from the host in long double.
// Stored per pair of modes (a, b) = (2p, 2p+1) as A = (G_a + G_b)/(2n),
// B = (G_a - G_b)/(2n) for k = 0..n/2, layout [k][p][A|B].
#include "aao_internal.cuh"

namespace aao {

namespace {

// principal square root, cancellation-free form: for Re z >= 0,
// sqrt z = t + i Im(z)/(2t) with t = sqrt((|z| + Re z)/2); otherwise
// sqrt z = |Im z|/(2t) + i sign(Im z) t with t = sqrt((|z| - Re z)/2).
__device__ __forceinline__ double2 csqrt_principal(double2 z) {
  const double r = hypot(z.x, z.y);
  double2 s;
  if (z.x >= 0.0) {
    const double t = sqrt(0.5 * (r + z.x));
    s.x = t;
    s.y = (t > 0.0) ? z.y / (2.0 * t) : 0.0;
  } else {
    const double t = sqrt(0.5 * (r - z.x));
    s.x = fabs(z.y) / (2.0 * t);
    s.y = copysign(t, z.y);
  }
  return s;
}

struct SpecArgs {
  int d, N, n, m, npairs;
  double coefT;   // c2 tau^2 / 2
  double inv2n;   // 1/(2n)
};

__global__ void __launch_bounds__(256) k_spectral(SpecArgs a, const double* __restrict__ mu,
                                                  const double2* __restrict__ wq,
                                                  double2* __restrict__ ab64, float2* __restrict__ ab32,
                                                  double* __restrict__ mm) {
  const long long total = (long long)(a.n / 2 + 1) * a.npairs;
  const long long idx = (long long)blockIdx.x * 256 + threadIdx.x;
  double smin = 1e300, smax = 0.0;
  if (idx < total) {
    const int k = (int)(idx / a.npairs);
    const int p = (int)(idx % a.npairs);
    const double2 w2 = wq[2 * k];      // (1 - a theta^k)^2
    const double2 qk = wq[2 * k + 1];  // 1 + a^2 theta^{2k}
    double2 G[2];
    for (int e = 0; e < 2; ++e) {
      const int s = 2 * p + e;
      if (s >= a.m) { G[e] = make_double2(0.0, 0.0); continue; }
      int ix = s % a.N, rest = s / a.N;
      double musum = mu[ix];
      if (a.d >= 2) { musum += mu[rest % a.N]; rest /= a.N; }
      if (a.d >= 3) { musum += mu[rest]; }
      const double lm1 = a.coefT * musum;  // Lambda_s - 1
      double2 sg;
      sg.x = fma(lm1, qk.x, w2.x);
      sg.y = fma(lm1, qk.y, w2.y);
      const double mag = hypot(sg.x, sg.y);
      smin = fmin(smin, mag);
      smax = fmax(smax, mag);
      const double2 sq = csqrt_principal(sg);
      const double q = sq.x * sq.x + sq.y * sq.y;
      G[e] = make_double2(sq.x / q, -sq.y / q);   // 1 / sqrt(Sigma)
    }
    const double2 A = make_double2((G[0].x + G[1].x) * a.inv2n, (G[0].y + G[1].y) * a.inv2n);
    const double2 B = make_double2((G[0].x - G[1].x) * a.inv2n, (G[0].y - G[1].y) * a.inv2n);
    const long long o = idx * 2;
    ab64[o] = A;
    ab64[o + 1] = B;
    if (ab32) {
      ab32[o] = make_float2((float)A.x, (float)A.y);
      ab32[o + 1] = make_float2((float)B.x, (float)B.y);
    }
  }
  // block min / max of |Sigma|
  __shared__ double rmin[256], rmax[256];
  rmin[threadIdx.x] = smin;
  rmax[threadIdx.x] = smax;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      rmin[threadIdx.x] = fmin(rmin[threadIdx.x], rmin[threadIdx.x + o]);
      rmax[threadIdx.x] = fmax(rmax[threadIdx.x], rmax[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    mm[2 * blockIdx.x] = rmin[0];
    mm[2 * blockIdx.x + 1] = rmax[0];
  }
}

__global__ void k_split_df(const double2* __restrict__ in, dfl2* __restrict__ out, long long count) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const double2 v = in[i];
    out[i] = dfl2{dfl(v.x), dfl(v.y)};
  }
}

}  // namespace

cudaError_t launch_split_df(const double2* in, dfl2* out, size_t count, cudaStream_t s, uint64_t* nl) {
  if (nl) ++*nl;
  long long nb = ((long long)count + 255) / 256;
  if (nb > 152 * 8) nb = 152 * 8;
  if (nb < 1) nb = 1;
  k_split_df<<<(unsigned)nb, 256, 0, s>>>(in, out, (long long)count);
  return cudaGetLastError();
}

cudaError_t launch_spectral_table(const Plan& P, const double* mu1d, const double2* wq,
                                  double2* ab64, float2* ab32, double* mm, int* nblocks,
                                  cudaStream_t s, uint64_t* nl) {
  if (nl) ++*nl;
  SpecArgs a;
  a.d = P.d;
  a.N = P.N;
  a.n = P.n;
  a.m = P.m;
  a.npairs = P.npairs;
  a.coefT = 0.5 * P.c2 * P.tau * P.tau;
  a.inv2n = 1.0 / (2.0 * P.n);
  const long long total = (long long)(P.n / 2 + 1) * P.npairs;
  const int nb = (int)((total + 255) / 256);
  if (nblocks) *nblocks = nb;
  k_spectral<<<nb, 256, 0, s>>>(a, mu1d, wq, ab64, ab32, mm);
  return cudaGetLastError();
}

}  // namespace aao
