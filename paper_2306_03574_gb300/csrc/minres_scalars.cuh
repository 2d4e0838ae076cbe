// The scalar recurrences of preconditioned MINRES (the Lanczos + Givens form written
// out at the top of k_minres.cu) on the device, and the tail that runs one of their
// steps inside the kernel that produced its partial sums.
//
// Every reduction is two-level and deterministic: the blocks of a producer write one
// partial sum each, and one warp per right-hand side adds them in a fixed order.  The
// step can run either as its own one-warp-per-right-hand-side launch (k_scalars) or in
// the producer: each block, after writing its partial, counts itself in with an atomic;
// the last block of a right-hand side to arrive runs the step on the partials with the
// same code and order, so both give the same bits.  A step fused this way removes a
// launch from every MINRES iteration; the last block's fence, atomic and dependent
// partial reads form a serial chain of a few microseconds, about what a kernel node of
// the captured graph costs on GB300, so the fused form is an option (AAO_FUSED_SCALARS)
// rather than the default.  Nothing waits: a block that is not last simply exits.
#pragma once

#include "aao_internal.cuh"

namespace aao {

__device__ __forceinline__ double warp_sum_all(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <bool CG>
__device__ __forceinline__ double ld_partial(const double* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

// deterministic sum of nb partials of right-hand side r by one warp
// (eight independent running sums per lane keep eight loads in flight; fixed order)
template <bool CG>
__device__ __forceinline__ double sum_partials(const double* p, int nb) {
  double t[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  int i = threadIdx.x;
  for (; i + 7 * 32 < nb; i += 8 * 32) {
#pragma unroll
    for (int u = 0; u < 8; ++u) t[u] += ld_partial<CG>(p + i + 32 * u);
  }
  for (; i < nb; i += 32) t[0] += ld_partial<CG>(p + i);
  return warp_sum_all(((t[0] + t[1]) + (t[2] + t[3])) + ((t[4] + t[5]) + (t[6] + t[7])));
}

// One warp: the scalar step of one right-hand side from its partial sums p1 (and, at
// step 0, p2 and p3), in a fixed order.  CG: the partials are read from L2 (they were
// written by other blocks of the running kernel).
template <bool CG>
__device__ __forceinline__ void scalars_body(int step, MinresScalars& S, const double* __restrict__ p1,
                                             int nb1, const double* __restrict__ p2, int nb2,
                                             const double* __restrict__ p3, int nb3, double rtol, int maxit,
                                             const double* __restrict__ prm) {
  const double s1 = sum_partials<CG>(p1, nb1);
  double s2 = 0.0, s3 = 0.0;
  if (step == 0) {
    s2 = sum_partials<CG>(p2, nb2);
    s3 = sum_partials<CG>(p3, nb3);
  }
  if (threadIdx.x != 0) return;
  if (step == 0) {
    // s1 = <z1, v1>, s2 = <b, b>, s3 = <v1, v1>; rtol and maxit from prm when given
    S.rtol = prm ? prm[0] : rtol;
    S.maxit = prm ? (int)prm[1] : maxit;
    S.iters = 0;
    S.status = AAO_OK;
    S.done = 0;
    S.bnorm2 = (s2 > 0.0) ? s2 : 1.0;
    S.relres_true = sqrt(s3 / S.bnorm2);
    S.relres_est = 1.0;
    S.gam_prev = 1.0;
    S.c = S.c_prev = 1.0;
    S.s = S.s_prev = 0.0;
    S.delta = 0.0;
    for (int i = 0; i < 3; ++i) S.cv[i] = 0.0;
    for (int i = 0; i < 4; ++i) S.cw[i] = 0.0;
    if (s1 < 0.0) { S.status = AAO_EBREAKDOWN; S.done = 1; }
    if (s1 == 0.0 || S.relres_true <= S.rtol) S.done = 1;
    S.gam = S.done ? 0.0 : sqrt(s1);
    S.gam1 = S.gam;
    S.eta = S.gam;
    return;
  }
  if (S.done) {
    for (int i = 0; i < 3; ++i) S.cv[i] = 0.0;
    for (int i = 0; i < 4; ++i) S.cw[i] = 0.0;
    return;
  }
  if (step == 1) {
    const double g = S.gam;
    S.delta = s1 / (g * g);
    S.cv[0] = 1.0 / g;
    S.cv[1] = -S.delta / g;
    S.cv[2] = -g / S.gam_prev;
  } else if (step == 2) {
    if (s1 < 0.0) {
      S.status = AAO_EBREAKDOWN;
      S.done = 1;
      for (int i = 0; i < 4; ++i) S.cw[i] = 0.0;
      return;
    }
    const double gn = sqrt(s1);
    const double g = S.gam, dl = S.delta;
    const double a0 = S.c * dl - S.c_prev * S.s * g;
    const double a1 = sqrt(a0 * a0 + gn * gn);
    const double a2 = S.s * dl + S.c_prev * S.c * g;
    const double a3 = S.s_prev * g;
    if (a1 == 0.0) {
      S.status = AAO_EBREAKDOWN;
      S.done = 1;
      for (int i = 0; i < 4; ++i) S.cw[i] = 0.0;
      return;
    }
    const double cn = a0 / a1, sn = gn / a1;
    S.cw[0] = 1.0 / (g * a1);
    S.cw[1] = -a3 / a1;
    S.cw[2] = -a2 / a1;
    S.cw[3] = cn * S.eta;
    S.eta = -sn * S.eta;
    S.gam_prev = g;
    S.gam = gn;
    S.c_prev = S.c;
    S.c = cn;
    S.s_prev = S.s;
    S.s = sn;
    S.iters += 1;
    S.relres_est = fabs(S.eta) / S.gam1;
  } else if (step == 4) {
    // stop on the recurrence estimate (inner solves of the refinement loop, whose
    // outer loop recomputes the true residual)
    if (S.relres_est <= S.rtol) {
      S.done = 1;
      S.status = AAO_OK;
    } else if (S.iters >= S.maxit || S.gam == 0.0) {
      S.done = 1;
      S.status = AAO_ENOTCONV;
    }
  } else if (step == 3) {
    S.relres_true = sqrt(s1 / S.bnorm2);
    if (S.relres_true <= S.rtol) {
      S.done = 1;
      S.status = AAO_OK;
    } else if (S.iters >= S.maxit || S.gam == 0.0) {
      S.done = 1;
      S.status = AAO_ENOTCONV;
    }
  }
}

// Loop control of the graph-captured solve (one thread): counts `count` trips and sets
// the WHILE condition to "some right-hand side still iterating and trips < limit" (the
// limit bounds the loop whatever the scalar state holds).  CG: the done flags are read
// from L2 (written by other blocks of the running kernel).
template <bool CG>
__device__ __forceinline__ void loop_cond_body(cudaGraphConditionalHandle hw, const MinresScalars* sc, int nrhs,
                                               int* trips, int trip_limit, int count, const double* prm) {
  if (prm) trip_limit = (int)prm[1] / 2 + 2;  // two iterations per trip
  const int t = *trips + count;
  *trips = t;
  bool any = false;
  for (int r = 0; r < nrhs; ++r) {
    const int dn = CG ? __ldcg(&sc[r].done) : sc[r].done;
    if (!dn) any = true;
  }
  cudaGraphSetConditional(hw, (any && t < trip_limit) ? 1u : 0u);
}

// The work of the last block (its first warp): the step, the counter reset and the
// loop condition.  (The producers cap their registers at their own budget; whatever
// this part needs beyond it is spilled, once per right-hand side and launch.)
__device__ __forceinline__ void scalar_tail_last(const ScalarTail& t, int r, const double* p1r, int npart) {
  scalars_body<true>(t.step, t.sc[r], p1r, npart, nullptr, 0, nullptr, 0, 0.0, 0, nullptr);
  if (threadIdx.x != 0) return;
  t.arrive[r] = 0u;  // ready for the next producer (launches are stream-ordered)
  if (!t.cond) return;
  __threadfence();  // this right-hand side's scalars before its arrival
  if (atomicAdd(t.arrive + t.slot_all, 1u) != (unsigned)(t.nrhs - 1)) return;
  __threadfence();
  t.arrive[t.slot_all] = 0u;
  loop_cond_body<true>(t.hw, t.sc, t.nrhs, t.trips, t.trip_limit, 1, t.prm);
}

// The tail of a producer kernel (every thread of every block calls it, after thread 0
// wrote the block's partial): `blk_count` blocks of right-hand side r arrive; the last
// runs scalar step t.step of r on its npart partials p1r.  With t.cond, the last
// right-hand side to finish its step also sets the loop condition (one trip).
__device__ __forceinline__ void scalar_tail(const ScalarTail& t, int r, const double* p1r, int npart,
                                            int blk_count) {
  __shared__ unsigned s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();  // this block's partial before its arrival
    s_last = atomicAdd(t.arrive + r, 1u) == (unsigned)(blk_count - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();  // the other blocks' partials after their arrivals
  if (threadIdx.x < 32) scalar_tail_last(t, r, p1r, npart);
}

}  // namespace aao
