// Internal declarations shared by the CUDA translation units of libaao.so.
//
// Data layout (all FP64 vectors): time-major, (rhs, i, s) -> (rhs*n + i)*m + s,
// s lexicographic with x fastest.  Spatial lines along axis a have stride N^a.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "aao.h"
#include "dfloat.cuh"

namespace aao {

#define AAO_HD __host__ __device__ __forceinline__

// ---------------------------------------------------------------------------
// complex helpers (double2 / float2 = re, im)
// ---------------------------------------------------------------------------
AAO_HD double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
AAO_HD double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
AAO_HD double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -(a.y * b.y)), fma(a.x, b.y, a.y * b.x));
}
// a * conj(b)
AAO_HD double2 cmulc(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -(a.x * b.y)));
}
AAO_HD float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
AAO_HD float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
AAO_HD float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -(a.y * b.y)), fmaf(a.x, b.y, a.y * b.x));
}
AAO_HD float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -(a.x * b.y)));
}

template <typename R> struct Cplx;
template <> struct Cplx<double> { using T = double2; };
template <> struct Cplx<float> { using T = float2; };
template <> struct Cplx<dfl> { using T = dfl2; };

// ---------------------------------------------------------------------------
// problem plan: sizes and device tables, built once by aao_create
// ---------------------------------------------------------------------------
template <typename R>
struct PrecTables {
  using C = typename Cplx<R>::T;
  const C* tw_space = nullptr;  // M entries, exp(-2 pi i q / M)
  const R* sinw = nullptr;      // M/2+1 entries, sqrt(2/M) sin(pi j / M) / 2
  const C* tw_time = nullptr;   // n entries, exp(-2 pi i q / n)
  const R* dinv = nullptr;      // n entries, alpha^{-t/n}
  const R* d2 = nullptr;        // n entries, alpha^{2t/n}
  const C* ab = nullptr;        // (n/2+1) * npairs * 2 entries: A_k, B_k per mode pair
  R cq = 0;                     // sqrt(2/M) / 4
  // inputs of the spectral factors computed on the fly (FP32 tables only):
  const C* wq = nullptr;        // 2n entries: (1 - a theta^k)^2, 1 + a^2 theta^{2k}
  const R* lm1 = nullptr;       // m entries: Lambda_s - 1
  R inv2n = 0;                  // 1/(2n)
};

// Small-problem tiles: one warp per CTA and the fewest mode pairs (time pipeline) or
// line pairs (DST) the radix-4 stage plan allows (128/L, at least 1), so that a problem
// of a few thousand unknowns spreads over tens of SMs instead of one CTA.
constexpr int TIME_VARIANT_SMALL = 30;
constexpr int DST_VARIANT_SMALL = 8;
constexpr int SMALL_NT = 32;
constexpr int small_pairs(int L) { return L >= 128 ? 1 : 128 / L; }
// stencil / DST-basis operator kernels: threads per CTA (one spatial point each) and time
// levels per thread run, standard and for small problems
constexpr int YT_THREADS = 256;
constexpr int YT_CH_STD = 32;
constexpr int YT_CH_SMALL = 4;

struct Plan {
  int d = 0, N = 0, M = 0, n = 0, m = 0, npairs = 0;
  double tau = 0, alpha = 0, c2 = 0, h = 0;
  double coef = 0;  // c2 tau^2 / (2 h^2): L w = w - coef * (sum of neighbour differences)
  // time-kernel variant per precision (k_time.cuh): for 0..7, bit 0 = radix-16 stage
  // plan, bit 1 = half-size tile, bit 2 = interleaved padded shared-memory layout with
  // the table slice staged in shared memory; higher numbers add batched loads, bulk-copy
  // staging or integer conversions (k_time.cuh, k_time32.cu).  Defaults measured on
  // GB300: FP64 (FP64-pipe bound) radix-16 + half tile; FP32 on FP64 vectors variant 5
  // (radix-16, full tile, interleaved) with batched loads and integer store
  // conversions; double-float radix-16, full tile, interleaved without the staged table,
  // with batched loads.  Every precision also has TIME_VARIANT_SMALL (aao_create's
  // default when the standard tiles would leave most SMs idle).
  int time_variant64 = 3, time_variant32 = 24, time_variant_ff = 12;
  // DST variant: bit 0 = radix-16-first stage plan (else radix-4), bit 1 = batched
  // pre-processing loads, bit 2 = interleaved padded shared-memory layout (aao_create:
  // 1 for FP64 handles, 7 otherwise), or DST_VARIANT_SMALL
  int dst_variant = 1;
  // MINRES operator kernels: time levels per thread run of the stencil / DST-basis
  // operator (32; small problems 4) and the small shape of the w/x update (8 modes x 16
  // runs per CTA instead of 32 x 4), chosen with the small tiles
  int yt_ch = 32;
  int wx_small = 0;
  PrecTables<double> t64;
  PrecTables<float> t32;
  PrecTables<dfl> tff;  // double-float tables
};

template <typename R> inline const PrecTables<R>& tables(const Plan& P);
template <> inline const PrecTables<double>& tables<double>(const Plan& P) { return P.t64; }
template <> inline const PrecTables<float>& tables<float>(const Plan& P) { return P.t32; }
template <> inline const PrecTables<dfl>& tables<dfl>(const Plan& P) { return P.tff; }

// ---------------------------------------------------------------------------
// launchers (each returns the CUDA error of its launch and counts launches)
// ---------------------------------------------------------------------------
// Spatial DST-I along axis `axis` (0 = x) for nrhs*n time levels, in -> out (may alias).
template <typename R>
cudaError_t launch_dst_axis(const Plan& P, const R* in, R* out, int axis, int nrhs,
                            cudaStream_t s, uint64_t* nl);
// Time pipeline (all spatial modes), in -> out (may alias).
template <typename R>
cudaError_t launch_time(const Plan& P, const R* in, R* out, int nrhs, cudaStream_t s, uint64_t* nl);

struct ScalarTail;
// Stencil kernels.  mode 0: y = Y T x.  mode 1: y = Y T x and partial[b] = sum y*w.
// mode 2: no y; partial[b] = sum (w - Y T x)^2  (w = b, the true residual).
// Partials are laid out [rhs][blocks_per_rhs]; returns blocks per rhs in *nb.  tail
// (modes 1, 2; may be null): a MINRES scalar step run on the partials by the kernel.
cudaError_t launch_yt(const Plan& P, const double* x, double* y, const double* w, double* partial,
                      int mode, int nrhs, cudaStream_t s, uint64_t* nl, int* nb,
                      const ScalarTail* tail = nullptr);
int yt_blocks_per_rhs(const Plan& P);
// The operator in the DST basis (L -> diag(lam)); same modes and partial layout as launch_yt,
// plus mode 3: y = w - Y T^ x written out, partials of ||y||^2.
cudaError_t launch_ythat(const Plan& P, const double* lam, const double* x, double* y, const double* w,
                         double* partial, int mode, int nrhs, cudaStream_t s, uint64_t* nl, int* nb,
                         const ScalarTail* tail = nullptr);
// Time pipeline computed in FP32/complex64 on FP64 vectors (conversion in the load and store).
cudaError_t launch_time_mixed(const Plan& P, const double* in, double* out, int nrhs, cudaStream_t s,
                              uint64_t* nl);
// Spatial DST-I computed in double-float arithmetic on FP64 vectors.
cudaError_t launch_dst_axis_ff(const Plan& P, const double* in, double* out, int axis, int nrhs,
                               cudaStream_t s, uint64_t* nl);
// Time pipeline computed in double-float arithmetic on FP64 vectors.
cudaError_t launch_time_ff(const Plan& P, const double* in, double* out, int nrhs, cudaStream_t s,
                           uint64_t* nl);
// out[i] = nearest double-float of in[i] (complex), count entries.
cudaError_t launch_split_df(const double2* in, dfl2* out, size_t count, cudaStream_t s, uint64_t* nl);

cudaError_t launch_build_rhs(const Plan& P, const double* f, const double* psi0, const double* psi1,
                             double* b, int nrhs, cudaStream_t s, uint64_t* nl);
// The same for one right-hand side (f, psi0, psi1, b point at it) and the f levels
// k0 .. k0+cnt-1 only (they fill the b levels n-1-k0-cnt+1 .. n-1-k0).
cudaError_t launch_build_rhs_levels(const Plan& P, const double* f, const double* psi0, const double* psi1,
                                    double* b, int k0, int cnt, cudaStream_t s, uint64_t* nl);
// Variable coefficient (face arrays, see aao_set_coefficient): operator and right-hand side.
cudaError_t launch_yt_var(const Plan& P, const double* face, const double* x, double* y, const double* w,
                          double* partial, int mode, int nrhs, cudaStream_t s, uint64_t* nl, int* nb,
                          const ScalarTail* tail = nullptr);
cudaError_t launch_build_rhs_var(const Plan& P, const double* face, const double* f, const double* psi0,
                                 const double* psi1, double* b, int nrhs, cudaStream_t s, uint64_t* nl);

// Spectral factor table (device), returns min/max |Sigma| per block in mm (host-readable after sync).
// wq: 2n entries, wq[2k] = (1 - a theta^k)^2, wq[2k+1] = 1 + a^2 theta^{2k}.
cudaError_t launch_spectral_table(const Plan& P, const double* mu1d, const double2* wq,
                                  double2* ab64, float2* ab32, double* mm, int* nblocks,
                                  cudaStream_t s, uint64_t* nl);

// MINRES helpers -----------------------------------------------------------
struct MinresScalars {
  double gam, gam_prev, gam1, eta, c, c_prev, s, s_prev, delta;
  double bnorm2, relres_true, relres_est;
  double cv[3];  // v_{j+1} = cv0*T + cv1*v_j + cv2*v_{j-1}
  double cw[4];  // w_{j+1} = cw0*z_j + cw1*w_{j-1} + cw2*w_j ; x += cw3*w_{j+1}
  double rtol;
  int iters, maxit, done, status;
};

// A MINRES scalar step fused into the tail of the kernel that produces its partial sums
// (minres_scalars.cuh): the last block of each right-hand side to finish runs the step.
// sc == nullptr: no fused step (the caller launches k_scalars).
struct ScalarTail {
  MinresScalars* sc = nullptr;
  unsigned* arrive = nullptr;  // arrival counters [slot_all + 1], zero between launches
  int step = 0;
  int slot_all = 0;            // the counter over right-hand sides (cond)
  int nrhs = 0;
  // with cond: the last right-hand side to finish also sets the WHILE condition of the
  // graph-captured solve (one loop trip; as k_loop_cond)
  int cond = 0;
  cudaGraphConditionalHandle hw = 0;
  int* trips = nullptr;
  int trip_limit = 0;
  const double* prm = nullptr;
};

int dot_blocks_per_rhs(const Plan& P);
// partial[rhs*nb + b] = sum_i a_i*c_i over the rhs's n*m entries
cudaError_t launch_dot(const Plan& P, const double* a, const double* c, double* partial, int nrhs,
                       cudaStream_t s, uint64_t* nl, const ScalarTail* tail = nullptr);
// p1, p2, p3 = the partials of <a1, c1>, <a2, c2>, <a3, c3> in one pass, each bit for bit
// launch_dot's
cudaError_t launch_dot3(const Plan& P, const double* a1, const double* c1, const double* a2, const double* c2,
                        const double* a3, const double* c3, double* p1, double* p2, double* p3, int nrhs,
                        cudaStream_t s, uint64_t* nl);
// y[i] = deterministic pseudo-random values in (-1, 1) (autotuner input)
cudaError_t launch_fill_test(double* y, size_t count, cudaStream_t s);
// y = a0*x0 + a1*x1 + a2*x2 with coefficients sc[rhs].cv (which = 0) ; x2 may be null
cudaError_t launch_vupdate(const Plan& P, const double* T, const double* v, double* vprev_out,
                           const MinresScalars* sc, int nrhs, cudaStream_t s, uint64_t* nl);
cudaError_t launch_wxupdate(const Plan& P, const double* z, double* wprev_out, const double* w,
                            double* x, const MinresScalars* sc, int nrhs, cudaStream_t s,
                            uint64_t* nl, const ScalarTail* tail = nullptr);
// launch_wxupdate fused with the true residual ||b - Y T^ x||^2 of the updated x in the DST
// basis (partials [rhs][wxres_blocks_per_rhs], *nb = blocks per rhs); sc.done rhs untouched.
cudaError_t launch_wx_res(const Plan& P, const double* lam, const double* z, double* wprev_out,
                          const double* w, double* x, const double* b, const MinresScalars* sc,
                          double* partial, int nrhs, cudaStream_t s, uint64_t* nl, int* nb,
                          const ScalarTail* tail = nullptr);
int wxres_blocks_per_rhs(const Plan& P);
// y = x0 - x1 (used for r0 = b - A x0)
cudaError_t launch_sub(const Plan& P, const double* a, const double* b, double* y, int nrhs,
                       cudaStream_t s, uint64_t* nl);
// scalar steps: 0 = init (after z1, partial = <z1,v1>, partial2 = <b,b>, partial3 = <v1,v1>),
// 1 = delta (partial = <Az, z>), 2 = gamma + Givens (partial = <z_{j+1}, v_{j+1}>),
// 3 = true residual check (partial = sum r^2), 4 = recurrence-estimate check (no partial)
cudaError_t launch_scalars(int step, MinresScalars* sc, const double* partial, int nb,
                           const double* partial2, int nb2, const double* partial3, int nb3,
                           int nrhs, double rtol, int maxit, cudaStream_t s, uint64_t* nl,
                           const double* prm = nullptr);
// Graph WHILE-loop control: trips += count; condition = (any rhs not done) && trips < limit.
// With prm, the limit is prm[1]/2 + 2 (and step 0 of launch_scalars takes rtol = prm[0],
// maxit = prm[1]), so one captured graph serves every tolerance and iteration limit.
cudaError_t launch_loop_cond(cudaGraphConditionalHandle hw, const MinresScalars* sc, int nrhs, int* trips,
                             int trip_limit, int count, cudaStream_t s, uint64_t* nl,
                             const double* prm = nullptr);
// prm[0] = rtol, prm[1] = maxit (stream-ordered, ahead of a graph launch)
cudaError_t launch_set_params(double* prm, double rtol, int maxit, cudaStream_t s, uint64_t* nl);
// relres[r] = sqrt(sum of p1 partials / sum of p2 partials) per right-hand side
cudaError_t launch_relres(const double* p1, int nb1, const double* p2, int nb2, double* relres,
                          int nrhs, cudaStream_t s, uint64_t* nl);
cudaError_t launch_cast(const double* in, float* out, size_t count, cudaStream_t s, uint64_t* nl);
cudaError_t launch_uncast(const float* in, double* out, size_t count, cudaStream_t s, uint64_t* nl);
cudaError_t launch_axpy(double a, const double* x, double* y, size_t count, cudaStream_t s,
                        uint64_t* nl);

int dot_blocks_for(long long len);

// ---------------------------------------------------------------------------
// Grouped launches (serving): one launch performs the same MINRES step for up to
// GROUP_MAX independent problems of different sizes.  Problem r owns blocks
// [start[r], start[r+1]) of the launch (exclusive prefix sums of the problems' block
// counts); each block finds its problem by binary search and runs the same device
// code, on the same block decomposition, as the problem's solo launch, so a problem's
// results are bit for bit those of its solo solve.  Problems whose scalars say done
// are skipped.
// ---------------------------------------------------------------------------
constexpr int GROUP_MAX = 64;

struct GroupProblem {
  const double* z;   // z~_j (preconditioned Lanczos vector of this iteration)
  double* T;         // Y T^ z~_j (operator output)
  const double* v;   // v_j
  double* vp;        // v_{j-1} in, v_{j+1} out
  double* zn;        // z~_{j+1} (time-kernel output)
  const double* w;   // w_j
  double* wp;        // w_{j-1} in, w_{j+1} out
  double* x;         // iterate (DST basis)
  const double* b;   // right-hand side (DST basis)
  const double* lam; // Lambda_s
  MinresScalars* sc;
  double* partial;   // the problem's partial-sum slots
  int n, m;
  int yt_gx;         // spatial tiles of the operator (its blocks: yt_gx x ceil(n/32))
  int nb_dot;        // blocks of the dot product
  int nb_vu;         // blocks of the v update
};

struct GroupRound {
  int count;
  int* flags;        // device, count entries: done flag of each problem after the round
  int yt[GROUP_MAX + 1], dot[GROUP_MAX + 1], vu[GROUP_MAX + 1], wx[GROUP_MAX + 1];
  GroupProblem p[GROUP_MAX];
};

// Time-pipeline launch over the problems of one (precision, n) bucket.
template <typename R>
struct TimeGroupEntry {
  const double* in;
  double* out;
  const MinresScalars* sc;
  int m, npairs;
  PrecTables<R> tb;
};
template <typename R>
struct TimeGroup {
  int count;
  int tile[GROUP_MAX + 1];
  TimeGroupEntry<R> e[GROUP_MAX];
};

// the problem owning block b: the last r with start[r] <= b (start[0] = 0, count >= 1)
__device__ __forceinline__ int group_find(const int* __restrict__ start, int count, int b) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// blocks of each grouped launch for one problem of n time levels and m modes
int group_yt_tiles(int m);
int group_yt_blocks(int n, int m);
int group_wx_blocks(int m);
int group_vu_blocks(int n, int m);
// time-kernel tiles of a problem with m modes in the grouped launch of precision R
template <typename R>
int group_time_tiles(int L, int m);

// The grouped launches of one MINRES iteration (d_round: device copy of the round's
// descriptors; totals: the launch's block counts from the host copy).
cudaError_t launch_group_ythat(const GroupRound* d_round, int total_blocks, cudaStream_t s);
cudaError_t launch_group_scalars(int step, const GroupRound* d_round, int count, cudaStream_t s);
cudaError_t launch_group_vupdate(const GroupRound* d_round, int total_blocks, cudaStream_t s);
cudaError_t launch_group_dot(const GroupRound* d_round, int total_blocks, cudaStream_t s);
cudaError_t launch_group_wx_res(const GroupRound* d_round, int total_blocks, cudaStream_t s);
// the time-kernel variant that has a grouped form (the default one of the precision)
template <typename R>
int group_time_variant();
template <typename R>
cudaError_t launch_group_time(int L, int variant, const TimeGroup<R>* d_group, int total_tiles, cudaStream_t s);

}  // namespace aao

// Handle-level internals used by the serving runtime (defined in aao_api.cu).
aao_status aaoi_rebind(aao_handle* h, double tau, double alpha, double c2);
aao_status aaoi_solve_enqueue(aao_handle* h, const double* b, double* x, double rtol, int maxit,
                              cudaStream_t s);
aao_status aaoi_solve_collect(aao_handle* h, double rtol, aao_solve_info* info);
size_t aaoi_estimate_bytes(int dim, int N, int nt, int precision);
// Grouped serving: a handle carries one problem whose MINRES iterations are run by the
// grouped launches (GroupRound); see aao_api.cu for the contract of each call.
aao_status aaoi_serving_prepare(aao_handle* h);
aao_status aaoi_rebind_async(aao_handle* h, double tau, double alpha, double c2, cudaStream_t s);
aao_status aaoi_group_begin(aao_handle* h, const double* f, const double* psi0, const double* psi1, double* b,
                            double rtol, int maxit, cudaStream_t s);
void aaoi_group_problem(aao_handle* h, int parity, aao::GroupProblem* gp);
int aaoi_precision(const aao_handle* h);
int aaoi_nt(const aao_handle* h);
int aaoi_modes(const aao_handle* h);
int aaoi_time_variant(const aao_handle* h);
void aaoi_time_entry64(aao_handle* h, int parity, aao::TimeGroupEntry<double>* e);
void aaoi_time_entry_ff(aao_handle* h, int parity, aao::TimeGroupEntry<aao::dfl>* e);
aao_status aaoi_group_time_solo(aao_handle* h, int parity, cudaStream_t s);
aao_status aaoi_group_end(aao_handle* h, const double* b, double* x, cudaStream_t s);
aao_status aaoi_group_collect(aao_handle* h, double rtol, aao_solve_info* info);
