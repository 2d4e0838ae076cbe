// C ABI of libaao.so: handle management, tables, the P_alpha^{-1} pipeline and
// the MINRES driver (see include/aao.h for the contract of every entry point).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "aao_internal.cuh"

using namespace aao;

namespace {

thread_local std::string g_err;

aao_status fail(aao_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

#define AAO_CK(expr)                                                                 \
  do {                                                                               \
    cudaError_t e_ = (expr);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return fail(AAO_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));   \
  } while (0)

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

enum KClass {
  KC_DST_X64, KC_DST_Y64, KC_DST_Z64, KC_TIME64, KC_DST_X32, KC_DST_Y32, KC_DST_Z32, KC_TIME32,
  KC_YT, KC_YT_DOT, KC_YT_RES, KC_DOT, KC_VUPD, KC_WXUPD, KC_SCAL, KC_RHS, KC_SUB, KC_CAST,
  KC_AXPY, KC_TABLE, KC_TIMEFF, KC_DST_XFF, KC_DST_YFF, KC_DST_ZFF, KC_WXRES, KC_RESV, KC_N
};
const char* kc_name(int c) {
  static const char* names[KC_N] = {
      "dst_x_f64", "dst_y_f64", "dst_z_f64", "time_f64", "dst_x_f32", "dst_y_f32", "dst_z_f32",
      "time_f32", "yt", "yt_dot", "yt_res", "dot", "vupdate", "wxupdate", "scalars", "rhs", "sub",
      "cast", "axpy", "spectral_table", "time_f32x2", "dst_x_f32x2", "dst_y_f32x2", "dst_z_f32x2",
      "wx_res", "yt_resvec"};
  return (c >= 0 && c < KC_N) ? names[c] : "other";
}

struct ProfRec {
  int cls;
  cudaEvent_t a, b;
};

}  // namespace

struct aao_handle {
  Plan P;
  int precision = AAO_PREC_FP64;
  int nrhs_max = 1;
  int device = 0;
  uint64_t launches = 0;
  size_t bytes = 0;
  std::vector<void*> allocs;
  // tables
  double2* tw_space64 = nullptr; double* sinw64 = nullptr; double2* tw_time64 = nullptr;
  double* dinv64 = nullptr; double* d264 = nullptr; double2* ab64 = nullptr;
  float2* tw_space32 = nullptr; float* sinw32 = nullptr; float2* tw_time32 = nullptr;
  float* dinv32 = nullptr; float* d232 = nullptr; float2* ab32 = nullptr;
  float2* wq32 = nullptr; float* lm132 = nullptr;  // per-frequency Sigma terms, Lambda - 1 (FP32)
  dfl2* tw_time_ff = nullptr; dfl* dinv_ff = nullptr; dfl* d2_ff = nullptr; dfl2* ab_ff = nullptr;
  dfl2* tw_space_ff = nullptr; dfl* sinw_ff = nullptr;
  // workspace (nrhs_max * n * m doubles each)
  double* vT = nullptr; double* vv = nullptr; double* vvp = nullptr; double* vz = nullptr;
  double* vzn = nullptr; double* vw = nullptr; double* vwp = nullptr;
  double* vr = nullptr; double* vdx = nullptr;  // refinement (FP32_IR)
  double* vbh = nullptr;                         // right-hand side in the DST basis
  double* lam64 = nullptr;                       // Lambda_s, eigenvalues of L (m entries)
  double* relres_dev = nullptr;                  // nrhs_max per-rhs residual norms
  double* relres_host = nullptr;                 // pinned copy
  double* d_mu = nullptr;                        // 1D eigenvalues of -Delta_h (N)
  double2* d_wq = nullptr;                       // per-frequency Sigma terms (2n)
  double* d_mm = nullptr;                        // per-block min/max |Sigma|
  int mm_blocks = 0;
  double* face = nullptr;                        // variable coefficient on the faces (optional)
  bool var_on = false;                           // operator uses the face coefficients
  double* vxh = nullptr;                         // solution in the solve's working basis
  // the handle's own non-blocking stream: table builds in aao_create and re-binds run on
  // it, so creating or re-binding a handle never waits for work on other streams
  cudaStream_t own_stream = nullptr;
  // graph-captured solves
  bool use_graph = false;
  cudaStream_t cap_stream = nullptr;
  int* d_trips = nullptr;
  int* trips_host = nullptr;  // pinned
  double* d_prm = nullptr;    // rtol, maxit of the solve a graph launch runs
  struct GraphCache {
    long key;
    double rtol;
    int maxit;
    cudaGraphExec_t exec;
    uint64_t init_kernels, body_kernels;  // kernels in the initialisation / one loop trip
  };
  uint64_t last_init_kernels = 0, last_body_kernels = 0;
  std::vector<GraphCache> graphs;
  float* f32 = nullptr;                          // FP32 preconditioner buffer
  double* partial = nullptr; int partial_stride = 0;  // 3 * nrhs_max * partial_stride
  MinresScalars* sc = nullptr;
  MinresScalars* sc_host = nullptr;  // pinned
  // MINRES scalar steps fused into the kernels that produce their partial sums (off unless
  // AAO_FUSED_SCALARS=1: on GB300 the serial tail costs about what the graph node it
  // removes costs); arrive: their arrival counters [nrhs_max + 1], zero between launches
  bool fuse_scalars = false;
  unsigned* arrive = nullptr;
  // host-solve staging (allocated on first aao_solve_host)
  double* hs_f = nullptr; double* hs_psi = nullptr; double* hs_b = nullptr; double* hs_x = nullptr;
  cudaStream_t hs_copy = nullptr;    // copy stream of the pipelined host-buffer solve
  cudaStream_t hs_work[2] = {nullptr, nullptr};  // its two chunk-compute streams
  std::vector<cudaEvent_t> hs_ev;    // its chunk events (created on first use)
  // serving: pinned host staging of an asynchronous re-bind (aaoi_serving_prepare)
  void* pin = nullptr;
  double2* pin_wq = nullptr; double* pin_dinv = nullptr; double* pin_d2 = nullptr; double* pin_lam = nullptr;
  dfl* pin_dinv_ff = nullptr; dfl* pin_d2_ff = nullptr; double* pin_mm = nullptr;
  int pin_nb = 0;  // spectral-table blocks of the last asynchronous re-bind (0: none pending)
  // kernel timing
  bool prof_on = false;
  std::vector<ProfRec> prof;
  std::vector<cudaEvent_t> ev_pool;

  cudaEvent_t take_event() {
    if (!ev_pool.empty()) {
      cudaEvent_t e = ev_pool.back();
      ev_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }
  void clear_prof() {
    for (auto& r : prof) { ev_pool.push_back(r.a); ev_pool.push_back(r.b); }
    prof.clear();
  }
  ~aao_handle() {
    for (auto& g : graphs) cudaGraphExecDestroy(g.exec);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (own_stream) cudaStreamDestroy(own_stream);
    if (hs_copy) cudaStreamDestroy(hs_copy);
    for (cudaStream_t w : hs_work)
      if (w) cudaStreamDestroy(w);
    for (cudaEvent_t e : hs_ev) cudaEventDestroy(e);
    clear_prof();
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    for (void* p : allocs) cudaFree(p);
    if (sc_host) cudaFreeHost(sc_host);
    if (relres_host) cudaFreeHost(relres_host);
    if (trips_host) cudaFreeHost(trips_host);
    if (pin) cudaFreeHost(pin);
  }
  template <typename T>
  aao_status alloc(T** p, size_t count) {
    void* q = nullptr;
    const size_t b = count * sizeof(T);
    cudaError_t e = cudaMalloc(&q, b);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(AAO_ENOMEM, "cudaMalloc of " + std::to_string(b) + " bytes failed: " +
                                  cudaGetErrorString(e));
    }
    allocs.push_back(q);
    bytes += b;
    *p = static_cast<T*>(q);
    return AAO_OK;
  }
  size_t vlen() const { return (size_t)P.n * P.m; }
};

namespace {

#define AAO_TRY(expr)                 \
  do {                                \
    aao_status st_ = (expr);          \
    if (st_ != AAO_OK) return st_;    \
  } while (0)

// start / stop event of one timed launch (no-ops unless profiling is on)
int prof_begin(aao_handle* h, int cls, cudaStream_t s) {
  if (!h->prof_on) return -1;
  ProfRec r{cls, h->take_event(), h->take_event()};
  if (!r.a || !r.b) return -1;
  cudaEventRecord(r.a, s);
  h->prof.push_back(r);
  return (int)h->prof.size() - 1;
}
void prof_end(aao_handle* h, int idx, cudaStream_t s) {
  if (idx >= 0) cudaEventRecord(h->prof[idx].b, s);
}

// launch one kernel through its launcher, timed when profiling is on
#define AAO_KL(h, cls, s, expr)                 \
  do {                                          \
    const int pr_ = prof_begin((h), (cls), (s)); \
    AAO_CK(expr);                               \
    prof_end((h), pr_, (s));                    \
  } while (0)

// host tables in long double, rounded to double
void host_twiddles(int L, int sign, std::vector<double2>& out) {
  out.resize(L);
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int q = 0; q < L; ++q) {
    const long double ang = 2.0L * pi * (long double)q / (long double)L;
    out[q] = make_double2((double)cosl(ang), (double)(sign * sinl(ang)));
  }
}

// stream-ordered upload from (pageable) host memory; the caller synchronises the stream
template <typename T>
aao_status upload_on(const std::vector<T>& h, T* d, cudaStream_t s) {
  AAO_CK(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  return AAO_OK;
}

std::vector<float2> to_f2(const std::vector<double2>& v) {
  std::vector<float2> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = make_float2((float)v[i].x, (float)v[i].y);
  return o;
}
std::vector<float> to_f(const std::vector<double>& v) {
  std::vector<float> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = (float)v[i];
  return o;
}
std::vector<dfl> to_df(const std::vector<double>& v) {
  std::vector<dfl> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = dfl(v[i]);
  return o;
}
std::vector<dfl2> to_df2(const std::vector<double2>& v) {
  std::vector<dfl2> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = dfl2{dfl(v[i].x), dfl(v[i].y)};
  return o;
}

aao_status check_handle(const aao_handle* h) {
  if (!h) return fail(AAO_EINVAL, "null handle");
  return AAO_OK;
}

aao_status check_call(aao_handle* h, int nrhs) {
  AAO_TRY(check_handle(h));
  if (nrhs < 1 || nrhs > h->nrhs_max)
    return fail(AAO_EINVAL, "nrhs must be in [1, nrhs_max=" + std::to_string(h->nrhs_max) + "]");
  AAO_CK(cudaSetDevice(h->device));
  return AAO_OK;
}

// Device buffers of aao_solve_host (f, b, x, psi0 and psi1 for nrhs_max right-hand
// sides), its copy stream, two chunk-compute streams and its events: reserved by
// aao_create when opts.host_staging is set, else by the first aao_solve_host.
constexpr int HOST_CHUNK = 32;  // time levels per pipelined copy chunk (n is a power of two >= 64)
aao_status reserve_host_staging(aao_handle* h) {
  const size_t vl = (size_t)h->nrhs_max * h->vlen();
  AAO_TRY(h->alloc(&h->hs_f, vl));
  AAO_TRY(h->alloc(&h->hs_b, vl));
  AAO_TRY(h->alloc(&h->hs_x, vl));
  AAO_TRY(h->alloc(&h->hs_psi, (size_t)2 * h->nrhs_max * h->P.m));
  AAO_CK(cudaStreamCreateWithFlags(&h->hs_copy, cudaStreamNonBlocking));
  for (cudaStream_t& w : h->hs_work) AAO_CK(cudaStreamCreateWithFlags(&w, cudaStreamNonBlocking));
  const int nch = h->nrhs_max * (h->P.n / HOST_CHUNK);
  while ((int)h->hs_ev.size() < 2 * nch + 8) {
    cudaEvent_t e = nullptr;
    AAO_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    h->hs_ev.push_back(e);
  }
  return AAO_OK;
}

// P^{-1} applied in the handle's precision: in -> out (FP64 vectors, may alias)
aao_status prec_apply(aao_handle* h, const double* in, double* out, int nrhs, cudaStream_t s) {
  const Plan& P = h->P;
  if (h->precision == AAO_PREC_FP64) {
    AAO_KL(h, KC_DST_X64, s, launch_dst_axis<double>(P, in, out, 0, nrhs, s, &h->launches));
    for (int ax = 1; ax < P.d; ++ax)
      AAO_KL(h, KC_DST_X64 + ax, s, launch_dst_axis<double>(P, out, out, ax, nrhs, s, &h->launches));
    AAO_KL(h, KC_TIME64, s, launch_time<double>(P, out, out, nrhs, s, &h->launches));
    for (int ax = P.d - 1; ax >= 0; --ax)
      AAO_KL(h, KC_DST_X64 + ax, s, launch_dst_axis<double>(P, out, out, ax, nrhs, s, &h->launches));
  } else if (h->precision == AAO_PREC_F32X2) {
    AAO_KL(h, KC_DST_XFF, s, launch_dst_axis_ff(P, in, out, 0, nrhs, s, &h->launches));
    for (int ax = 1; ax < P.d; ++ax)
      AAO_KL(h, KC_DST_XFF + ax, s, launch_dst_axis_ff(P, out, out, ax, nrhs, s, &h->launches));
    AAO_KL(h, KC_TIMEFF, s, launch_time_ff(P, out, out, nrhs, s, &h->launches));
    for (int ax = P.d - 1; ax >= 0; --ax)
      AAO_KL(h, KC_DST_XFF + ax, s, launch_dst_axis_ff(P, out, out, ax, nrhs, s, &h->launches));
  } else {
    const size_t cnt = (size_t)nrhs * h->vlen();
    AAO_KL(h, KC_CAST, s, launch_cast(in, h->f32, cnt, s, &h->launches));
    for (int ax = 0; ax < P.d; ++ax)
      AAO_KL(h, KC_DST_X32 + ax, s, launch_dst_axis<float>(P, h->f32, h->f32, ax, nrhs, s, &h->launches));
    AAO_KL(h, KC_TIME32, s, launch_time<float>(P, h->f32, h->f32, nrhs, s, &h->launches));
    for (int ax = P.d - 1; ax >= 0; --ax)
      AAO_KL(h, KC_DST_X32 + ax, s, launch_dst_axis<float>(P, h->f32, h->f32, ax, nrhs, s, &h->launches));
    AAO_KL(h, KC_CAST, s, launch_uncast(h->f32, out, cnt, s, &h->launches));
  }
  return AAO_OK;
}

// ---------------------------------------------------------------------------
// MINRES in the DST basis.
//
// U = S (x) .. (x) S is orthogonal and symmetric, so with x^ = (I (x) U) x,
// b^ = (I (x) U) b the system Y T x = b is Y T^ x^ = b^ with T^ = T after L -> Lambda
// (diagonal), and P_alpha^{-1} becomes its time part alone.  MINRES on the
// transformed system produces the transformed iterates (inner products and 2-norms
// are unchanged by U), so each iteration needs only the time pipeline and the
// pointwise-in-space operator; the DSTs run on b at the start and on x^ at the end.
// ---------------------------------------------------------------------------

// time part of P^{-1} in the handle's precision: in -> out (FP64 vectors)
aao_status time_apply(aao_handle* h, const double* in, double* out, int nrhs, cudaStream_t s) {
  if (h->precision == AAO_PREC_FP64)
    AAO_KL(h, KC_TIME64, s, launch_time<double>(h->P, in, out, nrhs, s, &h->launches));
  else if (h->precision == AAO_PREC_F32X2)
    AAO_KL(h, KC_TIMEFF, s, launch_time_ff(h->P, in, out, nrhs, s, &h->launches));
  else
    AAO_KL(h, KC_TIME32, s, launch_time_mixed(h->P, in, out, nrhs, s, &h->launches));
  return AAO_OK;
}

// (I (x) U) in -> out (FP64 vectors; out may equal in); double-float arithmetic for the
// AAO_PREC_F32X2 and AAO_PREC_FP32_IR handles (the refinement's b^ and x need ~1e-14
// relative accuracy, which double-float gives at two thirds of the FP64 cost), FP64
// otherwise
aao_status dst_apply(aao_handle* h, const double* in, double* out, int nrhs, cudaStream_t s) {
  if (h->precision == AAO_PREC_F32X2 || h->precision == AAO_PREC_FP32_IR) {
    AAO_KL(h, KC_DST_XFF, s, launch_dst_axis_ff(h->P, in, out, 0, nrhs, s, &h->launches));
    for (int ax = 1; ax < h->P.d; ++ax)
      AAO_KL(h, KC_DST_XFF + ax, s, launch_dst_axis_ff(h->P, out, out, ax, nrhs, s, &h->launches));
    return AAO_OK;
  }
  AAO_KL(h, KC_DST_X64, s, launch_dst_axis<double>(h->P, in, out, 0, nrhs, s, &h->launches));
  for (int ax = 1; ax < h->P.d; ++ax)
    AAO_KL(h, KC_DST_X64 + ax, s, launch_dst_axis<double>(h->P, out, out, ax, nrhs, s, &h->launches));
  return AAO_OK;
}

// (I (x) U) on nlev consecutive time levels starting at in / out (the levels of a DST
// are independent), in the arithmetic dst_apply uses
aao_status dst_apply_levels(aao_handle* h, const double* in, double* out, int nlev, cudaStream_t s) {
  Plan Q = h->P;
  Q.n = nlev;
  const bool ff = h->precision == AAO_PREC_F32X2 || h->precision == AAO_PREC_FP32_IR;
  for (int ax = 0; ax < Q.d; ++ax) {
    const double* src = ax == 0 ? in : out;
    if (ff) AAO_KL(h, KC_DST_XFF + ax, s, launch_dst_axis_ff(Q, src, out, ax, 1, s, &h->launches));
    else AAO_KL(h, KC_DST_X64 + ax, s, launch_dst_axis<double>(Q, src, out, ax, 1, s, &h->launches));
  }
  return AAO_OK;
}

// The physical operator Y T (constant or variable coefficient), modes as launch_yt.
cudaError_t launch_op(aao_handle* h, const double* x, double* y, const double* w, double* partial, int mode,
                      int nrhs, cudaStream_t s, int* nb, const ScalarTail* tail = nullptr) {
  if (h->var_on) return launch_yt_var(h->P, h->face, x, y, w, partial, mode, nrhs, s, &h->launches, nb, tail);
  return launch_yt(h->P, x, y, w, partial, mode, nrhs, s, &h->launches, nb, tail);
}

cudaError_t launch_rhs(aao_handle* h, const double* f, const double* psi0, const double* psi1, double* b,
                       int nrhs, cudaStream_t s) {
  if (h->var_on) return launch_build_rhs_var(h->P, h->face, f, psi0, psi1, b, nrhs, s, &h->launches);
  return launch_build_rhs(h->P, f, psi0, psi1, b, nrhs, s, &h->launches);
}

// Preconditioned MINRES on Y T^ x^ = bh (DST basis) from x^ = (use_x0 ? xh : 0).
// physical: run on the physical system instead (operator launch_op, preconditioner the
// full P_alpha^{-1} with its DSTs) -- used when the coefficient is variable.
// true_res: stop on the true relative residual ||bh - Y T^ x^|| / ||bh|| recomputed every
// iteration (the solver's contract); otherwise on the recurrence estimate (inner
// refinement solves, whose outer loop recomputes the residual).
struct MinresBufs {
  double *v, *vp, *z, *zn, *w, *wp;
};

struct MinresCtx {
  aao_handle* h;
  const double* bh;
  double* xh;
  int nrhs;
  double rtol;
  int maxit;
  cudaStream_t s;
  bool true_res, physical;
  const double* prm = nullptr;  // graph capture: rtol, maxit read from device memory
  // graph capture: the WHILE condition handle and the trip limit of the loop body
  bool in_graph = false;
  cudaGraphConditionalHandle hw = 0;
  int trip_limit = 0;
  cudaError_t op(const double* xx, double* yy, const double* ww, double* part, int mode, int* nbp,
                 const ScalarTail* tail = nullptr) const {
    return physical ? launch_op(h, xx, yy, ww, part, mode, nrhs, s, nbp, tail)
                    : launch_ythat(h->P, h->lam64, xx, yy, ww, part, mode, nrhs, s, &h->launches, nbp, tail);
  }
  aao_status prec(const double* in, double* out) const {
    return physical ? prec_apply(h, in, out, nrhs, s) : time_apply(h, in, out, nrhs, s);
  }
};

aao_status get_graph(const MinresCtx& c, int use_x0, cudaGraphExec_t* out);
aao_status set_params(aao_handle* h, double tau, double alpha, double c2, cudaStream_t s);

// Initialisation kernels (stream-ordered, no host synchronisation).
aao_status minres_enqueue_init(const MinresCtx& c, int use_x0, const MinresBufs& B) {
  aao_handle* h = c.h;
  const Plan& P = h->P;
  const cudaStream_t s = c.s;
  const size_t vb = (size_t)c.nrhs * h->vlen() * sizeof(double);
  double* p1 = h->partial;
  double* p2 = h->partial + (size_t)h->nrhs_max * h->partial_stride;
  double* p3 = h->partial + (size_t)2 * h->nrhs_max * h->partial_stride;
  const int nb_dot = dot_blocks_per_rhs(P);
  uint64_t* nl = &h->launches;
  int nb_yt = 0;
  if (use_x0) {
    AAO_KL(h, KC_YT, s, c.op(c.xh, h->vT, nullptr, nullptr, 0, &nb_yt));
    AAO_KL(h, KC_SUB, s, launch_sub(P, c.bh, h->vT, B.v, c.nrhs, s, nl));
  } else {
    AAO_CK(cudaMemsetAsync(c.xh, 0, vb, s));
    AAO_CK(cudaMemcpyAsync(B.v, c.bh, vb, cudaMemcpyDeviceToDevice, s));
  }
  AAO_CK(cudaMemsetAsync(B.vp, 0, vb, s));
  AAO_CK(cudaMemsetAsync(B.w, 0, vb, s));
  AAO_CK(cudaMemsetAsync(B.wp, 0, vb, s));
  AAO_TRY(c.prec(B.v, B.z));
  AAO_KL(h, KC_DOT, s, launch_dot3(P, B.z, B.v, c.bh, c.bh, B.v, B.v, p1, p2, p3, c.nrhs, s, nl));
  AAO_KL(h, KC_SCAL, s, launch_scalars(0, h->sc, p1, nb_dot, p2, nb_dot, p3, nb_dot, c.nrhs, c.rtol,
                                       c.maxit, s, nl, c.prm));
  return AAO_OK;
}

// One MINRES iteration with buffers B (stream-ordered, no host synchronisation);
// afterwards the roles rotate: (v, vp), (z, zn), (w, wp) swap.  With fused scalar steps
// (h->fuse_scalars) each step runs in the tail of the kernel that produces its partial
// sums, with the same code and summation order as k_scalars (same bits), and an
// iteration is five launches in the DST basis: operator + delta, v update,
// preconditioner, dot + gamma/Givens, w/x update + residual + stop test.  ends_trip (graph
// capture): this iteration's stop test also sets the loop condition (no k_loop_cond).
aao_status minres_enqueue_iter(const MinresCtx& c, const MinresBufs& B, bool ends_trip = false) {
  aao_handle* h = c.h;
  const Plan& P = h->P;
  const cudaStream_t s = c.s;
  double* p1 = h->partial;
  const int nb_dot = dot_blocks_per_rhs(P);
  uint64_t* nl = &h->launches;
  const int nrhs = c.nrhs;
  const bool fz = h->fuse_scalars;
  auto tail = [&](int step, bool cond) {
    ScalarTail t;
    t.sc = h->sc;
    t.arrive = h->arrive;
    t.step = step;
    t.slot_all = h->nrhs_max;
    t.nrhs = nrhs;
    if (cond && c.in_graph) {
      t.cond = 1;
      t.hw = c.hw;
      t.trips = h->d_trips;
      t.trip_limit = c.trip_limit;
      t.prm = c.prm;
    }
    return t;
  };
  auto scal = [&](int step, int nb) {
    return launch_scalars(step, h->sc, p1, nb, nullptr, 0, nullptr, 0, nrhs, c.rtol, c.maxit, s, nl);
  };
  const ScalarTail t1 = tail(1, false), t2 = tail(2, false), tl = tail(c.true_res ? 3 : 4, ends_trip);
  int nb_yt = 0;
  AAO_KL(h, KC_YT_DOT, s, c.op(B.z, h->vT, B.z, p1, 1, &nb_yt, fz ? &t1 : nullptr));
  if (!fz) AAO_KL(h, KC_SCAL, s, scal(1, nb_yt));
  AAO_KL(h, KC_VUPD, s, launch_vupdate(P, h->vT, B.v, B.vp, h->sc, nrhs, s, nl));  // vp <- v_{j+1}
  AAO_TRY(c.prec(B.vp, B.zn));
  AAO_KL(h, KC_DOT, s, launch_dot(P, B.zn, B.vp, p1, nrhs, s, nl, fz ? &t2 : nullptr));
  if (!fz) AAO_KL(h, KC_SCAL, s, scal(2, nb_dot));
  if (c.true_res && !c.physical) {
    // DST basis: the update and the true residual of the new iterate in one pass
    AAO_KL(h, KC_WXRES, s, launch_wx_res(P, h->lam64, B.z, B.wp, B.w, c.xh, c.bh, h->sc, p1, nrhs, s, nl,
                                         &nb_yt, fz ? &tl : nullptr));  // wp <- w_{j+1}
    if (!fz) AAO_KL(h, KC_SCAL, s, scal(3, nb_yt));
    return AAO_OK;
  }
  if (c.true_res) {
    AAO_KL(h, KC_WXUPD, s, launch_wxupdate(P, B.z, B.wp, B.w, c.xh, h->sc, nrhs, s, nl));  // wp <- w_{j+1}
    AAO_KL(h, KC_YT_RES, s, c.op(c.xh, nullptr, c.bh, p1, 2, &nb_yt, fz ? &tl : nullptr));
    if (!fz) AAO_KL(h, KC_SCAL, s, scal(3, nb_yt));
  } else {
    AAO_KL(h, KC_WXUPD, s, launch_wxupdate(P, B.z, B.wp, B.w, c.xh, h->sc, nrhs, s, nl, fz ? &tl : nullptr));
    if (!fz) AAO_KL(h, KC_SCAL, s, scal(4, 0));
  }
  return AAO_OK;
}

MinresBufs rotate(const MinresBufs& B) { return MinresBufs{B.vp, B.v, B.zn, B.z, B.wp, B.w}; }

aao_status minres_collect(aao_handle* h, int nrhs, aao_solve_info* info) {
  aao_status worst = AAO_OK;
  for (int r = 0; r < nrhs; ++r) {
    const MinresScalars& S = h->sc_host[r];
    aao_status st = (aao_status)S.status;
    if (!S.done && st == AAO_OK) st = AAO_ENOTCONV;
    if (info) {
      info[r].iters = S.iters;
      info[r].status = st;
      info[r].relres_true = S.relres_true;
      info[r].relres_est = S.relres_est;
      info[r].ir_steps = 0;
      info[r].reserved = 0;
    }
    if (st != AAO_OK && worst == AAO_OK) worst = st;
  }
  return worst;
}

// Capture the whole solve (initialisation, then a device-side WHILE loop whose body is
// two buffer-rotated iterations and a condition kernel) into one executable graph.
// Every pointer it touches belongs to the handle, so the graph is reused across solves.
aao_status build_graph(const MinresCtx& c, int use_x0, cudaGraphExec_t* out) {
  aao_handle* h = c.h;
  const uint64_t l0 = h->launches;  // launcher calls during capture are not launches
  MinresCtx cc = c;
  cudaStream_t cs = h->cap_stream;
  cc.s = cs;
  cc.prm = h->d_prm;  // rtol and maxit are set before each launch, not captured
  const MinresBufs B0{h->vv, h->vvp, h->vz, h->vzn, h->vw, h->vwp};
  const int trip_limit = c.maxit / 2 + 2;
  cc.in_graph = true;
  cc.trip_limit = trip_limit;
  cudaGraph_t g = nullptr;
  AAO_CK(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle hw;
  auto fail_cleanup = [&](cudaError_t e, const char* what) {
    cudaStreamCaptureStatus cst;
    if (cudaStreamIsCapturing(cs, &cst) == cudaSuccess && cst != cudaStreamCaptureStatusNone) {
      cudaGraph_t tmp = nullptr;
      cudaStreamEndCapture(cs, &tmp);
      if (tmp && tmp != g) cudaGraphDestroy(tmp);
    }
    cudaGraphDestroy(g);
    cudaGetLastError();
    return fail(AAO_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  };
  cudaError_t e = cudaGraphConditionalHandleCreate(&hw, g, 0, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return fail_cleanup(e, "cudaGraphConditionalHandleCreate");
  cc.hw = hw;
  e = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return fail_cleanup(e, "cudaStreamBeginCaptureToGraph");
  if (cudaMemsetAsync(h->d_trips, 0, sizeof(int), cs) != cudaSuccess ||
      minres_enqueue_init(cc, use_x0, B0) != AAO_OK ||
      launch_loop_cond(hw, h->sc, c.nrhs, h->d_trips, trip_limit, 0, cs, &h->launches, h->d_prm) != cudaSuccess) {
    h->launches = l0;
    return fail_cleanup(cudaGetLastError(), "graph initialisation capture");
  }
  const uint64_t init_k = h->launches - l0;
  cudaStreamCaptureStatus cst;
  cudaGraph_t capg = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &capg, &deps, nullptr, &ndeps);
  if (e != cudaSuccess) return fail_cleanup(e, "cudaStreamGetCaptureInfo");
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hw;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t wnode;
  e = cudaGraphAddNode(&wnode, capg, deps, nullptr, ndeps, &cp);
  if (e != cudaSuccess) return fail_cleanup(e, "cudaGraphAddNode(while)");
  e = cudaStreamUpdateCaptureDependencies(cs, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e != cudaSuccess) return fail_cleanup(e, "cudaStreamUpdateCaptureDependencies");
  cudaGraph_t gend = nullptr;
  e = cudaStreamEndCapture(cs, &gend);
  if (e != cudaSuccess) return fail_cleanup(e, "cudaStreamEndCapture");
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return fail_cleanup(e, "capture of the loop body");
  const MinresBufs B1 = rotate(B0);
  // the second iteration's stop test sets the loop condition when the steps are fused
  if (minres_enqueue_iter(cc, B0) != AAO_OK || minres_enqueue_iter(cc, B1, true) != AAO_OK ||
      (!h->fuse_scalars &&
       launch_loop_cond(hw, h->sc, c.nrhs, h->d_trips, trip_limit, 1, cs, &h->launches, h->d_prm) != cudaSuccess)) {
    h->launches = l0;
    return fail_cleanup(cudaGetLastError(), "loop body capture");
  }
  h->last_init_kernels = init_k;
  h->last_body_kernels = h->launches - l0 - init_k;
  h->launches = l0;
  cudaGraph_t bend = nullptr;
  e = cudaStreamEndCapture(cs, &bend);
  if (e != cudaSuccess) return fail_cleanup(e, "cudaStreamEndCapture(body)");
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(AAO_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  }
  return AAO_OK;
}

// Preconditioned MINRES on Y T^ x^ = bh (DST basis) from x^ = (use_x0 ? xh : 0).
// true_res: stop on the true relative residual ||bh - Y T^ x^|| / ||bh|| recomputed every
// iteration (the solver's contract); otherwise on the recurrence estimate (inner
// refinement solves).  physical: the physical system instead (operator launch_op,
// preconditioner the full P_alpha^{-1}; used for a variable coefficient).
// With graphs enabled (and kernel timing off) the loop runs on the device from one
// captured graph per (batch size, mode); bh and xh must then be handle workspace.
// Graph path, after the stream has reached the end of the launched graph: count its
// kernels and read the scalars copied to the host.
aao_status minres_finish_graph(aao_handle* h, int nrhs, aao_solve_info* info) {
  // kernels the graph ran: the initialisation plus one body per loop trip
  h->launches += h->last_init_kernels + (uint64_t)(*h->trips_host) * h->last_body_kernels;
  return minres_collect(h, nrhs, info);
}

// deferred (graph path only; may be null): enqueue the solve and the copies of its
// scalars and return with *deferred = true; the caller synchronises s (after enqueuing
// more work of its own) and then calls minres_finish_graph.  One host round trip per
// solve instead of two.
aao_status minres_spectral(aao_handle* h, const double* bh, double* xh, int use_x0, int nrhs,
                           double rtol, int maxit, aao_solve_info* info, cudaStream_t s, bool true_res,
                           bool physical = false, bool* deferred = nullptr) {
  MinresCtx c{h, bh, xh, nrhs, rtol, maxit, s, true_res, physical};
  const size_t scb = (size_t)nrhs * sizeof(MinresScalars);
  const MinresBufs B0{h->vv, h->vvp, h->vz, h->vzn, h->vw, h->vwp};
  if (h->use_graph && !h->prof_on) {
    // rtol and maxit go to device memory ahead of the launch and the captured
    // initialisation and loop condition read them there; the graph is keyed on the rest.
    cudaGraphExec_t ex = nullptr;
    if (get_graph(c, use_x0, &ex) != AAO_OK) {
      // keep solving with the host-driven loop (aao_last_error keeps the reason)
      h->use_graph = false;
      return minres_spectral(h, bh, xh, use_x0, nrhs, rtol, maxit, info, s, true_res, physical);
    }
    AAO_CK(launch_set_params(h->d_prm, rtol, maxit, s, &h->launches));
    AAO_CK(cudaGraphLaunch(ex, s));
    AAO_CK(cudaMemcpyAsync(h->sc_host, h->sc, scb, cudaMemcpyDeviceToHost, s));
    AAO_CK(cudaMemcpyAsync(h->trips_host, h->d_trips, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (deferred) {
      *deferred = true;
      return AAO_OK;
    }
    AAO_CK(cudaStreamSynchronize(s));
    return minres_finish_graph(h, nrhs, info);
  }
  AAO_TRY(minres_enqueue_init(c, use_x0, B0));
  AAO_CK(cudaMemcpyAsync(h->sc_host, h->sc, scb, cudaMemcpyDeviceToHost, s));
  AAO_CK(cudaStreamSynchronize(s));
  auto all_done = [&]() {
    for (int r = 0; r < nrhs; ++r)
      if (!h->sc_host[r].done) return false;
    return true;
  };
  MinresBufs B = B0;
  for (int it = 0; it < maxit && !all_done(); ++it) {
    AAO_TRY(minres_enqueue_iter(c, B));
    B = rotate(B);
    AAO_CK(cudaMemcpyAsync(h->sc_host, h->sc, scb, cudaMemcpyDeviceToHost, s));
    AAO_CK(cudaStreamSynchronize(s));
  }
  return minres_collect(h, nrhs, info);
}

// ||b - Y T x|| / ||b|| per rhs in the physical basis (stencil), copied into info.
// The physical residual check in two halves: the kernels and the copy of the relative
// residuals to the host (stream-ordered), then, after the stream is synchronised, the
// residuals into info and the status.
aao_status physical_check_enqueue(aao_handle* h, const double* b, const double* x, int nrhs, cudaStream_t s) {
  double* p1 = h->partial;
  double* p2 = h->partial + (size_t)h->nrhs_max * h->partial_stride;
  int nb = 0;
  AAO_KL(h, KC_YT_RES, s, launch_op(h, x, nullptr, b, p1, 2, nrhs, s, &nb));
  AAO_KL(h, KC_DOT, s, launch_dot(h->P, b, b, p2, nrhs, s, &h->launches));
  AAO_KL(h, KC_SCAL, s, launch_relres(p1, nb, p2, dot_blocks_per_rhs(h->P), h->relres_dev, nrhs, s,
                                      &h->launches));
  AAO_CK(cudaMemcpyAsync(h->relres_host, h->relres_dev, nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
  return AAO_OK;
}

void physical_check_finish(aao_handle* h, int nrhs, double rtol, aao_solve_info* info, aao_status* worst) {
  for (int r = 0; r < nrhs; ++r) {
    if (info) info[r].relres_true = h->relres_host[r];
    if (h->relres_host[r] > rtol && *worst == AAO_OK) *worst = AAO_ENOTCONV;
    if (info && h->relres_host[r] > rtol && info[r].status == AAO_OK) info[r].status = AAO_ENOTCONV;
  }
}

aao_status physical_check(aao_handle* h, const double* b, const double* x, int nrhs, double rtol,
                          aao_solve_info* info, aao_status* worst, cudaStream_t s) {
  AAO_TRY(physical_check_enqueue(h, b, x, nrhs, s));
  AAO_CK(cudaStreamSynchronize(s));
  physical_check_finish(h, nrhs, rtol, info, worst);
  return AAO_OK;
}

// FP64 solve: DST b, MINRES in the DST basis, DST x^ back, physical residual check.
// (Variable coefficient: the same on the physical system, with b and x copied in/out.)
aao_status solve_fp64(aao_handle* h, const double* b, double* x, int use_x0, int nrhs, double rtol,
                      int maxit, aao_solve_info* info, cudaStream_t s) {
  std::vector<aao_solve_info> loc(nrhs);
  aao_solve_info* inf = info ? info : loc.data();
  const size_t vb = (size_t)nrhs * h->vlen() * sizeof(double);
  if (h->var_on) {  // operator not diagonal in the DST basis: physical-basis MINRES
    AAO_CK(cudaMemcpyAsync(h->vbh, b, vb, cudaMemcpyDeviceToDevice, s));
    if (use_x0) AAO_CK(cudaMemcpyAsync(h->vxh, x, vb, cudaMemcpyDeviceToDevice, s));
    aao_status w = minres_spectral(h, h->vbh, h->vxh, use_x0, nrhs, rtol, maxit, inf, s, true, true);
    AAO_CK(cudaMemcpyAsync(x, h->vxh, vb, cudaMemcpyDeviceToDevice, s));
    AAO_CK(cudaStreamSynchronize(s));
    if (w != AAO_OK) g_err = std::string("MINRES: ") + aao_status_str(w);
    return w;
  }
  AAO_TRY(dst_apply(h, b, h->vbh, nrhs, s));
  if (use_x0) AAO_TRY(dst_apply(h, x, h->vxh, nrhs, s));
  // graph path: the solve, the inverse DSTs and the physical check are enqueued back to
  // back and the host waits once
  bool deferred = false;
  aao_status worst = minres_spectral(h, h->vbh, h->vxh, use_x0, nrhs, rtol, maxit, inf, s, true, false, &deferred);
  AAO_TRY(dst_apply(h, h->vxh, x, nrhs, s));
  AAO_TRY(physical_check_enqueue(h, b, x, nrhs, s));
  AAO_CK(cudaStreamSynchronize(s));
  if (deferred) worst = minres_finish_graph(h, nrhs, inf);
  physical_check_finish(h, nrhs, rtol, inf, &worst);
  if (worst != AAO_OK) g_err = std::string("MINRES: ") + aao_status_str(worst);
  return worst;
}

// Mixed precision: FP64 iterative refinement in the DST basis around MINRES whose
// preconditioner (the time pipeline) runs in FP32/complex64.
// bh_ready (DST basis, zero initial guess): b^ is already in the handle's b^ vector (the
// pipelined host-buffer solve transformed it chunk by chunk); the call then ends with x^
// in the handle's x^ vector and the refinement status, and the caller runs the inverse
// DSTs and the physical check.
aao_status solve_ir(aao_handle* h, const double* b, double* x, int use_x0, int nrhs, double rtol,
                    int maxit, aao_solve_info* info, cudaStream_t s, bool bh_ready = false) {
  const Plan& P = h->P;
  const size_t vb = (size_t)nrhs * h->vlen() * sizeof(double);
  double* p1 = h->partial;
  double* p2 = h->partial + (size_t)h->nrhs_max * h->partial_stride;
  uint64_t* nl = &h->launches;
  const bool phys = h->var_on;  // variable coefficient: refine in the physical basis
  double* bh = h->vbh;
  double* xh = h->vxh;
  std::vector<aao_solve_info> inner(nrhs), loc(nrhs);
  aao_solve_info* acc = info ? info : loc.data();
  for (int r = 0; r < nrhs; ++r) acc[r] = aao_solve_info{0, AAO_ENOTCONV, 1.0, 1.0, 0, 0};
  if (bh_ready) {
    if (phys || use_x0) return fail(AAO_EINVAL, "internal: pre-transformed refinement solve");
  } else if (!phys) {
    AAO_TRY(dst_apply(h, b, bh, nrhs, s));
    if (use_x0) AAO_TRY(dst_apply(h, x, xh, nrhs, s));
  } else {
    AAO_CK(cudaMemcpyAsync(bh, b, vb, cudaMemcpyDeviceToDevice, s));
    if (use_x0) AAO_CK(cudaMemcpyAsync(xh, x, vb, cudaMemcpyDeviceToDevice, s));
  }
  if (!use_x0) AAO_CK(cudaMemsetAsync(xh, 0, vb, s));
  const int nb_dot = dot_blocks_per_rhs(P);
  AAO_KL(h, KC_DOT, s, launch_dot(P, bh, bh, p2, nrhs, s, nl));
  std::vector<double> hp((size_t)nrhs * std::max(nb_dot, yt_blocks_per_rhs(P)));
  AAO_CK(cudaMemcpyAsync(hp.data(), p2, (size_t)nrhs * nb_dot * sizeof(double), cudaMemcpyDeviceToHost, s));
  AAO_CK(cudaStreamSynchronize(s));
  std::vector<double> bn(nrhs, 0.0);
  for (int r = 0; r < nrhs; ++r) {
    double t = 0;
    for (int i = 0; i < nb_dot; ++i) t += hp[(size_t)r * nb_dot + i];
    bn[r] = std::sqrt(t > 0 ? t : 1.0);
  }
  const int max_ir = 40;
  int total_its = 0;
  for (int ir = 0; ir < max_ir; ++ir) {
    // r^ = b^ - Y T^ x^ in FP64 and its norm (one fused pass in the DST basis)
    int nb_yt = 0, nb_r = nb_dot;
    if (phys) {
      AAO_KL(h, KC_YT, s, launch_op(h, xh, h->vT, nullptr, nullptr, 0, nrhs, s, &nb_yt));
      AAO_KL(h, KC_SUB, s, launch_sub(P, bh, h->vT, h->vr, nrhs, s, nl));
      AAO_KL(h, KC_DOT, s, launch_dot(P, h->vr, h->vr, p1, nrhs, s, nl));
    } else {
      AAO_KL(h, KC_RESV, s, launch_ythat(P, h->lam64, xh, h->vr, bh, p1, 3, nrhs, s, nl, &nb_r));
    }
    AAO_CK(cudaMemcpyAsync(hp.data(), p1, (size_t)nrhs * nb_r * sizeof(double), cudaMemcpyDeviceToHost, s));
    AAO_CK(cudaStreamSynchronize(s));
    bool all = true;
    double worst_rel = 0.0;
    for (int r = 0; r < nrhs; ++r) {
      double t = 0;
      for (int i = 0; i < nb_r; ++i) t += hp[(size_t)r * nb_r + i];
      const double rel = std::sqrt(t) / bn[r];
      acc[r].relres_true = rel;
      acc[r].ir_steps = ir;
      if (rel <= rtol) acc[r].status = AAO_OK;
      else all = false;
      if (acc[r].status != AAO_OK) worst_rel = std::max(worst_rel, rel);
    }
    if (all || total_its >= maxit) break;
    // inner solve Y T^ dx^ = r^ to the relative accuracy that reaches rtol overall
    double inner_tol = std::max(0.5 * rtol / worst_rel, 1e-7);
    inner_tol = std::min(inner_tol, 1e-2);
    minres_spectral(h, h->vr, h->vdx, 0, nrhs, inner_tol, maxit - total_its, inner.data(), s, false, phys);
    int its = 0;
    for (int r = 0; r < nrhs; ++r) {
      its = std::max(its, inner[r].iters);
      acc[r].iters += inner[r].iters;
      acc[r].relres_est = inner[r].relres_est;
    }
    total_its += std::max(its, 1);
    for (int r = 0; r < nrhs; ++r) {
      if (acc[r].status == AAO_OK) continue;
      AAO_KL(h, KC_AXPY, s, launch_axpy(1.0, h->vdx + (size_t)r * h->vlen(), xh + (size_t)r * h->vlen(),
                                        h->vlen(), s, nl));
    }
  }
  aao_status worst = AAO_OK;
  for (int r = 0; r < nrhs; ++r)
    if (acc[r].status != AAO_OK && worst == AAO_OK) worst = (aao_status)acc[r].status;
  if (bh_ready) return worst;
  if (!phys) AAO_TRY(dst_apply(h, xh, x, nrhs, s));
  else AAO_CK(cudaMemcpyAsync(x, xh, vb, cudaMemcpyDeviceToDevice, s));
  AAO_TRY(physical_check(h, b, x, nrhs, rtol, acc, &worst, s));
  if (worst != AAO_OK)
    g_err = std::string("MINRES (FP32 preconditioner + FP64 refinement): ") + aao_status_str(worst);
  return worst;
}

// Parameter-dependent host tables of a handle for (tau, alpha, c2): the per-frequency
// terms of Sigma (wq, 2n), D_alpha^{-1} and D_alpha^2 (n each) and Lambda (m), computed in
// long double and rounded; also sets the plan's tau, alpha, c2 and stencil coefficient.
void param_tables(Plan& P, double tau, double alpha, double c2, double2* wq, double* dinv, double* d2,
                  double* lam, float* lm1_32 = nullptr) {
  const int nt = P.n, M = P.M;
  P.tau = tau;
  P.alpha = alpha;
  P.c2 = c2;
  P.coef = c2 * tau * tau / (2.0 * P.h * P.h);
  const long double pi = 3.141592653589793238462643383279502884L;
  const long double la = logl((long double)alpha);
  {
    // per-frequency terms of Sigma = (1 - a theta^k)^2 + (Lambda - 1)(1 + a^2 theta^{2k})
    const long double a = expl(la / nt), one_minus_a = -expm1l(la / nt);
    for (int k = 0; k < nt; ++k) {
      const long double phi = 2.0L * pi * (long double)k / (long double)nt;
      const long double sh = sinl(phi / 2.0L), c = cosl(phi), sn = sinl(phi);
      const long double wr = one_minus_a + 2.0L * a * sh * sh, wi = -a * sn;
      wq[2 * k] = make_double2((double)((wr - wi) * (wr + wi)), (double)(2.0L * wr * wi));
      const long double qr = one_minus_a * (1.0L + a) + 2.0L * a * a * c * c;
      wq[2 * k + 1] = make_double2((double)qr, (double)(2.0L * a * a * sn * c));
    }
  }
  for (int t = 0; t < nt; ++t) {
    dinv[t] = (double)expl(-la * (long double)t / (long double)nt);
    d2[t] = (double)expl(2.0L * la * (long double)t / (long double)nt);
  }
  // Lambda_s = 1 + (c2 tau^2/2) sum_axes mu(i_axis), lexicographic s (x fastest)
  const long double hl = 1.0L / (long double)M;
  std::vector<long double> mul(P.N);
  for (int i = 0; i < P.N; ++i) {
    const long double sv = sinl((long double)(i + 1) * pi * hl / 2.0L);
    mul[i] = 4.0L / (hl * hl) * sv * sv;
  }
  const long double ct = 0.5L * (long double)c2 * (long double)tau * (long double)tau;
  for (long long s_ = 0; s_ < P.m; ++s_) {
    long long rest = s_;
    long double sum = 0.0L;
    for (int ax = 0; ax < P.d; ++ax) { sum += mul[rest % P.N]; rest /= P.N; }
    lam[(size_t)s_] = (double)(1.0L + ct * sum);
    if (lm1_32) lm1_32[(size_t)s_] = (float)(ct * sum);  // Lambda_s - 1 without cancellation
  }
}

// Device side of a (re-)bind, stream-ordered on s from host arrays (pinned for a truly
// asynchronous copy): uploads, the spectral table (and its double-float split), and the
// per-block min/max |Sigma| copied to mm_host (nblocks pairs).
aao_status bind_tables(aao_handle* h, const double2* wq, const double* dinv, const double* d2,
                       const double* lam, const float* dinv32, const float* d232, const float2* wq32,
                       const float* lm132, const dfl* dinv_ff,
                       const dfl* d2_ff, double* mm_host, int* nblocks, cudaStream_t s) {
  Plan& P = h->P;
  const size_t nt = (size_t)P.n;
  const bool fp32 = (h->precision == AAO_PREC_FP32_IR);
  AAO_CK(cudaMemcpyAsync(h->dinv64, dinv, nt * sizeof(double), cudaMemcpyHostToDevice, s));
  AAO_CK(cudaMemcpyAsync(h->d264, d2, nt * sizeof(double), cudaMemcpyHostToDevice, s));
  AAO_CK(cudaMemcpyAsync(h->d_wq, wq, 2 * nt * sizeof(double2), cudaMemcpyHostToDevice, s));
  AAO_CK(cudaMemcpyAsync(h->lam64, lam, (size_t)P.m * sizeof(double), cudaMemcpyHostToDevice, s));
  if (fp32) {
    AAO_CK(cudaMemcpyAsync(h->dinv32, dinv32, nt * sizeof(float), cudaMemcpyHostToDevice, s));
    AAO_CK(cudaMemcpyAsync(h->d232, d232, nt * sizeof(float), cudaMemcpyHostToDevice, s));
    AAO_CK(cudaMemcpyAsync(h->wq32, wq32, 2 * nt * sizeof(float2), cudaMemcpyHostToDevice, s));
    AAO_CK(cudaMemcpyAsync(h->lm132, lm132, (size_t)P.m * sizeof(float), cudaMemcpyHostToDevice, s));
  }
  if (h->precision == AAO_PREC_F32X2) {
    AAO_CK(cudaMemcpyAsync(h->dinv_ff, dinv_ff, nt * sizeof(dfl), cudaMemcpyHostToDevice, s));
    AAO_CK(cudaMemcpyAsync(h->d2_ff, d2_ff, nt * sizeof(dfl), cudaMemcpyHostToDevice, s));
  }
  AAO_CK(launch_spectral_table(P, h->d_mu, h->d_wq, h->ab64, fp32 ? h->ab32 : nullptr, h->d_mm, nblocks,
                               s, &h->launches));
  if (h->precision == AAO_PREC_F32X2)
    AAO_CK(launch_split_df(h->ab64, h->ab_ff, (size_t)(P.n / 2 + 1) * P.npairs * 2, s, &h->launches));
  AAO_CK(cudaMemcpyAsync(mm_host, h->d_mm, (size_t)2 * *nblocks * sizeof(double), cudaMemcpyDeviceToHost, s));
  return AAO_OK;
}

// min |Sigma| against max |Sigma| from the per-block pairs (Remark c1badperformremark)
aao_status check_sigma(const double* mm, int nb) {
  double smin = 1e300, smax = 0.0;
  for (int i = 0; i < nb; ++i) {
    smin = std::min(smin, mm[2 * i]);
    smax = std::max(smax, mm[2 * i + 1]);
  }
  if (!(smin > 1e-12 * smax))
    return fail(AAO_ESINGULAR, "min |Sigma| / max |Sigma| = " + std::to_string(smin / smax) +
                                   " below 1e-12: preconditioner singular");
  return AAO_OK;
}

// Parameter-dependent tables of a handle: D_alpha, D_alpha^2, the per-frequency terms
// of Sigma, Lambda, and the spectral table (built on the device); checks min |Sigma|.
// Used by aao_create (synchronous on stream s).
aao_status set_params(aao_handle* h, double tau, double alpha, double c2, cudaStream_t s) {
  Plan& P = h->P;
  const int nt = P.n;
  std::vector<double2> wq(2 * (size_t)nt);
  std::vector<double> dinv(nt), d2(nt), lam((size_t)P.m);
  std::vector<float> lm132((size_t)P.m);
  param_tables(P, tau, alpha, c2, wq.data(), dinv.data(), d2.data(), lam.data(), lm132.data());
  const std::vector<float> dinv32 = to_f(dinv), d232 = to_f(d2);
  const std::vector<float2> wq32 = to_f2(wq);
  const std::vector<dfl> dinv_ff = to_df(dinv), d2_ff = to_df(d2);
  std::vector<double> mm((size_t)2 * h->mm_blocks);
  int nb = 0;
  AAO_TRY(bind_tables(h, wq.data(), dinv.data(), d2.data(), lam.data(), dinv32.data(), d232.data(), wq32.data(),
                      lm132.data(),
                      dinv_ff.data(), d2_ff.data(), mm.data(), &nb, s));
  AAO_CK(cudaStreamSynchronize(s));  // pageable host arrays: wait before they go
  return check_sigma(mm.data(), nb);
}

aao_status get_graph(const MinresCtx& c, int use_x0, cudaGraphExec_t* out) {
  aao_handle* h = c.h;
  const long key = ((long)c.nrhs << 8) | (use_x0 ? 1 : 0) | (c.true_res ? 2 : 0) | (c.physical ? 4 : 0) |
                   ((c.bh == h->vr) ? 8 : 0);
  for (auto& gc : h->graphs)
    if (gc.key == key) {  // rtol and maxit are device parameters of the graph
      *out = gc.exec;
      h->last_init_kernels = gc.init_kernels;
      h->last_body_kernels = gc.body_kernels;
      return AAO_OK;
    }
  AAO_TRY(build_graph(c, use_x0, out));
  h->graphs.push_back(aao_handle::GraphCache{key, c.rtol, c.maxit, *out, h->last_init_kernels,
                                             h->last_body_kernels});
  return AAO_OK;
}

}  // namespace

// ---- internal entry points for the serving runtime (aao_serve.cu) ----
aao_status aaoi_rebind(aao_handle* h, double tau, double alpha, double c2) {
  if (!h) return fail(AAO_EINVAL, "null handle");
  if (!(tau > 0.0) || !(alpha > 0.0 && alpha <= 1.0) || !(c2 > 0.0))
    return fail(AAO_EINVAL, "bad tau/alpha/c2");
  AAO_CK(cudaSetDevice(h->device));
  return set_params(h, tau, alpha, c2, h->own_stream);
}

// Enqueue one complete FP64 solve (DST of b, the graph-captured MINRES, DST back,
// physical residual) on stream s without waiting; aaoi_solve_collect reads the result
// once the stream has reached the end of this work.
aao_status aaoi_solve_enqueue(aao_handle* h, const double* b, double* x, double rtol, int maxit,
                              cudaStream_t s) {
  if (!h || !b || !x) return fail(AAO_EINVAL, "null pointer");
  if ((h->precision != AAO_PREC_FP64 && h->precision != AAO_PREC_F32X2) || h->var_on || !h->use_graph)
    return fail(AAO_EINVAL, "asynchronous solves need an FP64 or double-float, constant-coefficient, graph handle");
  AAO_TRY(dst_apply(h, b, h->vbh, 1, s));
  MinresCtx c{h, h->vbh, h->vxh, 1, rtol, maxit, s, true, false};
  cudaGraphExec_t ex = nullptr;
  AAO_TRY(get_graph(c, 0, &ex));
  AAO_CK(launch_set_params(h->d_prm, rtol, maxit, s, &h->launches));
  AAO_CK(cudaGraphLaunch(ex, s));
  AAO_CK(cudaMemcpyAsync(h->sc_host, h->sc, sizeof(MinresScalars), cudaMemcpyDeviceToHost, s));
  AAO_CK(cudaMemcpyAsync(h->trips_host, h->d_trips, sizeof(int), cudaMemcpyDeviceToHost, s));
  AAO_TRY(dst_apply(h, h->vxh, x, 1, s));
  double* p1 = h->partial;
  double* p2 = h->partial + (size_t)h->nrhs_max * h->partial_stride;
  int nb = 0;
  AAO_CK(launch_op(h, x, nullptr, b, p1, 2, 1, s, &nb));
  AAO_CK(launch_dot(h->P, b, b, p2, 1, s, &h->launches));
  AAO_CK(launch_relres(p1, nb, p2, dot_blocks_per_rhs(h->P), h->relres_dev, 1, s, &h->launches));
  AAO_CK(cudaMemcpyAsync(h->relres_host, h->relres_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
  return AAO_OK;
}

// DST default: the FP64 DST is bound by the FP64 pipe (radix-16 plan; the other axes
// change nothing); the double-float DSTs (the handle's DSTs in the other modes) gain from
// batched loads and the interleaved shared-memory layout (measured on GB300: 0.660 ->
// 0.622 ms for both axes at 255^2 x 256, 5.02 -> 4.56 ms at 511^2 x 512).
static int default_dst_variant(int precision) { return precision == AAO_PREC_FP64 ? 1 : 7; }

// Small problems: where the standard tiles give fewer CTAs than a quarter of the 152
// SMs, kernels with smaller tiles spread the work wider (1D 63 x 64: the time pipeline
// and the DST run on 16 CTAs instead of 1, the operator on 16 instead of 2): the
// one-warp time and DST tiles (when even the half tile -- 2048/n mode pairs, 2048/(N+1)
// line pairs -- is too coarse), short stencil runs, the small w/x update shape.
static void choose_small_tiles(Plan& P) {
  constexpr long long few = 152 / 4;
  const int nt = P.n, M = P.M;
  if ((P.npairs + 2048 / nt - 1) / (2048 / nt) < few)
    P.time_variant64 = P.time_variant32 = P.time_variant_ff = TIME_VARIANT_SMALL;
  const long long lines = (long long)nt * P.m / P.N, ns = 2048 / M;
  if ((lines + 2 * ns - 1) / (2 * ns) < few) P.dst_variant = DST_VARIANT_SMALL;
  if ((long long)((P.m + YT_THREADS - 1) / YT_THREADS) * ((nt + YT_CH_STD - 1) / YT_CH_STD) < few)
    P.yt_ch = YT_CH_SMALL;
  if ((P.m + 31) / 32 < few) P.wx_small = 1;
}

// Back to the standard tiles (the variants of a handle created without small tiles).
static void use_standard_tiles(Plan& P, int precision) {
  const Plan standard;
  if (P.time_variant64 == TIME_VARIANT_SMALL) P.time_variant64 = standard.time_variant64;
  if (P.time_variant32 == TIME_VARIANT_SMALL) P.time_variant32 = standard.time_variant32;
  if (P.time_variant_ff == TIME_VARIANT_SMALL) P.time_variant_ff = standard.time_variant_ff;
  if (P.dst_variant == DST_VARIANT_SMALL) P.dst_variant = default_dst_variant(precision);
  P.yt_ch = standard.yt_ch;
  P.wx_small = standard.wx_small;
}

// ---- grouped serving (aao_serve.cu): one problem per handle, iterations run by grouped launches ----
aao_status aaoi_serving_prepare(aao_handle* h) {
  if (!h) return fail(AAO_EINVAL, "null handle");
  if (h->pin) return AAO_OK;
  // served problems run their iterations in grouped launches, which take the standard
  // tiles: a small problem keeps them too (its CTAs share the grouped grid)
  use_standard_tiles(h->P, h->precision);
  const Plan& P = h->P;
  const size_t nt = (size_t)P.n;
  const size_t bytes = 2 * nt * sizeof(double2) + 2 * nt * sizeof(double) + (size_t)P.m * sizeof(double) +
                       2 * nt * sizeof(dfl) + (size_t)2 * h->mm_blocks * sizeof(double) + 64;
  AAO_CK(cudaSetDevice(h->device));
  AAO_CK(cudaMallocHost(&h->pin, bytes));
  char* q = static_cast<char*>(h->pin);
  auto carve = [&](size_t b) { char* r = q; q += (b + 15) & ~size_t(15); return r; };
  h->pin_wq = reinterpret_cast<double2*>(carve(2 * nt * sizeof(double2)));
  h->pin_dinv = reinterpret_cast<double*>(carve(nt * sizeof(double)));
  h->pin_d2 = reinterpret_cast<double*>(carve(nt * sizeof(double)));
  h->pin_dinv_ff = reinterpret_cast<dfl*>(carve(nt * sizeof(dfl)));
  h->pin_d2_ff = reinterpret_cast<dfl*>(carve(nt * sizeof(dfl)));
  h->pin_mm = reinterpret_cast<double*>(carve((size_t)2 * h->mm_blocks * sizeof(double)));
  h->pin_lam = reinterpret_cast<double*>(carve((size_t)P.m * sizeof(double)));
  return AAO_OK;
}

// Re-bind to (tau, alpha, c2) stream-ordered on s with no host synchronisation: host
// tables into the pinned staging, then bind_tables; the |Sigma| check waits for
// aaoi_group_collect.  The caller guarantees the staging is no longer in use (the
// handle's previous solve has completed).
aao_status aaoi_rebind_async(aao_handle* h, double tau, double alpha, double c2, cudaStream_t s) {
  if (!h || !h->pin) return fail(AAO_EINVAL, "handle not prepared for serving");
  if (!(tau > 0.0) || !(alpha > 0.0 && alpha <= 1.0) || !(c2 > 0.0)) return fail(AAO_EINVAL, "bad tau/alpha/c2");
  if (h->precision != AAO_PREC_FP64 && h->precision != AAO_PREC_F32X2)
    return fail(AAO_EINVAL, "served precision must be FP64 or double-float");
  Plan& P = h->P;
  param_tables(P, tau, alpha, c2, h->pin_wq, h->pin_dinv, h->pin_d2, h->pin_lam);
  if (h->precision == AAO_PREC_F32X2)
    for (int t = 0; t < P.n; ++t) {
      h->pin_dinv_ff[t] = dfl(h->pin_dinv[t]);
      h->pin_d2_ff[t] = dfl(h->pin_d2[t]);
    }
  return bind_tables(h, h->pin_wq, h->pin_dinv, h->pin_d2, h->pin_lam, nullptr, nullptr, nullptr, nullptr,
                     h->pin_dinv_ff, h->pin_d2_ff, h->pin_mm, &h->pin_nb, s);
}

// b = Y f, b^ = (I (x) U) b and the MINRES initialisation from a zero guess (no graph),
// stream-ordered on s; afterwards iteration j runs on the buffers of parity j & 1.
aao_status aaoi_group_begin(aao_handle* h, const double* f, const double* psi0, const double* psi1, double* b,
                            double rtol, int maxit, cudaStream_t s) {
  if (!h || !f || !psi0 || !psi1 || !b) return fail(AAO_EINVAL, "null pointer");
  AAO_KL(h, KC_RHS, s, launch_rhs(h, f, psi0, psi1, b, 1, s));
  AAO_TRY(dst_apply(h, b, h->vbh, 1, s));
  MinresCtx c{h, h->vbh, h->vxh, 1, rtol, maxit, s, true, false};
  const MinresBufs B0{h->vv, h->vvp, h->vz, h->vzn, h->vw, h->vwp};
  return minres_enqueue_init(c, 0, B0);
}

static MinresBufs group_bufs(aao_handle* h, int parity) {
  const MinresBufs B0{h->vv, h->vvp, h->vz, h->vzn, h->vw, h->vwp};
  return parity ? rotate(B0) : B0;
}

void aaoi_group_problem(aao_handle* h, int parity, GroupProblem* gp) {
  const Plan& P = h->P;
  const MinresBufs B = group_bufs(h, parity);
  gp->z = B.z; gp->T = h->vT; gp->v = B.v; gp->vp = B.vp; gp->zn = B.zn; gp->w = B.w; gp->wp = B.wp;
  gp->x = h->vxh; gp->b = h->vbh; gp->lam = h->lam64; gp->sc = h->sc; gp->partial = h->partial;
  gp->n = P.n; gp->m = P.m;
  gp->yt_gx = group_yt_tiles(P.m);
  gp->nb_dot = dot_blocks_per_rhs(P);
  gp->nb_vu = group_vu_blocks(P.n, P.m);
}

int aaoi_precision(const aao_handle* h) { return h->precision; }
int aaoi_nt(const aao_handle* h) { return h->P.n; }
int aaoi_modes(const aao_handle* h) { return h->P.m; }
int aaoi_time_variant(const aao_handle* h) {
  return h->precision == AAO_PREC_F32X2 ? h->P.time_variant_ff : h->P.time_variant64;
}

void aaoi_time_entry64(aao_handle* h, int parity, TimeGroupEntry<double>* e) {
  const MinresBufs B = group_bufs(h, parity);
  e->in = B.vp; e->out = B.zn; e->sc = h->sc; e->m = h->P.m; e->npairs = h->P.npairs; e->tb = h->P.t64;
}
void aaoi_time_entry_ff(aao_handle* h, int parity, TimeGroupEntry<dfl>* e) {
  const MinresBufs B = group_bufs(h, parity);
  e->in = B.vp; e->out = B.zn; e->sc = h->sc; e->m = h->P.m; e->npairs = h->P.npairs; e->tb = h->P.tff;
}

// the time step of iteration `parity` as a solo launch (variants without a grouped form)
aao_status aaoi_group_time_solo(aao_handle* h, int parity, cudaStream_t s) {
  const MinresBufs B = group_bufs(h, parity);
  return time_apply(h, B.vp, B.zn, 1, s);
}

// x = (I (x) U) x^, the physical residual ||b - Y T x|| / ||b|| and the copies of the
// scalars and the residual to the handle's pinned mirrors, stream-ordered on s
aao_status aaoi_group_end(aao_handle* h, const double* b, double* x, cudaStream_t s) {
  AAO_TRY(dst_apply(h, h->vxh, x, 1, s));
  double* p1 = h->partial;
  double* p2 = h->partial + (size_t)h->nrhs_max * h->partial_stride;
  int nb = 0;
  AAO_CK(launch_op(h, x, nullptr, b, p1, 2, 1, s, &nb));
  AAO_CK(launch_dot(h->P, b, b, p2, 1, s, &h->launches));
  AAO_CK(launch_relres(p1, nb, p2, dot_blocks_per_rhs(h->P), h->relres_dev, 1, s, &h->launches));
  AAO_CK(cudaMemcpyAsync(h->sc_host, h->sc, sizeof(MinresScalars), cudaMemcpyDeviceToHost, s));
  AAO_CK(cudaMemcpyAsync(h->relres_host, h->relres_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
  return AAO_OK;
}

// after the stream passed aaoi_group_end: the request's result
aao_status aaoi_group_collect(aao_handle* h, double rtol, aao_solve_info* info) {
  aao_status st = minres_collect(h, 1, info);
  info->relres_true = h->relres_host[0];
  if (info->relres_true > rtol && info->status == AAO_OK) info->status = AAO_ENOTCONV;
  if (h->pin_nb > 0) {
    const aao_status sg = check_sigma(h->pin_mm, h->pin_nb);
    h->pin_nb = 0;
    if (sg != AAO_OK) info->status = sg;
  }
  if (info->status != AAO_OK && st == AAO_OK) st = (aao_status)info->status;
  if (info->status != AAO_OK) st = (aao_status)info->status;
  return st;
}

aao_status aaoi_solve_collect(aao_handle* h, double rtol, aao_solve_info* info) {
  h->launches += h->last_init_kernels + (uint64_t)(*h->trips_host) * h->last_body_kernels;
  aao_status st = minres_collect(h, 1, info);
  info->relres_true = h->relres_host[0];
  if (info->relres_true > rtol && info->status == AAO_OK) info->status = AAO_ENOTCONV;
  if (info->status != AAO_OK && st == AAO_OK) st = (aao_status)info->status;
  return st;
}

size_t aaoi_estimate_bytes(int dim, int N, int nt, int precision) {
  size_t m = 1;
  for (int i = 0; i < dim; ++i) m *= (size_t)N;
  const size_t npairs = (m + 1) / 2;
  const size_t vec = (size_t)nt * m * sizeof(double);
  const size_t nbyt = std::max(((m + 255) / 256) * (((size_t)nt + 31) / 32), (m + 31) / 32);
  const size_t table = (size_t)(nt / 2 + 1) * npairs * 2 * sizeof(double2);  // FP64 (and dfl2) table
  return 9 * vec + (precision == AAO_PREC_F32X2 ? 2 : 1) * table + m * sizeof(double) +
         3 * std::max(nbyt, (size_t)296) * sizeof(double) + (1 << 16);
}

extern "C" {

const char* aao_status_str(aao_status s) {
  switch (s) {
    case AAO_OK: return "AAO_OK";
    case AAO_EINVAL: return "AAO_EINVAL";
    case AAO_EUNSUPPORTED: return "AAO_EUNSUPPORTED";
    case AAO_ENOMEM: return "AAO_ENOMEM";
    case AAO_ECUDA: return "AAO_ECUDA";
    case AAO_ENOTCONV: return "AAO_ENOTCONV";
    case AAO_EBREAKDOWN: return "AAO_EBREAKDOWN";
    case AAO_ESINGULAR: return "AAO_ESINGULAR";
    case AAO_EBUSY: return "AAO_EBUSY";
    case AAO_EPENDING: return "AAO_EPENDING";
    case AAO_ETIMEOUT: return "AAO_ETIMEOUT";
  }
  return "AAO_UNKNOWN";
}

const char* aao_last_error(void) { return g_err.c_str(); }

// A time-kernel variant number of a precision mode, or the small-tile variant (any
// other number is folded onto the range the mode has).
static int clamp_time_variant(int v, int prec) {
  if (v == TIME_VARIANT_SMALL) return v;
  if (prec == AAO_PREC_FP32_IR) return v >= 0 && v < 34 ? v : v & 31;
  return v & (prec == AAO_PREC_FP64 ? 7 : 15);
}
static int clamp_dst_variant(int v) { return v == DST_VARIANT_SMALL ? v : v & 7; }

aao_status aao_create(const aao_grid* grid, int nt, double tau, double alpha, aao_scheme scheme,
                      const aao_opts* opts, aao_handle** out) {
  g_err.clear();
  if (!grid || !out) return fail(AAO_EINVAL, "null grid or out pointer");
  *out = nullptr;
  if (grid->dim < 1 || grid->dim > 3) return fail(AAO_EINVAL, "dim must be 1, 2 or 3");
  if (!(tau > 0.0) || !std::isfinite(tau)) return fail(AAO_EINVAL, "tau must be > 0");
  if (!(alpha > 0.0 && alpha <= 1.0)) return fail(AAO_EINVAL, "alpha must be in (0, 1]");
  if (!(grid->c2 > 0.0) || !std::isfinite(grid->c2)) return fail(AAO_EINVAL, "c2 must be > 0");
  if (scheme != AAO_SCHEME_IMPLICIT_LEAPFROG) return fail(AAO_EINVAL, "unknown scheme");
  if (nt < 2) return fail(AAO_EINVAL, "nt must be >= 2");
  const int M = grid->N + 1;
  if (!is_pow2(M) || M < 64 || M > 512)
    return fail(AAO_EUNSUPPORTED, "N+1 must be a power of two in [64, 512]");
  if (!is_pow2(nt) || nt < 64 || nt > 1024)
    return fail(AAO_EUNSUPPORTED, "nt must be a power of two in [64, 1024]");
  aao_opts o{};
  o.precision = AAO_PREC_FP64;
  o.nrhs_max = 1;
  if (opts) o = *opts;
  if (o.nrhs_max < 1) o.nrhs_max = 1;
  if (o.precision != AAO_PREC_FP64 && o.precision != AAO_PREC_FP32_IR && o.precision != AAO_PREC_F32X2)
    return fail(AAO_EINVAL, "unknown precision");
  for (int i = 0; i < 3; ++i)
    if (o.reserved[i] != 0) return fail(AAO_EINVAL, "opts.reserved must be zero");

  aao_handle* h = new aao_handle();
  cudaGetDevice(&h->device);
  if (cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    h->own_stream = nullptr;
    delete h;
    return fail(AAO_ECUDA, "cudaStreamCreate failed");
  }
  h->precision = o.precision;
  h->nrhs_max = o.nrhs_max;
  Plan& P = h->P;
  P.d = grid->dim;
  P.N = grid->N;
  P.M = M;
  P.n = nt;
  P.m = 1;
  for (int i = 0; i < P.d; ++i) P.m *= P.N;
  P.npairs = (P.m + 1) / 2;
  P.tau = tau;
  P.alpha = alpha;
  P.c2 = grid->c2;
  P.h = 1.0 / (double)M;
  P.coef = P.c2 * tau * tau / (2.0 * P.h * P.h);
  P.dst_variant = default_dst_variant(o.precision);
  {
    const char* st_env = getenv("AAO_SMALL_TILES");
    if (!st_env || atoi(st_env) != 0) choose_small_tiles(P);
  }
  if (const char* tv = getenv("AAO_TIME_VARIANT")) {  // tuning override: "v64,v32,vff"
    int a = 0, b = -1;
    int c = -1;
    if (sscanf(tv, "%d,%d,%d", &a, &b, &c) >= 1) {
      P.time_variant64 = clamp_time_variant(a, AAO_PREC_FP64);
      P.time_variant32 = clamp_time_variant(b >= 0 ? b : a, AAO_PREC_FP32_IR);
      P.time_variant_ff = clamp_time_variant(c >= 0 ? c : (b >= 0 ? b : a), AAO_PREC_F32X2);
    }
  }
  if (const char* dv = getenv("AAO_DST_VARIANT")) P.dst_variant = clamp_dst_variant(atoi(dv));

  auto bail = [&](aao_status st) { delete h; return st; };

  // ---- static host tables (long double, rounded): twiddles, DST weights, 1D eigenvalues ----
  const long double pi = 3.141592653589793238462643383279502884L;
  std::vector<double2> twS, twT;
  host_twiddles(M, -1, twS);
  host_twiddles(nt, -1, twT);
  std::vector<double> sinw(M / 2 + 1), mu(P.N);
  const long double cM = sqrtl(2.0L / (long double)M);
  for (int j = 0; j <= M / 2; ++j) sinw[j] = (double)(cM * sinl(pi * j / (long double)M) / 2.0L);
  const long double hl = 1.0L / (long double)M;
  for (int i = 0; i < P.N; ++i) {
    const long double sv = sinl((long double)(i + 1) * pi * hl / 2.0L);
    mu[i] = (double)(4.0L / (hl * hl) * sv * sv);
  }

  // ---- device allocations ----
  aao_status st;
  const size_t tabn = (size_t)(nt / 2 + 1) * P.npairs * 2;
  const long long ntab = (long long)(nt / 2 + 1) * P.npairs;
  h->mm_blocks = (int)((ntab + 255) / 256);
  if ((st = h->alloc(&h->tw_space64, M)) || (st = h->alloc(&h->sinw64, M / 2 + 1)) ||
      (st = h->alloc(&h->tw_time64, nt)) || (st = h->alloc(&h->dinv64, nt)) ||
      (st = h->alloc(&h->d264, nt)) || (st = h->alloc(&h->ab64, tabn)) ||
      (st = h->alloc(&h->d_mu, P.N)) || (st = h->alloc(&h->d_wq, 2 * (size_t)nt)) ||
      (st = h->alloc(&h->d_mm, (size_t)2 * h->mm_blocks)))
    return bail(st);
  const bool fp32 = (o.precision == AAO_PREC_FP32_IR);
  const bool ff = (o.precision == AAO_PREC_F32X2);
  const bool ff_dst = ff || fp32;  // double-float DSTs (see dst_apply)
  if (ff_dst) {
    if ((st = h->alloc(&h->tw_space_ff, M)) || (st = h->alloc(&h->sinw_ff, M / 2 + 1))) return bail(st);
  }
  if (ff) {
    if ((st = h->alloc(&h->tw_time_ff, nt)) || (st = h->alloc(&h->dinv_ff, nt)) ||
        (st = h->alloc(&h->d2_ff, nt)) || (st = h->alloc(&h->ab_ff, tabn)))
      return bail(st);
  }
  if (fp32) {
    if ((st = h->alloc(&h->tw_space32, M)) || (st = h->alloc(&h->sinw32, M / 2 + 1)) ||
        (st = h->alloc(&h->tw_time32, nt)) || (st = h->alloc(&h->dinv32, nt)) ||
        (st = h->alloc(&h->d232, nt)) || (st = h->alloc(&h->ab32, tabn)) ||
        (st = h->alloc(&h->wq32, 2 * (size_t)nt)) || (st = h->alloc(&h->lm132, (size_t)P.m)))
      return bail(st);
  }
  const size_t vl = (size_t)h->nrhs_max * (size_t)nt * P.m;
  if ((st = h->alloc(&h->vT, vl)) || (st = h->alloc(&h->vv, vl)) || (st = h->alloc(&h->vvp, vl)) ||
      (st = h->alloc(&h->vz, vl)) || (st = h->alloc(&h->vzn, vl)) || (st = h->alloc(&h->vw, vl)) ||
      (st = h->alloc(&h->vwp, vl)) || (st = h->alloc(&h->vbh, vl)) || (st = h->alloc(&h->vxh, vl)) ||
      (st = h->alloc(&h->lam64, (size_t)P.m)) || (st = h->alloc(&h->relres_dev, (size_t)h->nrhs_max)))
    return bail(st);
  if (o.graph) {
    h->use_graph = true;
    if ((st = h->alloc(&h->d_trips, 1)) || (st = h->alloc(&h->d_prm, 2))) return bail(st);
    if (cudaMallocHost(&h->trips_host, sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      h->trips_host = nullptr;
      return bail(fail(AAO_ENOMEM, "cudaMallocHost failed"));
    }
    *h->trips_host = 0;
    if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return bail(fail(AAO_ECUDA, "cudaStreamCreate failed"));
    }
  }
  if (o.variable_coefficient) {
    size_t fsz = (size_t)P.d * (P.N + 1);
    for (int i = 1; i < P.d; ++i) fsz *= P.N;
    if ((st = h->alloc(&h->face, fsz))) return bail(st);
  }
  if (fp32) {  // refinement vectors and the FP32 buffer of aao_apply_prec
    if ((st = h->alloc(&h->vr, vl)) || (st = h->alloc(&h->vdx, vl)) || (st = h->alloc(&h->f32, vl)))
      return bail(st);
  }
  if (o.host_staging && (st = reserve_host_staging(h))) return bail(st);
  h->partial_stride = std::max(std::max(yt_blocks_per_rhs(P), dot_blocks_per_rhs(P)), wxres_blocks_per_rhs(P));
  if ((st = h->alloc(&h->partial, (size_t)3 * h->nrhs_max * h->partial_stride)) ||
      (st = h->alloc(&h->sc, (size_t)h->nrhs_max)) || (st = h->alloc(&h->arrive, (size_t)h->nrhs_max + 1)))
    return bail(st);
  if (const char* fz = getenv("AAO_FUSED_SCALARS")) h->fuse_scalars = atoi(fz) != 0;
  if (cudaMallocHost(&h->sc_host, sizeof(MinresScalars) * h->nrhs_max) != cudaSuccess ||
      cudaMallocHost(&h->relres_host, sizeof(double) * h->nrhs_max) != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(AAO_ENOMEM, "cudaMallocHost failed"));
  }

  auto run = [&]() -> aao_status {
    const cudaStream_t os = h->own_stream;
    AAO_CK(cudaMemsetAsync(h->arrive, 0, ((size_t)h->nrhs_max + 1) * sizeof(unsigned), os));
    AAO_TRY(upload_on(twS, h->tw_space64, os));
    AAO_TRY(upload_on(sinw, h->sinw64, os));
    AAO_TRY(upload_on(twT, h->tw_time64, os));
    AAO_TRY(upload_on(mu, h->d_mu, os));
    if (fp32) {
      AAO_TRY(upload_on(to_f2(twS), h->tw_space32, os));
      AAO_TRY(upload_on(to_f(sinw), h->sinw32, os));
      AAO_TRY(upload_on(to_f2(twT), h->tw_time32, os));
    }
    P.t64.tw_space = h->tw_space64; P.t64.sinw = h->sinw64; P.t64.tw_time = h->tw_time64;
    P.t64.dinv = h->dinv64; P.t64.d2 = h->d264; P.t64.ab = h->ab64;
    P.t64.cq = (double)(cM / 4.0L);
    if (fp32) {
      P.t32.tw_space = h->tw_space32; P.t32.sinw = h->sinw32; P.t32.tw_time = h->tw_time32;
      P.t32.dinv = h->dinv32; P.t32.d2 = h->d232; P.t32.ab = h->ab32;
      P.t32.wq = h->wq32; P.t32.lm1 = h->lm132; P.t32.inv2n = (float)(1.0 / (2.0 * nt));
      P.t32.cq = (float)(cM / 4.0L);
    }
    if (ff_dst) {
      AAO_TRY(upload_on(to_df2(twS), h->tw_space_ff, os));
      AAO_TRY(upload_on(to_df(sinw), h->sinw_ff, os));
      P.tff.tw_space = h->tw_space_ff; P.tff.sinw = h->sinw_ff;
      P.tff.cq = dfl((double)(cM / 4.0L));
    }
    if (ff) {
      AAO_TRY(upload_on(to_df2(twT), h->tw_time_ff, os));
      P.tff.tw_time = h->tw_time_ff; P.tff.dinv = h->dinv_ff; P.tff.d2 = h->d2_ff; P.tff.ab = h->ab_ff;
    }
    AAO_TRY(set_params(h, tau, alpha, grid->c2, os));
    AAO_CK(cudaStreamSynchronize(os));  // this handle's work only, not the whole device
    return AAO_OK;
  };
  st = run();
  if (st != AAO_OK) return bail(st);
  *out = h;
  return AAO_OK;
}

// the time-kernel variant field used by a precision mode
static int& tvar(Plan& P, int prec) {
  return prec == AAO_PREC_FP64 ? P.time_variant64 : prec == AAO_PREC_F32X2 ? P.time_variant_ff : P.time_variant32;
}

aao_status aao_autotune(aao_handle* h, const char* tune_file, int* chosen) {
  AAO_TRY(check_handle(h));
  AAO_CK(cudaSetDevice(h->device));
  Plan& P = h->P;
  const int prec = h->precision;
  if (tune_file) {  // cached choice?
    if (FILE* fh = fopen(tune_file, "r")) {
      int d, N, n, pr, tv, dv;
      bool found = false;
      while (fscanf(fh, "%d %d %d %d %d %d", &d, &N, &n, &pr, &tv, &dv) == 6)
        if (d == P.d && N == P.N && n == P.n && pr == prec) {
          tvar(P, prec) = clamp_time_variant(tv, prec);
          P.dst_variant = clamp_dst_variant(dv);
          found = true;
        }
      fclose(fh);
      if (found) {
        if (chosen) {
          chosen[0] = tvar(P, prec);
          chosen[1] = P.dst_variant;
        }
        AAO_CK(cudaDeviceSynchronize());
        for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
        h->graphs.clear();
        return AAO_OK;
      }
    }
  }
  cudaStream_t s = 0;
  const size_t vb = h->vlen() * sizeof(double);
  AAO_CK(launch_fill_test(h->vv, vb / sizeof(double), s));  // not zeros: see launch_fill_test
  cudaEvent_t e0, e1;
  AAO_CK(cudaEventCreate(&e0));
  AAO_CK(cudaEventCreate(&e1));
  auto timeit = [&](auto&& launch) -> float {
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
      cudaEventRecord(e0, s);
      launch();
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) best = std::min(best, ms);  // first run warms caches and attributes
    }
    return best;
  };
  // The default variants stay unless another is faster by more than 1 % (run-to-run
  // timing noise is a few tenths of a percent; near-ties keep the choice reproducible).
  const int def_tv = tvar(P, prec), def_dv = P.dst_variant;
  // double-float has six more time variants (8..11: interleaved layout, no staged table;
  // 12, 13: 9 and 11 with batched loads), the FP32 pipeline on FP64 vectors sixteen
  // (8..15: the tile staged by bulk copies; 16, 17: variants 5 and 7 with integer
  // conversions; 18..21: with batched loads; 22, 23: 18, 19 with the spectral table
  // computed on the fly instead of read; 24..29: 18, 19 with the store, load or both
  // conversions by integer operations)
  // conversions by integer operations; 31..33: 27, 29, 26 without the staged table
  // slice); every mode also has the small tile (30)
  const int ntv = prec == AAO_PREC_F32X2 ? 15 : prec == AAO_PREC_FP32_IR ? 34 : 8;
  std::vector<int> tvs, dvs = {0, 1, 2, 3, 4, 5, 6, 7, DST_VARIANT_SMALL};
  for (int v = 0; v < ntv; ++v)
    if (v != TIME_VARIANT_SMALL) tvs.push_back(v);
  tvs.push_back(TIME_VARIANT_SMALL);
  auto pick = [](const std::vector<int>& vs, const std::vector<float>& t, int def) {
    size_t b = 0, d = 0;
    for (size_t i = 0; i < vs.size(); ++i) {
      if (t[i] < t[b]) b = i;
      if (vs[i] == def) d = i;
    }
    return t[b] < 0.99f * t[d] ? vs[b] : def;
  };
  std::vector<float> tt(tvs.size()), td(dvs.size());
  for (size_t i = 0; i < tvs.size(); ++i) {
    tvar(P, prec) = tvs[i];
    tt[i] = timeit([&]() {
      if (prec == AAO_PREC_FP64) launch_time<double>(P, h->vv, h->vz, 1, s, nullptr);
      else if (prec == AAO_PREC_F32X2) launch_time_ff(P, h->vv, h->vz, 1, s, nullptr);
      else launch_time_mixed(P, h->vv, h->vz, 1, s, nullptr);
    });
  }
  const int best_tv = pick(tvs, tt, def_tv);
  tvar(P, prec) = best_tv;
  for (size_t i = 0; i < dvs.size(); ++i) {
    P.dst_variant = dvs[i];
    td[i] = timeit([&]() {  // every axis: a variant can suit the contiguous one only
      for (int ax = 0; ax < P.d; ++ax) {
        if (prec == AAO_PREC_F32X2 || prec == AAO_PREC_FP32_IR) launch_dst_axis_ff(P, h->vv, h->vz, ax, 1, s, nullptr);
        else launch_dst_axis<double>(P, h->vv, h->vz, ax, 1, s, nullptr);
      }
    });
  }
  const int best_dv = pick(dvs, td, def_dv);
  P.dst_variant = best_dv;
  if (chosen) {
    chosen[0] = best_tv;
    chosen[1] = best_dv;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  AAO_CK(cudaGetLastError());
  AAO_CK(cudaDeviceSynchronize());
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);  // captured with the old variants
  h->graphs.clear();
  if (tune_file) {
    if (FILE* fh = fopen(tune_file, "a")) {
      fprintf(fh, "%d %d %d %d %d %d\n", P.d, P.N, P.n, prec, best_tv, best_dv);
      fclose(fh);
    }
  }
  return AAO_OK;
}

aao_status aao_set_coefficient(aao_handle* h, const double* a_face, void* stream) {
  AAO_TRY(check_handle(h));
  if (!a_face) return fail(AAO_EINVAL, "null pointer");
  if (!h->face) return fail(AAO_EINVAL, "handle was created without opts.variable_coefficient");
  AAO_CK(cudaSetDevice(h->device));
  size_t fsz = (size_t)h->P.d * (h->P.N + 1);
  for (int i = 1; i < h->P.d; ++i) fsz *= h->P.N;
  AAO_CK(cudaMemcpyAsync(h->face, a_face, fsz * sizeof(double), cudaMemcpyDeviceToDevice,
                         (cudaStream_t)stream));
  h->var_on = true;
  return AAO_OK;
}

aao_status aao_destroy(aao_handle* h) {
  if (!h) return AAO_OK;
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  delete h;
  return AAO_OK;
}

size_t aao_workspace_bytes(const aao_handle* h) { return h ? h->bytes : 0; }

uint64_t aao_launch_count(const aao_handle* h) { return h ? h->launches : 0; }

aao_status aao_profile_enable(aao_handle* h, int on) {
  if (!h) return fail(AAO_EINVAL, "null handle");
  if (on) {
    for (auto& r : h->prof) cudaEventSynchronize(r.b);
    h->clear_prof();
  }
  h->prof_on = (on != 0);
  return AAO_OK;
}

int aao_profile_read(aao_handle* h, aao_kernel_stat* out, int max) {
  if (!h) { fail(AAO_EINVAL, "null handle"); return -1; }
  uint64_t cnt[KC_N] = {0};
  double ms[KC_N] = {0};
  for (auto& r : h->prof) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) { fail(AAO_ECUDA, "event sync failed"); return -1; }
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) { fail(AAO_ECUDA, "event time failed"); return -1; }
    cnt[r.cls] += 1;
    ms[r.cls] += t;
  }
  int n = 0;
  for (int c = 0; c < KC_N; ++c) {
    if (!cnt[c]) continue;
    if (out && n < max) {
      std::memset(out[n].name, 0, sizeof(out[n].name));
      std::strncpy(out[n].name, kc_name(c), sizeof(out[n].name) - 1);
      out[n].launches = cnt[c];
      out[n].total_ms = ms[c];
    }
    ++n;
  }
  return n;
}

aao_status aao_build_rhs(aao_handle* h, const double* f, const double* psi0, const double* psi1,
                         double* b, int nrhs, void* stream) {
  AAO_TRY(check_call(h, nrhs));
  if (!f || !psi0 || !psi1 || !b) return fail(AAO_EINVAL, "null pointer");
  AAO_KL(h, KC_RHS, (cudaStream_t)stream, launch_rhs(h, f, psi0, psi1, b, nrhs, (cudaStream_t)stream));
  return AAO_OK;
}

aao_status aao_apply_op(aao_handle* h, const double* x, double* y, int nrhs, void* stream) {
  AAO_TRY(check_call(h, nrhs));
  if (!x || !y) return fail(AAO_EINVAL, "null pointer");
  if (x == y) return fail(AAO_EINVAL, "x and y must not alias");
  AAO_KL(h, KC_YT, (cudaStream_t)stream, launch_op(h, x, y, nullptr, nullptr, 0, nrhs, (cudaStream_t)stream, nullptr));
  return AAO_OK;
}

aao_status aao_apply_prec(aao_handle* h, const double* r, double* z, int nrhs, void* stream) {
  AAO_TRY(check_call(h, nrhs));
  if (!r || !z) return fail(AAO_EINVAL, "null pointer");
  return prec_apply(h, r, z, nrhs, (cudaStream_t)stream);
}

aao_status aao_apply_dst(aao_handle* h, const double* x, double* y, int nrhs, void* stream) {
  AAO_TRY(check_call(h, nrhs));
  if (!x || !y) return fail(AAO_EINVAL, "null pointer");
  return dst_apply(h, x, y, nrhs, (cudaStream_t)stream);
}

aao_status aao_apply_time(aao_handle* h, const double* x, double* y, int nrhs, void* stream) {
  AAO_TRY(check_call(h, nrhs));
  if (!x || !y) return fail(AAO_EINVAL, "null pointer");
  return time_apply(h, x, y, nrhs, (cudaStream_t)stream);
}

aao_status aao_minres_solve(aao_handle* h, const double* b, double* x, int use_x0, int nrhs,
                            double rtol, int maxit, aao_solve_info* info, void* stream) {
  AAO_TRY(check_call(h, nrhs));
  if (!b || !x) return fail(AAO_EINVAL, "null pointer");
  if (b == x) return fail(AAO_EINVAL, "b and x must not alias");
  if (!(rtol >= 0.0) || maxit < 1) return fail(AAO_EINVAL, "rtol must be >= 0 and maxit >= 1");
  cudaStream_t s = (cudaStream_t)stream;
  if (h->precision == AAO_PREC_FP32_IR) return solve_ir(h, b, x, use_x0, nrhs, rtol, maxit, info, s);
  return solve_fp64(h, b, x, use_x0, nrhs, rtol, maxit, info, s);
}

aao_status aao_residual_norm(aao_handle* h, const double* b, const double* x, double* relres,
                             int nrhs, void* stream) {
  AAO_TRY(check_call(h, nrhs));
  if (!b || !x || !relres) return fail(AAO_EINVAL, "null pointer");
  cudaStream_t s = (cudaStream_t)stream;
  double* p1 = h->partial;
  double* p2 = h->partial + (size_t)h->nrhs_max * h->partial_stride;
  int nb = 0;
  AAO_KL(h, KC_YT_RES, s, launch_op(h, x, nullptr, b, p1, 2, nrhs, s, &nb));
  AAO_KL(h, KC_DOT, s, launch_dot(h->P, b, b, p2, nrhs, s, &h->launches));
  AAO_KL(h, KC_SCAL, s, launch_relres(p1, nb, p2, dot_blocks_per_rhs(h->P), relres, nrhs, s, &h->launches));
  return AAO_OK;
}

aao_status aao_solve_host(aao_handle* h, const double* f, const double* psi0, const double* psi1,
                          double* u, int nrhs, double rtol, int maxit, aao_solve_info* info,
                          void* stream) {
  AAO_TRY(check_call(h, nrhs));
  if (!f || !psi0 || !psi1 || !u) return fail(AAO_EINVAL, "null pointer");
  const Plan& P = h->P;
  if (!h->hs_f) AAO_TRY(reserve_host_staging(h));  // handles created without opts.host_staging
  cudaStream_t s = (cudaStream_t)stream;
  const size_t vb = (size_t)nrhs * h->vlen() * sizeof(double);
  const size_t pb = (size_t)nrhs * P.m * sizeof(double);
  double* d_psi0 = h->hs_psi;
  double* d_psi1 = h->hs_psi + (size_t)h->nrhs_max * P.m;
  if (h->var_on) {  // physical-basis solve: whole-vector copies around it
    AAO_CK(cudaMemcpyAsync(h->hs_f, f, vb, cudaMemcpyHostToDevice, s));
    AAO_CK(cudaMemcpyAsync(d_psi0, psi0, pb, cudaMemcpyHostToDevice, s));
    AAO_CK(cudaMemcpyAsync(d_psi1, psi1, pb, cudaMemcpyHostToDevice, s));
    AAO_KL(h, KC_RHS, s, launch_rhs(h, h->hs_f, d_psi0, d_psi1, h->hs_b, nrhs, s));
    aao_status st = aao_minres_solve(h, h->hs_b, h->hs_x, 0, nrhs, rtol, maxit, info, stream);
    if (st != AAO_OK && st != AAO_ENOTCONV && st != AAO_EBREAKDOWN) return st;
    AAO_CK(cudaMemcpyAsync(u, h->hs_x, vb, cudaMemcpyDeviceToHost, s));
    AAO_CK(cudaStreamSynchronize(s));
    return st;
  }
  if (!(rtol >= 0.0) || maxit < 1) return fail(AAO_EINVAL, "rtol must be >= 0 and maxit >= 1");
  // Pipelined (DST-basis solve): the copies run on a second stream in chunks of CH time
  // levels, so the upload of f overlaps the right-hand side and the forward DSTs of the
  // chunks already there, and the download of x overlaps the inverse DSTs of later
  // chunks.  Every level of the right-hand side and of the DSTs depends on its own f
  // level (and psi0, psi1) only, so chunking changes no value.  The chunks' kernels
  // alternate between two streams: one chunk's DST grid fills only part of the GPU, and
  // two chunks side by side keep it busy.
  const int CH = HOST_CHUNK;
  const int per = P.n / CH, nch = nrhs * per;
  const size_t lb = (size_t)P.m * sizeof(double);
  cudaStream_t cs = h->hs_copy;
  cudaEvent_t* ev = h->hs_ev.data();
  AAO_CK(cudaEventRecord(ev[2 * nch], s));  // the copy stream follows the caller's stream
  AAO_CK(cudaStreamWaitEvent(cs, ev[2 * nch], 0));
  AAO_CK(cudaMemcpyAsync(d_psi0, psi0, pb, cudaMemcpyHostToDevice, cs));
  AAO_CK(cudaMemcpyAsync(d_psi1, psi1, pb, cudaMemcpyHostToDevice, cs));
  for (int c = 0; c < nch; ++c) {  // f chunk c: rhs r, levels k0 .. k0+CH-1
    const size_t off = (size_t)(c / per) * P.n * P.m + (size_t)(c % per) * CH * P.m;
    AAO_CK(cudaMemcpyAsync(h->hs_f + off, f + off, CH * lb, cudaMemcpyHostToDevice, cs));
    AAO_CK(cudaEventRecord(ev[c], cs));
  }
  cudaStream_t* ws = h->hs_work;
  auto fork = [&](cudaEvent_t e) -> aao_status {  // both work streams follow s
    AAO_CK(cudaEventRecord(e, s));
    for (int i = 0; i < 2; ++i) AAO_CK(cudaStreamWaitEvent(ws[i], e, 0));
    return AAO_OK;
  };
  auto join = [&](cudaEvent_t e0, cudaEvent_t e1) -> aao_status {  // s follows both
    AAO_CK(cudaEventRecord(e0, ws[0]));
    AAO_CK(cudaEventRecord(e1, ws[1]));
    AAO_CK(cudaStreamWaitEvent(s, e0, 0));
    AAO_CK(cudaStreamWaitEvent(s, e1, 0));
    return AAO_OK;
  };
  AAO_TRY(fork(ev[2 * nch + 2]));
  for (int c = 0; c < nch; ++c) {
    const int r = c / per, k0 = (c % per) * CH;
    const size_t rb = (size_t)r * P.n * P.m;
    cudaStream_t w = ws[c & 1];
    AAO_CK(cudaStreamWaitEvent(w, ev[c], 0));
    AAO_KL(h, KC_RHS, w, launch_build_rhs_levels(P, h->hs_f + rb, d_psi0 + (size_t)r * P.m,
                                                 d_psi1 + (size_t)r * P.m, h->hs_b + rb, k0, CH, w,
                                                 &h->launches));
    const size_t bo = rb + (size_t)(P.n - k0 - CH) * P.m;  // the b levels this chunk filled
    AAO_TRY(dst_apply_levels(h, h->hs_b + bo, h->vbh + bo, CH, w));
  }
  AAO_TRY(join(ev[2 * nch + 3], ev[2 * nch + 4]));
  std::vector<aao_solve_info> loc(nrhs);
  aao_solve_info* inf = info ? info : loc.data();
  aao_status worst = h->precision == AAO_PREC_FP32_IR
                         ? solve_ir(h, nullptr, nullptr, 0, nrhs, rtol, maxit, inf, s, true)
                         : minres_spectral(h, h->vbh, h->vxh, 0, nrhs, rtol, maxit, inf, s, true);
  if (worst != AAO_OK && worst != AAO_ENOTCONV && worst != AAO_EBREAKDOWN) return worst;
  AAO_TRY(fork(ev[2 * nch + 5]));
  for (int c = 0; c < nch; ++c) {
    const size_t off = (size_t)(c / per) * P.n * P.m + (size_t)(c % per) * CH * P.m;
    cudaStream_t w = ws[c & 1];
    AAO_TRY(dst_apply_levels(h, h->vxh + off, h->hs_x + off, CH, w));
    AAO_CK(cudaEventRecord(ev[nch + c], w));
    AAO_CK(cudaStreamWaitEvent(cs, ev[nch + c], 0));
    AAO_CK(cudaMemcpyAsync(u + off, h->hs_x + off, CH * lb, cudaMemcpyDeviceToHost, cs));
  }
  AAO_TRY(join(ev[2 * nch + 6], ev[2 * nch + 7]));
  AAO_TRY(physical_check(h, h->hs_b, h->hs_x, nrhs, rtol, inf, &worst, s));
  AAO_CK(cudaEventRecord(ev[2 * nch + 1], cs));  // the caller's stream ends after the copies
  AAO_CK(cudaStreamWaitEvent(s, ev[2 * nch + 1], 0));
  AAO_CK(cudaStreamSynchronize(s));
  if (worst != AAO_OK) g_err = std::string("MINRES: ") + aao_status_str(worst);
  return worst;
}

}  // extern "C"
