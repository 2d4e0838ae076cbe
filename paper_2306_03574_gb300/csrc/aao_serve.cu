// Serving runtime: continuous batching of all-at-once wave solves of mixed sizes, wave
// speeds, alpha and tolerances onto one GPU (a runtime around the method; the paper
// solves one problem at a time).
//
// Admission.  A worker thread admits queued requests first-fit: a request starts as soon
// as a slot is free and an idle handle of its shape (dim, N, nt, precision) is in the
// pool; requests behind one that must wait are not held up by it.  Handles come from a
// pool bounded by an HBM budget.  A provisioner thread creates missing handles and
// destroys evicted ones (least recently used idle handles first), so cudaMalloc, cudaFree
// and the synchronous table build of aao_create never run on the worker's path; when a
// request takes the last idle handle of its shape, a spare is provisioned in the
// background while the pool stays within half the budget.  A
// pooled handle is re-bound to the request's tau, alpha and c2 on the device without a
// host synchronisation (its |Sigma| check is read when the request completes).
//
// Batching.  Admitted requests are grouped by size class (unknowns per request below
// 2^18, 2^21, 2^23, and above), one CUDA stream per class, so that small problems are
// not paced by large ones.  A class advances in ROUNDS: one round is one MINRES
// iteration of every request of the class, performed by grouped launches -- one
// operator (with the delta dot), one v update, one time-pipeline launch per (precision,
// n) bucket, one dot, one w/x update with the true residual and three scalar steps --
// so the launch count of a round does not grow with the number of requests in it.  A
// request joins the next round after its initialisation (right-hand side, DSTs, first
// preconditioner application, all on its class's stream) and leaves when the done flag
// of a completed round says it converged or reached maxit; its inverse DSTs and
// residual check follow on the same stream.  Every launch runs, for each request, the
// device code and block decomposition of the request's solo solve, so a result is bit
// for bit the same alone and in any mix.
//
// Host side.  The worker keeps up to ROUNDS_IN_FLIGHT rounds queued per class (requests
// that finished on the device are skipped by the launches until the host has seen their
// flag), reads flags and results from pinned memory once the recorded events complete,
// and never makes a blocking CUDA call.  Waits by callers are bounded.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "aao_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;
using aao::GROUP_MAX;

constexpr int NCLASS = 4;             // size classes
constexpr int ROUNDS_IN_FLIGHT = 3;   // rounds queued per class
constexpr int NBUCKET = 5;            // time lengths 64 .. 1024
constexpr int QUEUE_SCAN = 256;       // first-fit scan depth of the queue
constexpr int LARGE_ACTIVE = 2;       // requests active at once in the largest class

int size_class(long long unknowns) {
  if (unknowns < (1LL << 18)) return 0;
  if (unknowns < (1LL << 21)) return 1;
  if (unknowns < (1LL << 23)) return 2;
  return 3;
}

int bucket_of(int nt) {
  int b = 0;
  while ((64 << b) < nt) ++b;
  return b;
}

struct PoolEntry {
  aao_handle* h = nullptr;
  double* b = nullptr;  // right-hand side built by the server for this handle's requests
  int dim = 0, N = 0, nt = 0, precision = 0;
  size_t bytes = 0;     // reserved while provisioning, actual afterwards
  bool ready = false;   // created and prepared by the provisioner
  bool busy = false;    // bound to a request
  aao_status fail = AAO_OK;  // provisioning failed with this status
  uint64_t last_used = 0;
};

struct Pending {
  uint64_t ticket;
  aao_request req;
  double t_submit;
};

struct Active {  // an admitted request
  Pending p{};
  PoolEntry* pe = nullptr;
  int cls = 0;
  int iter = 0;          // iterations enqueued so far
  bool retired = false;  // left the rounds (finishing or finished)
  double t_start = 0;
  cudaEvent_t fin = nullptr;
};

// Descriptors of one round (pinned host copy and device copy).
struct RoundBuf {
  aao::GroupRound g;
  aao::TimeGroup<double> t64[NBUCKET];
  aao::TimeGroup<aao::dfl> tff[NBUCKET];
  int flags[GROUP_MAX];
};

struct Round {
  RoundBuf* host = nullptr;
  RoundBuf* dev = nullptr;
  cudaEvent_t ev = nullptr;
  std::vector<Active*> members;
};

struct SizeClass {
  cudaStream_t stream = nullptr;
  std::vector<Active*> active;  // requests that iterate in the next round
  std::deque<Round*> inflight;
  std::vector<Round*> free_rounds;
};

thread_local std::string g_serr;

aao_status sfail(aao_status st, const std::string& m) {
  g_serr = m;
  return st;
}

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

long long unknowns_of(const aao_request& q) {
  long long m = 1;
  for (int i = 0; i < q.dim; ++i) m *= q.N;
  return m * q.nt;
}

}  // namespace

struct aao_server {
  size_t budget = 0;
  int device = 0;
  int max_slots = 1;
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv;       // new work or stop (worker side)
  std::condition_variable done_cv;  // a result became ready (caller side)
  std::deque<Pending> pending;
  std::unordered_map<uint64_t, aao_serve_result> results;
  std::unordered_map<uint64_t, bool> ready;
  bool stop = false;
  uint64_t next_ticket = 1;
  aao_serve_stats st{};  // under mu

  // pool: shared by the worker and the provisioner (under pool_mu)
  std::mutex pool_mu;
  std::condition_variable prov_cv;
  std::vector<PoolEntry*> pool;
  std::deque<PoolEntry*> to_create, to_destroy;
  size_t pool_bytes = 0;
  bool prov_stop = false;
  std::thread provisioner;

  // worker-owned
  SizeClass cls[NCLASS];
  std::vector<Active*> finishing;
  std::vector<cudaEvent_t> ev_pool;
  int in_flight = 0;
  uint64_t tick = 0;
  std::thread worker;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

  void finish(const Pending& p, const aao_solve_info& info, double t_start, aao_status status) {
    aao_serve_result r{};
    r.info = info;
    r.info.status = status;
    r.ticket = p.ticket;
    r.t_submit = p.t_submit;
    r.t_start = t_start;
    r.t_done = now();
    std::lock_guard<std::mutex> lk(mu);
    results[p.ticket] = r;
    ready[p.ticket] = true;
    if (status == AAO_OK) st.completed++;
    else st.failed++;
    done_cv.notify_all();
  }

  cudaEvent_t take_event() {
    if (!ev_pool.empty()) {
      cudaEvent_t e = ev_pool.back();
      ev_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return e;
  }

  void publish_pool_stats() {  // pool_mu held
    std::lock_guard<std::mutex> lk(mu);
    st.pool_bytes = pool_bytes;
    st.peak_pool_bytes = std::max(st.peak_pool_bytes, (uint64_t)pool_bytes);
  }

  // ---- provisioner thread: creates and destroys handles off the worker's path ----
  void provision() {
    cudaSetDevice(device);
    while (true) {
      PoolEntry* job = nullptr;
      bool destroy = false;
      {
        std::unique_lock<std::mutex> lk(pool_mu);
        prov_cv.wait(lk, [&] { return prov_stop || !to_create.empty() || !to_destroy.empty(); });
        if (!to_destroy.empty()) {
          job = to_destroy.front();
          to_destroy.pop_front();
          destroy = true;
        } else if (!to_create.empty()) {
          job = to_create.front();
          to_create.pop_front();
        } else {
          break;  // stop requested, nothing left
        }
      }
      if (destroy) {
        if (job->b) cudaFree(job->b);
        aao_destroy(job->h);
        delete job;
        continue;
      }
      // a handle with neutral parameters; every request re-binds its own tau, alpha, c2
      aao_grid g{job->dim, job->N, 1.0};
      aao_opts o{};
      o.precision = job->precision;
      o.nrhs_max = 1;
      aao_handle* h = nullptr;
      aao_status s = aao_create(&g, job->nt, 1.0 / job->nt, 0.5, AAO_SCHEME_IMPLICIT_LEAPFROG, &o, &h);
      if (s == AAO_OK) s = aaoi_serving_prepare(h);
      double* b = nullptr;
      size_t m = 1;
      for (int i = 0; i < job->dim; ++i) m *= (size_t)job->N;
      const size_t vb = (size_t)job->nt * m * sizeof(double);
      if (s == AAO_OK && cudaMalloc(&b, vb) != cudaSuccess) {
        cudaGetLastError();
        s = AAO_ENOMEM;
      }
      std::lock_guard<std::mutex> lk(pool_mu);
      if (s != AAO_OK) {
        if (b) cudaFree(b);
        if (h) aao_destroy(h);
        pool_bytes -= job->bytes;
        job->bytes = 0;
        job->fail = s;  // the worker reports it to a waiting request and drops the entry
      } else {
        pool_bytes -= job->bytes;
        job->h = h;
        job->b = b;
        job->bytes = aao_workspace_bytes(h) + vb;
        pool_bytes += job->bytes;
        job->ready = true;
      }
      publish_pool_stats();
      cv.notify_all();
    }
  }

  // ---- worker: admission ----
  // Try to start request p; returns false if it must wait (it stays queued).
  bool try_admit(const Pending& p) {
    const aao_request& q = p.req;
    const int c = size_class(unknowns_of(q));
    if ((int)cls[c].active.size() >= GROUP_MAX) return false;
    // the largest class runs at most LARGE_ACTIVE requests at a time: each round of a
    // class runs one iteration of all its requests, and a GPU-filling request gains
    // nothing from sharing its rounds, while the requests behind it in the queue wait
    // the shorter for it (first come, first served within the class)
    if (c == NCLASS - 1 && (int)cls[c].active.size() >= LARGE_ACTIVE) return false;
    PoolEntry* pe = nullptr;
    {
      std::lock_guard<std::mutex> lk(pool_mu);
      bool provisioning = false;
      for (PoolEntry* e : pool) {
        if (e->dim != q.dim || e->N != q.N || e->nt != q.nt || e->precision != q.precision || e->busy) continue;
        if (e->fail != AAO_OK) {  // creation failed: report it to this request
          const aao_status fs = e->fail;
          pool.erase(std::find(pool.begin(), pool.end(), e));
          delete e;
          aao_solve_info info{};
          finish(p, info, now(), fs);
          return true;
        }
        if (e->ready) { pe = e; break; }
        provisioning = true;
      }
      if (!pe) {
        if (provisioning) return false;
        const size_t need = aaoi_estimate_bytes(q.dim, q.N, q.nt, q.precision) +
                            (size_t)unknowns_of(q) * sizeof(double);
        if (need > budget) {
          aao_solve_info info{};
          finish(p, info, now(), AAO_ENOMEM);
          return true;
        }
        while (pool_bytes + need > budget) {  // evict idle handles, least recently used first
          PoolEntry* lru = nullptr;
          for (PoolEntry* e : pool)
            if (e->ready && !e->busy && (!lru || e->last_used < lru->last_used)) lru = e;
          if (!lru) return false;  // wait for running solves to finish
          pool.erase(std::find(pool.begin(), pool.end(), lru));
          pool_bytes -= lru->bytes;
          to_destroy.push_back(lru);
          std::lock_guard<std::mutex> lk2(mu);
          st.evictions++;
        }
        post_create(q, need);
        return false;  // admitted once the handle is ready
      }
      pe->busy = true;
      // Spare: when this takes the last idle handle of its shape, provision another in
      // the background if the pool stays within half the budget (spares never evict) and
      // more than one request can be in flight, so that the next request of the shape
      // does not wait for a handle to be created.
      bool other = false;
      for (PoolEntry* e : pool)
        if (e != pe && e->dim == q.dim && e->N == q.N && e->nt == q.nt && e->precision == q.precision &&
            !e->busy && e->fail == AAO_OK)
          other = true;
      const size_t need = aaoi_estimate_bytes(q.dim, q.N, q.nt, q.precision) + (size_t)unknowns_of(q) * sizeof(double);
      if (!other && max_slots > 1 && pool_bytes + need <= budget / 2) post_create(q, need);
    }
    SizeClass& C = cls[c];
    aao_status s = aaoi_rebind_async(pe->h, q.tau, q.alpha, q.c2, C.stream);
    if (s == AAO_OK) s = aaoi_group_begin(pe->h, q.f, q.psi0, q.psi1, pe->b, q.rtol, q.maxit, C.stream);
    if (s != AAO_OK) {
      release(pe);
      aao_solve_info info{};
      finish(p, info, now(), s);
      return true;
    }
    Active* a = new Active();
    a->p = p;
    a->pe = pe;
    a->cls = c;
    a->t_start = now();
    C.active.push_back(a);
    ++in_flight;
    std::lock_guard<std::mutex> lk(mu);
    st.admitted++;
    st.in_flight = in_flight;
    return true;
  }

  // queue the creation of a handle of q's shape (pool_mu held); its bytes are reserved now
  void post_create(const aao_request& q, size_t need) {
    PoolEntry* e = new PoolEntry();
    e->dim = q.dim;
    e->N = q.N;
    e->nt = q.nt;
    e->precision = q.precision;
    e->bytes = need;
    pool.push_back(e);
    pool_bytes += need;
    to_create.push_back(e);
    {
      std::lock_guard<std::mutex> lk2(mu);
      st.handles_created++;
    }
    publish_pool_stats();
    prov_cv.notify_all();
  }

  void release(PoolEntry* pe) {
    std::lock_guard<std::mutex> lk(pool_mu);
    pe->busy = false;
    pe->last_used = ++tick;
  }

  bool admit() {
    bool progressed = false;
    std::vector<Pending> scan;
    {
      std::lock_guard<std::mutex> lk(mu);
      const size_t k = std::min(pending.size(), (size_t)QUEUE_SCAN);
      scan.assign(pending.begin(), pending.begin() + k);
    }
    std::vector<uint64_t> taken;
    for (const Pending& p : scan) {
      if (in_flight >= max_slots) break;
      if (try_admit(p)) {
        taken.push_back(p.ticket);
        progressed = true;
      }
    }
    if (!taken.empty()) {
      std::lock_guard<std::mutex> lk(mu);
      for (uint64_t t : taken)
        for (auto it = pending.begin(); it != pending.end(); ++it)
          if (it->ticket == t) {
            pending.erase(it);
            break;
          }
      st.pending = (int)pending.size();
    }
    return progressed;
  }

  // ---- worker: rounds ----
  Round* take_round(SizeClass& C) {
    if (C.free_rounds.empty()) return nullptr;
    Round* r = C.free_rounds.back();
    C.free_rounds.pop_back();
    return r;
  }

  // a round buffer (created by aao_serve_create, ROUNDS_IN_FLIGHT per class)
  Round* new_round() {
    Round* r = new Round();
    if (cudaMallocHost(&r->host, sizeof(RoundBuf)) != cudaSuccess ||
        cudaMalloc(&r->dev, sizeof(RoundBuf)) != cudaSuccess ||
        cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      if (r->host) cudaFreeHost(r->host);
      if (r->dev) cudaFree(r->dev);
      if (r->ev) cudaEventDestroy(r->ev);
      delete r;
      return nullptr;
    }
    return r;
  }

  // One MINRES iteration of every active request of class C, by grouped launches.
  bool enqueue_round(SizeClass& C) {
    if (C.active.empty() || (int)C.inflight.size() >= ROUNDS_IN_FLIGHT) return false;
    Round* R = take_round(C);
    if (!R) return false;
    RoundBuf& H = *R->host;
    aao::GroupRound& g = H.g;
    const int cnt = (int)C.active.size();
    g.count = cnt;
    g.flags = R->dev->flags;
    g.yt[0] = g.dot[0] = g.vu[0] = g.wx[0] = 0;
    int nt64[NBUCKET] = {0}, ntff[NBUCKET] = {0};
    for (int b = 0; b < NBUCKET; ++b) H.t64[b].tile[0] = H.tff[b].tile[0] = 0;
    std::vector<std::pair<aao_handle*, int>> solo_time;
    R->members = C.active;
    for (int i = 0; i < cnt; ++i) {
      Active* a = C.active[i];
      aao_handle* h = a->pe->h;
      const int par = a->iter & 1;
      aaoi_group_problem(h, par, &g.p[i]);
      const aao::GroupProblem& P = g.p[i];
      g.yt[i + 1] = g.yt[i] + aao::group_yt_blocks(P.n, P.m);
      g.dot[i + 1] = g.dot[i] + P.nb_dot;
      g.vu[i + 1] = g.vu[i] + P.nb_vu;
      g.wx[i + 1] = g.wx[i] + aao::group_wx_blocks(P.m);
      const int L = aaoi_nt(h), bk = bucket_of(L), v = aaoi_time_variant(h);
      if (aaoi_precision(h) == AAO_PREC_F32X2 && v == aao::group_time_variant<aao::dfl>()) {
        aao::TimeGroup<aao::dfl>& T = H.tff[bk];
        aaoi_time_entry_ff(h, par, &T.e[ntff[bk]]);
        T.tile[ntff[bk] + 1] = T.tile[ntff[bk]] + aao::group_time_tiles<aao::dfl>(L, P.m);
        ++ntff[bk];
      } else if (aaoi_precision(h) == AAO_PREC_FP64 && v == aao::group_time_variant<double>()) {
        aao::TimeGroup<double>& T = H.t64[bk];
        aaoi_time_entry64(h, par, &T.e[nt64[bk]]);
        T.tile[nt64[bk] + 1] = T.tile[nt64[bk]] + aao::group_time_tiles<double>(L, P.m);
        ++nt64[bk];
      } else {
        solo_time.emplace_back(h, par);
      }
      a->iter++;
    }
    for (int b = 0; b < NBUCKET; ++b) {
      H.t64[b].count = nt64[b];
      H.tff[b].count = ntff[b];
    }
    const cudaStream_t s = C.stream;
    bool ok = cudaMemcpyAsync(R->dev, R->host, offsetof(RoundBuf, flags), cudaMemcpyHostToDevice, s) == cudaSuccess;
    ok = ok && aao::launch_group_ythat(&R->dev->g, g.yt[cnt], s) == cudaSuccess;
    ok = ok && aao::launch_group_scalars(1, &R->dev->g, cnt, s) == cudaSuccess;
    ok = ok && aao::launch_group_vupdate(&R->dev->g, g.vu[cnt], s) == cudaSuccess;
    int launches = 3;
    for (int b = 0; b < NBUCKET && ok; ++b) {
      if (nt64[b]) {
        ok = aao::launch_group_time<double>(64 << b, aao::group_time_variant<double>(), &R->dev->t64[b],
                                            H.t64[b].tile[nt64[b]], s) == cudaSuccess;
        ++launches;
      }
      if (ok && ntff[b]) {
        ok = aao::launch_group_time<aao::dfl>(64 << b, aao::group_time_variant<aao::dfl>(), &R->dev->tff[b],
                                              H.tff[b].tile[ntff[b]], s) == cudaSuccess;
        ++launches;
      }
    }
    for (auto& hp : solo_time) {
      ok = ok && aaoi_group_time_solo(hp.first, hp.second, s) == AAO_OK;
      ++launches;
    }
    ok = ok && aao::launch_group_dot(&R->dev->g, g.dot[cnt], s) == cudaSuccess;
    ok = ok && aao::launch_group_scalars(2, &R->dev->g, cnt, s) == cudaSuccess;
    ok = ok && aao::launch_group_wx_res(&R->dev->g, g.wx[cnt], s) == cudaSuccess;
    ok = ok && aao::launch_group_scalars(3, &R->dev->g, cnt, s) == cudaSuccess;
    launches += 4;
    ok = ok && cudaMemcpyAsync(H.flags, R->dev->flags, cnt * sizeof(int), cudaMemcpyDeviceToHost, s) == cudaSuccess;
    ok = ok && cudaEventRecord(R->ev, s) == cudaSuccess;
    if (!ok) {
      // a launch failed (a CUDA error): every member fails
      cudaGetLastError();
      for (Active* a : R->members) a->iter = 1 << 30;
    }
    C.inflight.push_back(R);
    std::lock_guard<std::mutex> lk(mu);
    st.rounds++;
    st.round_problems += (uint64_t)cnt;
    st.grouped_launches += (uint64_t)launches;
    return true;
  }

  // Leave the rounds: inverse DSTs and the residual check on the class stream.
  void retire(Active* a) {
    a->retired = true;
    SizeClass& C = cls[a->cls];
    C.active.erase(std::find(C.active.begin(), C.active.end(), a));
    a->fin = take_event();
    aao_status s = aaoi_group_end(a->pe->h, a->pe->b, a->p.req.x, C.stream);
    if (s == AAO_OK && (!a->fin || cudaEventRecord(a->fin, C.stream) != cudaSuccess)) s = AAO_ECUDA;
    if (s != AAO_OK) {
      cudaGetLastError();
      if (a->fin) ev_pool.push_back(a->fin);
      a->fin = nullptr;
      aao_solve_info info{};
      complete(a, info, s);
      return;
    }
    finishing.push_back(a);
  }

  void complete(Active* a, const aao_solve_info& info, aao_status s) {
    release(a->pe);
    finish(a->p, info, a->t_start, s);
    --in_flight;
    {
      std::lock_guard<std::mutex> lk(mu);
      st.in_flight = in_flight;
    }
    delete a;
  }

  bool poll_rounds(SizeClass& C) {
    bool progressed = false;
    while (!C.inflight.empty()) {
      Round* R = C.inflight.front();
      const cudaError_t q = cudaEventQuery(R->ev);
      if (q == cudaErrorNotReady) break;
      if (q != cudaSuccess) cudaGetLastError();
      C.inflight.pop_front();
      for (size_t i = 0; i < R->members.size(); ++i) {
        Active* a = R->members[i];
        if (a->retired) continue;
        const bool done = q != cudaSuccess || R->host->flags[i] != 0 || a->iter > a->p.req.maxit + 8;
        if (done) retire(a);
      }
      R->members.clear();
      C.free_rounds.push_back(R);
      progressed = true;
    }
    return progressed;
  }

  bool poll_finishing() {
    bool progressed = false;
    for (size_t i = 0; i < finishing.size();) {
      Active* a = finishing[i];
      const cudaError_t q = cudaEventQuery(a->fin);
      if (q == cudaErrorNotReady) {
        ++i;
        continue;
      }
      aao_solve_info info{};
      aao_status s = AAO_ECUDA;
      if (q == cudaSuccess) s = aaoi_group_collect(a->pe->h, a->p.req.rtol, &info);
      else cudaGetLastError();
      ev_pool.push_back(a->fin);
      finishing[i] = finishing.back();
      finishing.pop_back();
      complete(a, info, s);
      progressed = true;
    }
    return progressed;
  }

  void free_classes() {
    for (SizeClass& C : cls) {
      if (C.stream) cudaStreamSynchronize(C.stream);
      for (Round* R : C.inflight) C.free_rounds.push_back(R);
      C.inflight.clear();
      for (Round* R : C.free_rounds) {
        cudaFreeHost(R->host);
        cudaFree(R->dev);
        cudaEventDestroy(R->ev);
        delete R;
      }
      C.free_rounds.clear();
      if (C.stream) cudaStreamDestroy(C.stream);
      C.stream = nullptr;
    }
  }

  void run() {
    cudaSetDevice(device);
    while (true) {
      bool progressed = poll_finishing();
      for (SizeClass& C : cls) progressed |= poll_rounds(C);
      progressed |= admit();
      for (SizeClass& C : cls)
        while (enqueue_round(C)) progressed = true;
      bool busy = in_flight > 0;
      std::unique_lock<std::mutex> lk(mu);
      if (stop && pending.empty() && !busy) break;
      if (!progressed) {
        if (busy) {
          lk.unlock();
          std::this_thread::sleep_for(std::chrono::microseconds(20));
        } else {
          cv.wait_for(lk, std::chrono::milliseconds(2));
        }
      }
    }
  }
};

extern "C" {

const char* aao_serve_last_error(void) { return g_serr.c_str(); }

aao_status aao_serve_create(size_t hbm_budget_bytes, int max_slots, aao_server** out) {
  g_serr.clear();
  if (!out) return sfail(AAO_EINVAL, "null out pointer");
  *out = nullptr;
  if (max_slots < 1 || max_slots > 64) return sfail(AAO_EINVAL, "max_slots must be in [1, 64]");
  if (hbm_budget_bytes == 0) return sfail(AAO_EINVAL, "zero budget");
  aao_server* s = new aao_server();
  s->budget = hbm_budget_bytes;
  s->st.budget = hbm_budget_bytes;
  s->max_slots = max_slots;
  s->t0 = Clock::now();
  cudaGetDevice(&s->device);
  // streams and round buffers (pinned and device descriptors) of every size class.  The
  // smaller the class, the higher its stream's priority: the CTAs of a small problem's
  // kernels are dispatched ahead of the pending CTAs of a large problem's (a 1D request
  // that solves in a third of a millisecond alone otherwise waits behind whole waves of
  // a 2D time kernel); running CTAs are never preempted, and no result changes.
  int prio_least = 0, prio_greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest) != cudaSuccess) {
    cudaGetLastError();
    prio_least = prio_greatest = 0;
  }
  bool ok = true;
  for (int c = 0; c < NCLASS; ++c) {
    SizeClass& C = s->cls[c];
    const int prio = prio_greatest + ((prio_least - prio_greatest) * c) / (NCLASS - 1);
    ok = ok && cudaStreamCreateWithPriority(&C.stream, cudaStreamNonBlocking, prio) == cudaSuccess;
    for (int i = 0; ok && i < ROUNDS_IN_FLIGHT; ++i) {
      Round* r = s->new_round();
      if (r) C.free_rounds.push_back(r);
      else ok = false;
    }
  }
  if (!ok) {
    cudaGetLastError();
    s->free_classes();
    delete s;
    return sfail(AAO_ECUDA, "stream or round-buffer creation failed");
  }
  s->provisioner = std::thread([s]() { s->provision(); });
  s->worker = std::thread([s]() { s->run(); });
  *out = s;
  return AAO_OK;
}

aao_status aao_serve_submit(aao_server* s, const aao_request* r, uint64_t* ticket) {
  if (!s || !r || !ticket) return sfail(AAO_EINVAL, "null pointer");
  if (!r->f || !r->psi0 || !r->psi1 || !r->x) return sfail(AAO_EINVAL, "null data pointer");
  if (r->dim < 1 || r->dim > 3 || !pow2(r->N + 1) || r->N + 1 < 64 || r->N + 1 > 512 || !pow2(r->nt) ||
      r->nt < 64 || r->nt > 1024)
    return sfail(AAO_EUNSUPPORTED, "size outside the supported set");
  if (!(r->tau > 0) || !(r->alpha > 0 && r->alpha <= 1) || !(r->c2 > 0) || !(r->rtol >= 0) || r->maxit < 1)
    return sfail(AAO_EINVAL, "bad parameters");
  if (r->precision != AAO_PREC_FP64 && r->precision != AAO_PREC_F32X2)
    return sfail(AAO_EINVAL, "served precision must be AAO_PREC_FP64 or AAO_PREC_F32X2");
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return sfail(AAO_EBUSY, "server is shutting down");
  const uint64_t t = s->next_ticket++;
  s->pending.push_back(Pending{t, *r, s->now()});
  s->ready[t] = false;
  s->st.submitted++;
  s->st.pending = (int)s->pending.size();
  *ticket = t;
  s->cv.notify_all();
  return AAO_OK;
}

aao_status aao_serve_poll(aao_server* s, uint64_t ticket, aao_serve_result* out) {
  if (!s) return sfail(AAO_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->ready.find(ticket);
  if (it == s->ready.end()) return sfail(AAO_EINVAL, "unknown ticket");
  if (!it->second) return AAO_EPENDING;
  const aao_serve_result r = s->results[ticket];
  if (out) *out = r;
  s->results.erase(ticket);
  s->ready.erase(it);
  return (aao_status)r.info.status;
}

aao_status aao_serve_wait(aao_server* s, uint64_t ticket, double timeout_s, aao_serve_result* out) {
  if (!s) return sfail(AAO_EINVAL, "null server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto pred = [&]() {
    auto it = s->ready.find(ticket);
    return it == s->ready.end() || it->second;
  };
  if (!s->done_cv.wait_for(lk, std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0), pred))
    return AAO_ETIMEOUT;
  lk.unlock();
  return aao_serve_poll(s, ticket, out);
}

aao_status aao_serve_stats_get(aao_server* s, aao_serve_stats* out) {
  if (!s || !out) return sfail(AAO_EINVAL, "null pointer");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  out->pending = (int)s->pending.size();
  return AAO_OK;
}

aao_status aao_serve_destroy(aao_server* s) {
  if (!s) return AAO_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  {
    std::lock_guard<std::mutex> lk(s->pool_mu);
    s->prov_stop = true;
    s->prov_cv.notify_all();
  }
  if (s->provisioner.joinable()) s->provisioner.join();
  s->free_classes();
  for (PoolEntry* pe : s->pool) {
    if (pe->b) cudaFree(pe->b);
    if (pe->h) aao_destroy(pe->h);
    delete pe;
  }
  for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
  delete s;
  return AAO_OK;
}

}  // extern "C"
