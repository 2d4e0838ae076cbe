// Serving runtime: continuous admission of all-at-once wave solves of mixed sizes,
// wave speeds, alpha and tolerances onto one GPU.
//
// A worker thread owns a pool of solver handles keyed by shape (dim, N, nt) and a set
// of slots (one CUDA stream + completion event each).  Whenever a slot is free and the
// HBM budget admits the request's handle (reusing an idle handle of the same shape,
// else creating one, evicting idle handles least-recently-used first if needed), the
// request is bound to the handle (its tau, alpha, c2 tables are rebuilt in place, no
// allocation), its right-hand side is built on the device and the whole solve -- the
// DSTs, the graph-captured MINRES loop that keeps the Krylov state on the device, the
// residual check -- is enqueued on the slot's stream.  Requests on different slots run
// concurrently on the device; a request never shares buffers with another, so its
// result is bit-for-bit the same alone or in any mix.  Completion is detected by
// polling events (no blocking CUDA call in the loop); waits by callers are bounded.
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

struct PoolEntry {
  aao_handle* h = nullptr;
  double* b = nullptr;  // right-hand side built by the server for this handle's requests
  int dim = 0, N = 0, nt = 0, precision = 0;
  size_t bytes = 0;
  bool busy = false;
  uint64_t last_used = 0;
};

struct Pending {
  uint64_t ticket;
  aao_request req;
  double t_submit;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  bool active = false;
  PoolEntry* pe = nullptr;
  Pending p{};
  double t_start = 0;
};

thread_local std::string g_serr;

aao_status sfail(aao_status st, const std::string& m) {
  g_serr = m;
  return st;
}

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

}  // namespace

struct aao_server {
  size_t budget = 0;
  int device = 0;
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv;       // new work or stop (worker side)
  std::condition_variable done_cv;  // a result became ready (caller side)
  std::deque<Pending> pending;
  std::unordered_map<uint64_t, aao_serve_result> results;
  std::unordered_map<uint64_t, bool> ready;
  bool stop = false;
  uint64_t next_ticket = 1;
  // worker-owned
  std::vector<PoolEntry*> pool;
  std::vector<Slot> slots;
  size_t pool_bytes = 0;
  uint64_t tick = 0;
  std::thread worker;
  // statistics (under mu)
  aao_serve_stats st{};

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

  void evict(PoolEntry* pe) {
    pool_bytes -= pe->bytes;
    if (pe->b) cudaFree(pe->b);
    aao_destroy(pe->h);
    pool.erase(std::find(pool.begin(), pool.end(), pe));
    delete pe;
    std::lock_guard<std::mutex> lk(mu);
    st.evictions++;
    st.pool_bytes = pool_bytes;
  }

  // Bind request p to a handle; returns nullptr (and leaves p pending) when memory is
  // short right now; sets *err for requests that can never run.
  PoolEntry* acquire(const aao_request& q, aao_status* err) {
    *err = AAO_OK;
    for (PoolEntry* pe : pool)
      if (!pe->busy && pe->dim == q.dim && pe->N == q.N && pe->nt == q.nt && pe->precision == q.precision)
        return pe;
    const size_t need = aaoi_estimate_bytes(q.dim, q.N, q.nt, q.precision) + (size_t)q.nt * 8 *
                        (size_t)std::pow((double)q.N, (double)q.dim);
    if (need > budget) {
      *err = AAO_ENOMEM;
      return nullptr;
    }
    while (pool_bytes + need > budget) {  // evict idle handles, least recently used first
      PoolEntry* lru = nullptr;
      for (PoolEntry* pe : pool)
        if (!pe->busy && (!lru || pe->last_used < lru->last_used)) lru = pe;
      if (!lru) return nullptr;  // wait for running solves to finish
      evict(lru);
    }
    aao_grid g{q.dim, q.N, q.c2};
    aao_opts o{};
    o.precision = q.precision;
    o.nrhs_max = 1;
    o.graph = 1;
    aao_handle* h = nullptr;
    aao_status s = aao_create(&g, q.nt, q.tau, q.alpha, AAO_SCHEME_IMPLICIT_LEAPFROG, &o, &h);
    if (s != AAO_OK) {
      *err = s;
      return nullptr;
    }
    const size_t vb = (size_t)q.nt * 8 * (size_t)std::pow((double)q.N, (double)q.dim);
    double* b = nullptr;
    if (cudaMalloc(&b, vb) != cudaSuccess) {
      cudaGetLastError();
      aao_destroy(h);
      *err = AAO_ENOMEM;
      return nullptr;
    }
    PoolEntry* pe = new PoolEntry();
    pe->h = h;
    pe->b = b;
    pe->dim = q.dim;
    pe->N = q.N;
    pe->nt = q.nt;
    pe->precision = q.precision;
    pe->bytes = aao_workspace_bytes(h) + vb;
    pool.push_back(pe);
    pool_bytes += pe->bytes;
    std::lock_guard<std::mutex> lk(mu);
    st.handles_created++;
    st.pool_bytes = pool_bytes;
    st.peak_pool_bytes = std::max(st.peak_pool_bytes, (uint64_t)pool_bytes);
    return pe;
  }

  void run() {
    cudaSetDevice(device);
    while (true) {
      bool progressed = false;
      // 1. completions
      for (Slot& sl : slots) {
        if (!sl.active) continue;
        cudaError_t q = cudaEventQuery(sl.ev);
        if (q == cudaErrorNotReady) continue;
        aao_solve_info info{};
        aao_status s = (q == cudaSuccess) ? aaoi_solve_collect(sl.pe->h, sl.p.req.rtol, &info) : AAO_ECUDA;
        if (q != cudaSuccess) cudaGetLastError();
        sl.pe->busy = false;
        sl.pe->last_used = ++tick;
        sl.active = false;
        finish(sl.p, info, sl.t_start, s);
        progressed = true;
        std::lock_guard<std::mutex> lk(mu);
        st.in_flight--;
      }
      // 2. admissions
      for (Slot& sl : slots) {
        if (sl.active) continue;
        Pending p;
        {
          std::lock_guard<std::mutex> lk(mu);
          if (pending.empty()) break;
          p = pending.front();
        }
        aao_status err = AAO_OK;
        PoolEntry* pe = acquire(p.req, &err);
        if (!pe && err == AAO_OK) break;  // memory busy: retry after completions
        {
          std::lock_guard<std::mutex> lk(mu);
          pending.pop_front();
          st.pending = (int)pending.size();
        }
        progressed = true;
        if (!pe) {
          aao_solve_info info{};
          finish(p, info, now(), err);
          continue;
        }
        double* b = pe->b;
        aao_status s = aaoi_rebind(pe->h, p.req.tau, p.req.alpha, p.req.c2);
        if (s == AAO_OK) s = aao_build_rhs(pe->h, p.req.f, p.req.psi0, p.req.psi1, b, 1, sl.stream);
        if (s == AAO_OK) s = aaoi_solve_enqueue(pe->h, b, p.req.x, p.req.rtol, p.req.maxit, sl.stream);
        if (s == AAO_OK && cudaEventRecord(sl.ev, sl.stream) != cudaSuccess) s = AAO_ECUDA;
        if (s != AAO_OK) {
          aao_solve_info info{};
          finish(p, info, now(), s);
          continue;
        }
        pe->busy = true;
        sl.pe = pe;
        sl.p = p;
        sl.t_start = now();
        sl.active = true;
        std::lock_guard<std::mutex> lk(mu);
        st.admitted++;
        st.in_flight++;
      }
      // 3. idle / stop
      bool any_active = false;
      for (Slot& sl : slots) any_active |= sl.active;
      std::unique_lock<std::mutex> lk(mu);
      if (stop && pending.empty() && !any_active) break;
      if (!progressed) {
        if (any_active) {
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
  s->t0 = Clock::now();
  cudaGetDevice(&s->device);
  s->slots.resize(max_slots);
  for (Slot& sl : s->slots) {
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      for (Slot& t : s->slots) {
        if (t.stream) cudaStreamDestroy(t.stream);
        if (t.ev) cudaEventDestroy(t.ev);
      }
      delete s;
      return sfail(AAO_ECUDA, "stream/event creation failed");
    }
  }
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
  for (PoolEntry* pe : s->pool) {
    if (pe->b) cudaFree(pe->b);
    aao_destroy(pe->h);
    delete pe;
  }
  for (Slot& sl : s->slots) {
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.ev) cudaEventDestroy(sl.ev);
  }
  delete s;
  return AAO_OK;
}

}  // extern "C"
