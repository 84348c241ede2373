// Continuous-batching solve server over resident hierarchies.
//
// Requests (a hierarchy, k right-hand sides in host memory, a tolerance) are
// queued by lg_serve_submit and admitted in arrival order by `slots` worker
// threads, each owning a CUDA stream and a cached solve workspace, as soon as
// a slot is free and the HBM budget (registered hierarchies + workspaces of
// running requests) has room. Admitted requests run concurrently on their
// own streams and finish independently, so a request that arrives while
// others are on the device starts as soon as one of them completes. Every
// request runs the same kernels with the same launch plans as lg_solve_batch,
// so its result does not depend on what else is running.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "lg_hier.h"

namespace lg {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  Hier* h = nullptr;
  int k = 1;
  const double* B = nullptr;
  double* X = nullptr;
  double tol = 1e-8;
  double ws_bytes = 0.0;
  Clock::time_point submitted;
  bool done = false;
  lg_info info{};
};

struct Slot {
  cudaStream_t stream = nullptr;
  DBuf<double> Bd, Xd;  // staging of the running request (grown as needed)
  size_t staged = 0;
};

// An idle solve workspace kept for reuse, so that a request does not pay for
// allocations, a CUDA graph capture and SpMM plans each time its slot served
// another graph before. Widths are powers of two.
struct Pooled {
  Hier* h = nullptr;
  int k = 0;
  double bytes = 0.0;
  uint64_t last_use = 0;
  std::unique_ptr<Workspace> ws;
};

struct Server {
  lg_serve_options o{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, Request*> requests;
  std::unordered_map<Hier*, double> resident;
  double resident_bytes = 0.0, inflight_bytes = 0.0;
  uint64_t next_ticket = 1;
  int running = 0;
  bool stopping = false;
  std::vector<Slot> slots;
  std::vector<Pooled> pool;  // idle workspaces
  double pooled_bytes = 0.0;
  uint64_t use_clock = 0;
  std::vector<std::thread> threads;
  std::vector<double> latencies_ms;
  int64_t completed = 0, failed = 0, rhs_done = 0;
  Clock::time_point created = Clock::now();
  int device = 0;
};

static int pow2_width(int k) {
  int p = 1;
  while (p < k) p <<= 1;
  return p;
}

// Device bytes of a solve workspace for k columns: per-level cycle vectors in
// both precisions, the FP64 Krylov vectors and reduction scratch.
static double workspace_bytes(const Hier& h, int k) {
  double b = 0.0;
  for (const auto& L : h.levels) {
    const double nv = (double)L->n * k;
    const int vecs = L->kind == LG_LEVEL_AGG ? 5 : 2;
    b += nv * vecs * (8.0 + 4.0);
    b += (double)(L->plan.plan.nchunks + L->mem_plan.plan.nchunks + L->pt_plan.plan.nchunks) * 8.0 * k;
  }
  b += (double)h.levels[0]->n * k * 8.0 * 11.0;  // Krylov vectors, transposes, the slot's B and X
  return b + (1 << 20);
}

// Under the server lock: the smallest idle workspace of h at least k wide
// (removed from the pool), or null.
static std::unique_ptr<Workspace> pool_take(Server* sv, Hier* h, int k) {
  int best = -1;
  for (int i = 0; i < (int)sv->pool.size(); ++i) {
    const Pooled& p = sv->pool[i];
    if (p.h == h && p.k >= k && (best < 0 || p.k < sv->pool[best].k)) best = i;
  }
  if (best < 0) return nullptr;
  std::unique_ptr<Workspace> ws = std::move(sv->pool[best].ws);
  sv->pooled_bytes -= sv->pool[best].bytes;
  sv->pool.erase(sv->pool.begin() + best);
  return ws;
}

// Under the server lock: move least recently used idle workspaces to `out`
// (freed by the caller outside the lock) until `need` more bytes fit.
static void pool_evict(Server* sv, double need, std::vector<std::unique_ptr<Workspace>>& out) {
  while (!sv->pool.empty() &&
         sv->resident_bytes + sv->inflight_bytes + sv->pooled_bytes + need > sv->o.hbm_budget_bytes) {
    int lru = 0;
    for (int i = 1; i < (int)sv->pool.size(); ++i)
      if (sv->pool[i].last_use < sv->pool[lru].last_use) lru = i;
    sv->pooled_bytes -= sv->pool[lru].bytes;
    out.push_back(std::move(sv->pool[lru].ws));
    sv->pool.erase(sv->pool.begin() + lru);
  }
}

static void serve_worker(Server* sv, int slot_id) {
  Slot& slot = sv->slots[slot_id];
  cudaSetDevice(sv->device);
  for (;;) {
    Request* rq = nullptr;
    std::unique_ptr<Workspace> ws;
    std::vector<std::unique_ptr<Workspace>> evicted;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      // admit the oldest request once it fits the budget (arrival order);
      // idle pooled workspaces give way to it
      sv->cv_work.wait(lk, [&] {
        if (sv->queue.empty()) return sv->stopping;
        Request* head = sv->queue.front();
        return sv->resident_bytes + sv->inflight_bytes + head->ws_bytes <= sv->o.hbm_budget_bytes ||
               sv->running == 0;
      });
      if (sv->queue.empty() && sv->stopping) return;
      rq = sv->queue.front();
      sv->queue.pop_front();
      ws = pool_take(sv, rq->h, rq->k);
      if (!ws) pool_evict(sv, rq->ws_bytes, evicted);
      sv->inflight_bytes += rq->ws_bytes;
      sv->running += 1;
    }
    evicted.clear();  // frees the evicted workspaces' device memory
    int st = LG_OK;
    lg_info worst{};
    try {
      const int64_t n = rq->h->levels[0]->n;
      if (!ws) ws = make_workspace(*rq->h, pow2_width(rq->k), slot.stream);
      const size_t need = (size_t)n * rq->k;
      if (slot.staged < need) {
        slot.Bd.alloc(need, slot.stream);
        slot.Xd.alloc(need, slot.stream);
        slot.staged = need;
      }
      LG_CUDA(cudaMemcpyAsync(slot.Bd.get(), rq->B, sizeof(double) * n * rq->k, cudaMemcpyHostToDevice, slot.stream));
      std::vector<lg_info> infos(rq->k);
      st = pcg_solve_batch(*rq->h, *ws, rq->k, slot.Bd.get(), slot.Xd.get(), rq->tol, sv->o.precision,
                           slot.stream, infos.data());
      LG_CUDA(cudaMemcpyAsync(rq->X, slot.Xd.get(), sizeof(double) * n * rq->k, cudaMemcpyDeviceToHost, slot.stream));
      LG_CUDA(cudaStreamSynchronize(slot.stream));
      worst = infos[0];
      for (auto& inf : infos) {
        worst.iterations = std::max(worst.iterations, inf.iterations);
        worst.relres = std::max(worst.relres, inf.relres);
      }
    } catch (const Error& e) {
      st = e.code;
      cudaGetLastError();
    } catch (...) {
      st = LG_ERR_CUDA;
    }
    const double ms = std::chrono::duration<double, std::milli>(Clock::now() - rq->submitted).count();
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      if (ws && st == LG_OK) {  // back to the pool (the slot's stream has finished with it)
        Pooled p;
        p.h = rq->h;
        p.k = ws->k;
        p.bytes = (double)ws->bytes;
        p.last_use = ++sv->use_clock;
        p.ws = std::move(ws);
        sv->pooled_bytes += p.bytes;
        sv->pool.push_back(std::move(p));
      }
      worst.status = st;
      worst.solve_ms = ms;
      rq->info = worst;
      rq->done = true;
      sv->inflight_bytes -= rq->ws_bytes;
      sv->running -= 1;
      if (st == LG_OK) {
        sv->completed += 1;
        sv->rhs_done += rq->k;
        sv->latencies_ms.push_back(ms);
      } else {
        sv->failed += 1;
      }
    }
    sv->cv_work.notify_all();
    sv->cv_done.notify_all();
  }
}

}  // namespace lg

extern "C" {

int lg_serve_options_default(lg_serve_options* o) {
  if (!o) return LG_ERR_INVALID;
  o->hbm_budget_bytes = 120e9;
  o->slots = 8;
  o->max_queue = 1 << 16;
  o->precision = LG_FP32_HIER;
  o->reserved = 0;
  return LG_OK;
}

int lg_serve_create(const lg_serve_options* o, lg_server_t* out) {
  if (!out) return LG_ERR_INVALID;
  *out = nullptr;
  lg_serve_options opt;
  if (o) opt = *o; else lg_serve_options_default(&opt);
  if (opt.slots < 1 || opt.slots > 64 || opt.max_queue < 1 || !(opt.hbm_budget_bytes > 0.0)) return LG_ERR_INVALID;
  auto* sv = new lg::Server();
  sv->o = opt;
  if (cudaGetDevice(&sv->device) != cudaSuccess) {
    delete sv;
    return LG_ERR_CUDA;
  }
  sv->slots.resize(opt.slots);
  for (auto& sl : sv->slots) {
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto& s2 : sv->slots)
        if (s2.stream) cudaStreamDestroy(s2.stream);
      delete sv;
      return LG_ERR_CUDA;
    }
  }
  for (int i = 0; i < opt.slots; ++i) sv->threads.emplace_back(lg::serve_worker, sv, i);
  *out = reinterpret_cast<lg_server_t>(sv);
  return LG_OK;
}

int lg_serve_register(lg_server_t s, lg_handle hh) {
  if (!s || !hh) return LG_ERR_INVALID;
  auto* sv = reinterpret_cast<lg::Server*>(s);
  auto* h = reinterpret_cast<lg::Hier*>(hh);
  if (h->fp32_only && sv->o.precision != LG_FP32_HIER) return LG_ERR_INVALID;  // no FP64 operators to serve
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->resident.count(h)) return LG_OK;
  const double b = (double)h->bytes;
  if (sv->resident_bytes + b > sv->o.hbm_budget_bytes) return LG_ERR_NOMEM;
  sv->resident[h] = b;
  sv->resident_bytes += b;
  return LG_OK;
}

int lg_serve_submit(lg_server_t s, lg_handle hh, int32_t k, const double* B, double* X, double tol,
                    uint64_t* ticket) {
  if (!s || !hh || !B || !X || !ticket || k < 1 || k > lg::kMaxCols || !(tol > 0.0)) return LG_ERR_INVALID;
  auto* sv = reinterpret_cast<lg::Server*>(s);
  auto* h = reinterpret_cast<lg::Hier*>(hh);
  auto* rq = new lg::Request();
  rq->h = h;
  rq->k = k;
  rq->B = B;
  rq->X = X;
  rq->tol = tol;
  rq->ws_bytes = lg::workspace_bytes(*h, lg::pow2_width(k));
  rq->submitted = lg::Clock::now();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (!sv->resident.count(h)) {
      delete rq;
      return LG_ERR_INVALID;
    }
    if (sv->stopping || (int64_t)sv->queue.size() >= sv->o.max_queue) {
      delete rq;
      return LG_ERR_BUSY;
    }
    if (sv->resident_bytes + rq->ws_bytes > sv->o.hbm_budget_bytes) {
      delete rq;
      return LG_ERR_NOMEM;
    }
    rq->ticket = sv->next_ticket++;
    sv->requests[rq->ticket] = rq;
    sv->queue.push_back(rq);
    *ticket = rq->ticket;
  }
  sv->cv_work.notify_one();
  return LG_OK;
}

int lg_serve_poll(lg_server_t s, uint64_t ticket, int32_t* done, lg_info* info) {
  if (!s || !done) return LG_ERR_INVALID;
  auto* sv = reinterpret_cast<lg::Server*>(s);
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->requests.find(ticket);
  if (it == sv->requests.end()) return LG_ERR_INVALID;
  lg::Request* rq = it->second;
  *done = rq->done ? 1 : 0;
  if (rq->done) {
    if (info) *info = rq->info;
    sv->requests.erase(it);
    delete rq;
  }
  return LG_OK;
}

int lg_serve_request_bytes(lg_handle hh, int32_t k, double* bytes) {
  if (!hh || !bytes || k < 1 || k > lg::kMaxCols) return LG_ERR_INVALID;
  *bytes = lg::workspace_bytes(*reinterpret_cast<lg::Hier*>(hh), lg::pow2_width(k));
  return LG_OK;
}

int lg_serve_stats(lg_server_t s, lg_serve_stats_t* st) {
  if (!s || !st) return LG_ERR_INVALID;
  auto* sv = reinterpret_cast<lg::Server*>(s);
  std::lock_guard<std::mutex> lk(sv->mu);
  std::memset(st, 0, sizeof(*st));
  std::vector<double> l = sv->latencies_ms;
  std::sort(l.begin(), l.end());
  if (!l.empty()) {
    auto pct = [&](double p) {
      const double pos = p * (double)(l.size() - 1);
      const size_t i = (size_t)pos;
      const double f = pos - (double)i;
      return i + 1 < l.size() ? l[i] * (1.0 - f) + l[i + 1] * f : l[i];
    };
    st->p50_ms = pct(0.50);
    st->p99_ms = pct(0.99);
    double sum = 0.0;
    for (double v : l) sum += v;
    st->mean_ms = sum / (double)l.size();
    st->max_ms = l.back();
  }
  const double secs = std::chrono::duration<double>(lg::Clock::now() - sv->created).count();
  st->solves_per_s = secs > 0 ? (double)sv->rhs_done / secs : 0.0;
  st->resident_bytes = sv->resident_bytes;
  st->completed = sv->completed;
  st->failed = sv->failed;
  st->pending = (int64_t)sv->queue.size();
  st->running = sv->running;
  return LG_OK;
}

void lg_serve_destroy(lg_server_t s) {
  if (!s) return;
  auto* sv = reinterpret_cast<lg::Server*>(s);
  {
    std::unique_lock<std::mutex> lk(sv->mu);
    sv->cv_done.wait(lk, [&] { return sv->queue.empty() && sv->running == 0; });
    sv->stopping = true;
  }
  sv->cv_work.notify_all();
  for (auto& t : sv->threads) t.join();
  sv->pool.clear();  // workspaces before the streams they were made on
  for (auto& sl : sv->slots) {
    sl.Bd.release();
    sl.Xd.release();
    if (sl.stream) {
      cudaStreamSynchronize(sl.stream);
      cudaStreamDestroy(sl.stream);
    }
  }
  for (auto& kv : sv->requests) delete kv.second;
  delete sv;
}

}  // extern "C"
