// Continuous-batching solve server over resident hierarchies.
//
// Requests (a hierarchy, k right-hand sides in host memory, a tolerance) are
// queued by lg_serve_submit and taken by `slots` worker threads, each owning a
// CUDA stream, as soon as a slot is free and the HBM budget (registered
// hierarchies + workspaces of running groups) has room. A worker takes work
// in groups:
//  - a multi-column group: the lead request plus every queued request on the
//    same hierarchy with the same tolerance, up to kMergeCols columns in all,
//    solved together as one SpMM batch (lg_batch.cu);
//  - a packed group: single-column requests on small graphs (many different
//    hierarchies), solved in one k_solve_many launch, a thread block per
//    graph (lg_many.cu).
// Groups run concurrently on the slots' streams, so requests that arrive
// while others are on the device join the next group that starts. Which path
// a request takes depends on the request alone, and both paths compute a
// column independently of the other columns and graphs in its group, so a
// request's result is bitwise the same alone and in any mix.
//
// Which request leads the next group (the policy of lg_serve_options):
//  - arrival order: the first admissible request; one that fits the budget
//    may pass a head request that does not, at most kMaxBypass times per
//    head request, after which the head waits for room and nothing passes it;
//  - least work first: the admissible request with the least work (k times
//    the entries of its hierarchy's operators), except that a request passed
//    over kMaxBypass times leads as soon as it is admissible (the oldest such
//    first, and nothing passes it while it waits for room). Short solves then
//    no longer queue behind long ones, and no request waits forever.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>

#include "lg_hier.h"

namespace lg {

using Clock = std::chrono::steady_clock;

constexpr int kMaxBypass = 16;        // times a later request may pass the head
constexpr int kMergeCols = 8;         // columns a merged group gathers (a wider request runs alone)
constexpr int64_t kPackMaxN = 16384;  // packed path: graphs up to this many vertices...
constexpr int kPackMaxGraphs = 2048;  // ...and this many graphs per launch

struct Request {
  uint64_t ticket = 0;
  Hier* h = nullptr;
  int k = 1;
  const double* B = nullptr;
  double* X = nullptr;
  double tol = 1e-8;
  double ws_bytes = 0.0;
  double work = 0.0;    // k times the entries of every level's operator
  bool packed = false;  // single column on a small graph: the packed path
  int bypassed = 0;     // groups that started with a younger request as lead
  Clock::time_point submitted;
  bool done = false;
  lg_info info{};
};

struct Slot {
  cudaStream_t stream = nullptr;
  DBuf<double> Bd, Xd;  // staging of the running group (grown as needed)
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
  // Every pooled workspace is allocated and freed on this stream, which is
  // never captured: a worker may free (evict) a workspace another slot made
  // while that slot's stream is capturing its solve graph.
  cudaStream_t alloc_stream = nullptr;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, Request*> requests;
  std::unordered_map<Hier*, double> resident;
  std::unordered_set<Hier*> packing;  // handles in a running packed launch (their default workspace is in use)
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
  int64_t completed = 0, failed = 0, rhs_done = 0, groups = 0, packed_groups = 0, ws_made = 0;
  double ws_ms = 0.0, copy_ms = 0.0, solve_ms = 0.0;  // host time per phase, summed over groups
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

// Under the server lock: the next group to run, taken off the queue (empty:
// nothing can start now). Sets `bytes` to the budget share it reserves.
static std::vector<Request*> take_group(Server* sv, double& bytes) {
  std::vector<Request*> group;
  bytes = 0.0;
  Request* lead = nullptr;
  size_t lead_at = 0;
  const bool least_work = sv->o.policy == LG_SERVE_LEAST_WORK;
  // room: the budget has space for the request (or nothing runs); busy: a
  // packed request whose handle is in a running launch (it waits for that)
  const auto room = [&](const Request* rq) {
    return rq->packed || sv->resident_bytes + sv->inflight_bytes + rq->ws_bytes <= sv->o.hbm_budget_bytes ||
           sv->running == 0;
  };
  const auto busy = [&](const Request* rq) { return rq->packed && sv->packing.count(rq->h) > 0; };
  if (!least_work) {
    for (size_t q = 0; q < sv->queue.size(); ++q) {
      Request* rq = sv->queue[q];
      if (!busy(rq) && room(rq)) {
        lead = rq;
        lead_at = q;
        break;
      }
      if (q == 0 && !rq->packed && rq->bypassed >= kMaxBypass) return group;  // the head has waited long enough
    }
    if (!lead) return group;
    if (lead_at > 0 && !sv->queue.front()->packed) sv->queue.front()->bypassed += 1;
  } else {
    for (size_t q = 0; q < sv->queue.size(); ++q) {
      Request* rq = sv->queue[q];
      if (busy(rq)) continue;
      if (rq->bypassed >= kMaxBypass) {  // the oldest aged request leads, or waits for room
        if (!room(rq)) return group;
        lead = rq;
        lead_at = q;
        break;
      }
      if (room(rq) && (!lead || rq->work < lead->work)) {
        lead = rq;
        lead_at = q;
      }
    }
    if (!lead) return group;
    for (size_t q = 0; q < lead_at; ++q) sv->queue[q]->bypassed += 1;  // every older request was passed
  }
  const size_t from = least_work ? 0 : lead_at + 1;  // merging looks at older requests too under least work
  std::vector<char> take(sv->queue.size(), 0);
  take[lead_at] = 1;
  group.push_back(lead);
  if (lead->packed) {
    // other single-column small-graph requests with the same tolerance, one per handle
    std::unordered_set<Hier*> seen{lead->h};
    for (size_t q = from; q < sv->queue.size() && (int)group.size() < kPackMaxGraphs; ++q) {
      Request* rq = sv->queue[q];
      if (take[q] || !rq->packed || rq->tol != lead->tol || seen.count(rq->h) || sv->packing.count(rq->h)) continue;
      seen.insert(rq->h);
      take[q] = 1;
      group.push_back(rq);
    }
    for (Request* rq : group) {
      sv->packing.insert(rq->h);
      bytes += rq->ws_bytes;
    }
  } else {
    // the queued requests on the same hierarchy and tolerance, up to the widest batch
    int cols = lead->k;
    bytes = lead->ws_bytes;
    for (size_t q = from; q < sv->queue.size(); ++q) {
      Request* rq = sv->queue[q];
      if (take[q] || rq->packed || rq->h != lead->h || rq->tol != lead->tol || cols + rq->k > kMergeCols) continue;
      const double b = workspace_bytes(*lead->h, pow2_width(cols + rq->k));
      if (sv->resident_bytes + sv->inflight_bytes + b > sv->o.hbm_budget_bytes) continue;  // the budget holds
      cols += rq->k;
      bytes = b;
      take[q] = 1;
      group.push_back(rq);
    }
  }
  std::deque<Request*> rest;
  for (size_t q = 0; q < sv->queue.size(); ++q)
    if (!take[q]) rest.push_back(sv->queue[q]);
  sv->queue.swap(rest);
  return group;
}

// A multi-column group: the columns of every request side by side, one
// batched solve, each request's columns back out. Returns per-request status
// and fills their infos (worst column).
static double ms_since(Clock::time_point t) {
  return std::chrono::duration<double, std::milli>(Clock::now() - t).count();
}

// Phase times of one group, added to the server's totals on completion.
struct GroupTimes {
  double ws = 0.0, copy = 0.0, solve = 0.0;
  int made = 0;
};

static void run_columns(Server* sv, Slot& slot, std::vector<Request*>& group, std::unique_ptr<Workspace>& ws,
                        std::vector<int>& status, GroupTimes& tm) {
  Hier& h = *group[0]->h;
  const int64_t n = h.levels[0]->n;
  int cols = 0;
  for (Request* rq : group) cols += rq->k;
  if (!ws) {
    const Clock::time_point t = Clock::now();
    ws = make_workspace(h, pow2_width(cols), sv->alloc_stream);
    LG_CUDA(cudaStreamSynchronize(sv->alloc_stream));
    tm.ws += ms_since(t);
    tm.made += 1;
  }
  const size_t need = (size_t)n * cols;
  if (slot.staged < need) {
    slot.Bd.alloc(need, slot.stream);
    slot.Xd.alloc(need, slot.stream);
    slot.staged = need;
  }
  Clock::time_point t = Clock::now();
  size_t off = 0;
  for (Request* rq : group) {
    LG_CUDA(cudaMemcpyAsync(slot.Bd.get() + off, rq->B, sizeof(double) * n * rq->k, cudaMemcpyHostToDevice,
                            slot.stream));
    off += (size_t)n * rq->k;
  }
  LG_CUDA(cudaStreamSynchronize(slot.stream));
  tm.copy += ms_since(t);
  t = Clock::now();
  std::vector<lg_info> infos(cols);
  pcg_solve_columns(h, *ws, cols, slot.Bd.get(), slot.Xd.get(), group[0]->tol, sv->o.precision, slot.stream,
                    infos.data());
  tm.solve += ms_since(t);
  t = Clock::now();
  off = 0;
  int c0 = 0;
  for (size_t g = 0; g < group.size(); ++g) {
    Request* rq = group[g];
    LG_CUDA(cudaMemcpyAsync(rq->X, slot.Xd.get() + off, sizeof(double) * n * rq->k, cudaMemcpyDeviceToHost,
                            slot.stream));
    off += (size_t)n * rq->k;
    lg_info worst = infos[c0];
    int st = LG_OK;
    for (int c = c0; c < c0 + rq->k; ++c) {
      worst.iterations = std::max(worst.iterations, infos[c].iterations);
      worst.relres = std::max(worst.relres, infos[c].relres);
      if (infos[c].status != LG_OK && st == LG_OK) st = infos[c].status;
    }
    rq->info = worst;
    status[g] = st;
    c0 += rq->k;
  }
  LG_CUDA(cudaStreamSynchronize(slot.stream));
  tm.copy += ms_since(t);
}

// A packed group: one k_solve_many launch over the requests' graphs.
static void run_packed(Server* sv, std::vector<Request*>& group, std::vector<int>& status, GroupTimes& tm) {
  const Clock::time_point t = Clock::now();
  const int count = (int)group.size();
  std::vector<Hier*> hs(count);
  std::vector<const double*> b(count);
  std::vector<double*> x(count);
  std::unique_ptr<bool[]> bd(new bool[count]), xd(new bool[count]);
  for (int g = 0; g < count; ++g) {
    hs[g] = group[g]->h;
    b[g] = group[g]->B;
    x[g] = group[g]->X;
    bd[g] = false;
    xd[g] = false;
  }
  std::vector<lg_info> infos(count);
  solve_many(count, hs.data(), b.data(), x.data(), bd.get(), xd.get(), group[0]->tol, infos.data(),
             sv->o.precision);
  tm.solve += ms_since(t);
  for (int g = 0; g < count; ++g) {
    group[g]->info = infos[g];
    status[g] = infos[g].status;
  }
}

static void serve_worker(Server* sv, int slot_id) {
  Slot& slot = sv->slots[slot_id];
  cudaSetDevice(sv->device);
  for (;;) {
    std::vector<Request*> group;
    double bytes = 0.0;
    std::unique_ptr<Workspace> ws;
    std::vector<std::unique_ptr<Workspace>> evicted;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      sv->cv_work.wait(lk, [&] {
        if (sv->queue.empty()) return sv->stopping;
        group = take_group(sv, bytes);
        return !group.empty();
      });
      if (group.empty()) return;  // stopping with nothing left
      if (!group[0]->packed) {
        int cols = 0;
        for (Request* rq : group) cols += rq->k;
        ws = pool_take(sv, group[0]->h, pow2_width(cols));
        if (!ws) pool_evict(sv, bytes, evicted);
      }
      sv->inflight_bytes += bytes;
      sv->running += 1;
    }
    evicted.clear();  // frees the evicted workspaces' device memory
    std::vector<int> status(group.size(), LG_OK);
    int err = LG_OK;
    GroupTimes tm;
    try {
      if (group[0]->packed) run_packed(sv, group, status, tm);
      else run_columns(sv, slot, group, ws, status, tm);
    } catch (const Error& e) {
      err = e.code;
      cudaGetLastError();
    } catch (...) {
      err = LG_ERR_CUDA;
    }
    const Clock::time_point now = Clock::now();
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      if (ws && err == LG_OK) {  // back to the pool (the slot's stream has finished with it)
        Pooled p;
        p.h = group[0]->h;
        p.k = ws->k;
        p.bytes = (double)ws->bytes;
        p.last_use = ++sv->use_clock;
        p.ws = std::move(ws);
        sv->pooled_bytes += p.bytes;
        sv->pool.push_back(std::move(p));
      }
      for (size_t g = 0; g < group.size(); ++g) {
        Request* rq = group[g];
        const int st = err != LG_OK ? err : status[g];
        const double ms = std::chrono::duration<double, std::milli>(now - rq->submitted).count();
        rq->info.status = st;
        rq->info.solve_ms = ms;
        rq->done = true;
        if (rq->packed) sv->packing.erase(rq->h);
        if (st == LG_OK) {
          sv->completed += 1;
          sv->rhs_done += rq->k;
          sv->latencies_ms.push_back(ms);
        } else {
          sv->failed += 1;
        }
      }
      sv->groups += 1;
      if (group[0]->packed) sv->packed_groups += 1;
      sv->ws_made += tm.made;
      sv->ws_ms += tm.ws;
      sv->copy_ms += tm.copy;
      sv->solve_ms += tm.solve;
      sv->inflight_bytes -= bytes;
      sv->running -= 1;
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
  o->policy = LG_SERVE_ARRIVAL;
  return LG_OK;
}

int lg_serve_create(const lg_serve_options* o, lg_server_t* out) {
  if (!out) return LG_ERR_INVALID;
  *out = nullptr;
  lg_serve_options opt;
  if (o) opt = *o; else lg_serve_options_default(&opt);
  if (opt.slots < 1 || opt.slots > 64 || opt.max_queue < 1 || !(opt.hbm_budget_bytes > 0.0) ||
      (opt.policy != LG_SERVE_ARRIVAL && opt.policy != LG_SERVE_LEAST_WORK))
    return LG_ERR_INVALID;
  auto* sv = new lg::Server();
  sv->o = opt;
  if (cudaGetDevice(&sv->device) != cudaSuccess) {
    delete sv;
    return LG_ERR_CUDA;
  }
  sv->slots.resize(opt.slots);
  // Workspaces come and go with the load: keep the memory they free in the
  // device's stream-ordered pool (up to the budget) instead of handing it
  // back at every synchronisation, so the next one is allocated without
  // mapping pages again. A process-local setting of this device's pool.
  {
    cudaMemPool_t pool = nullptr;
    if (cudaDeviceGetDefaultMemPool(&pool, sv->device) == cudaSuccess) {
      uint64_t keep = (uint64_t)opt.hbm_budget_bytes;
      uint64_t cur = 0;
      if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &cur) == cudaSuccess && cur < keep)
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
  }
  bool ok = cudaStreamCreateWithFlags(&sv->alloc_stream, cudaStreamNonBlocking) == cudaSuccess;
  for (auto& sl : sv->slots)
    ok = ok && cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) == cudaSuccess;
  if (!ok) {
    for (auto& s2 : sv->slots)
      if (s2.stream) cudaStreamDestroy(s2.stream);
    if (sv->alloc_stream) cudaStreamDestroy(sv->alloc_stream);
    delete sv;
    return LG_ERR_CUDA;
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
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->resident.count(h)) return LG_OK;
  }
  // what a first request would otherwise build inside its latency: the
  // multi-column plans and, for graphs the packed path serves, its views
  try {
    lg::prepare_columns(*h, 8, sv->o.precision);
    if (h->levels[0]->n <= lg::kPackMaxN && h->nnz0 <= lg::kManyMaxNnz && (int)h->levels.size() <= lg::kManyMaxLevels &&
        !h->opts.kcycle)
      lg::prepare_many(*h);
  } catch (const lg::Error& e) {
    lg::g_last_error = e.what ? e.what : "";
    return e.code;
  }
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->resident.count(h)) return LG_OK;
    const double b = (double)h->bytes;
    if (sv->resident_bytes + b > sv->o.hbm_budget_bytes) return LG_ERR_NOMEM;
    sv->resident[h] = b;
    sv->resident_bytes += b;
    // room for a ready workspace of kMergeCols columns as well?
    if (sv->resident_bytes + sv->inflight_bytes + sv->pooled_bytes + lg::workspace_bytes(*h, lg::kMergeCols) >
        sv->o.hbm_budget_bytes)
      return LG_OK;
  }
  // A workspace of kMergeCols columns with its solve loops captured, put in
  // the pool: the first requests on h need neither (captured on a stream of
  // this call, the workspace's memory on the server's allocation stream).
  try {
    auto ws = lg::make_workspace(*h, lg::kMergeCols, sv->alloc_stream);
    LG_CUDA(cudaStreamSynchronize(sv->alloc_stream));
    cudaStream_t cap = nullptr;
    LG_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    struct StreamGuard {
      cudaStream_t s;
      ~StreamGuard() {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
      }
    } guard{cap};
    lg::prepare_column_graphs(*h, *ws, sv->o.precision, cap);
    std::lock_guard<std::mutex> lk(sv->mu);
    lg::Pooled p;
    p.h = h;
    p.k = ws->k;
    p.bytes = (double)ws->bytes;
    p.last_use = ++sv->use_clock;
    p.ws = std::move(ws);
    sv->pooled_bytes += p.bytes;
    sv->pool.push_back(std::move(p));
  } catch (const lg::Error& e) {  // the hierarchy is registered; its first request builds what it needs
    lg::g_last_error = e.what ? e.what : "";
    cudaGetLastError();
  }
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
  rq->packed = k == 1 && h->levels[0]->n <= lg::kPackMaxN && h->nnz0 <= lg::kManyMaxNnz &&
               (int)h->levels.size() <= lg::kManyMaxLevels && !h->opts.kcycle;
  // a packed request runs in its handle's default workspace: only its staging is extra
  rq->ws_bytes = rq->packed ? 16.0 * (double)h->levels[0]->n + 4096.0 : lg::workspace_bytes(*h, lg::pow2_width(k));
  for (const auto& L : h->levels) rq->work += (double)(L->nnz + L->n);
  rq->work *= k;
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
  st->groups = sv->groups;
  st->packed_groups = sv->packed_groups;
  st->workspaces_made = sv->ws_made;
  st->workspace_ms = sv->ws_ms;
  st->copy_ms = sv->copy_ms;
  st->solve_ms = sv->solve_ms;
  return LG_OK;
}

int lg_serve_reset_stats(lg_server_t s) {
  if (!s) return LG_ERR_INVALID;
  auto* sv = reinterpret_cast<lg::Server*>(s);
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->latencies_ms.clear();
  sv->completed = sv->failed = sv->rhs_done = sv->groups = sv->packed_groups = sv->ws_made = 0;
  sv->ws_ms = sv->copy_ms = sv->solve_ms = 0.0;
  sv->created = lg::Clock::now();
  return LG_OK;
}

int lg_serve_set_policy(lg_server_t s, int32_t policy) {
  if (!s || (policy != LG_SERVE_ARRIVAL && policy != LG_SERVE_LEAST_WORK)) return LG_ERR_INVALID;
  auto* sv = reinterpret_cast<lg::Server*>(s);
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->o.policy = policy;
  }
  sv->cv_work.notify_all();
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
  sv->pool.clear();  // workspaces before the stream they were made on
  for (auto& sl : sv->slots) {
    sl.Bd.release();
    sl.Xd.release();
    if (sl.stream) {
      cudaStreamSynchronize(sl.stream);
      cudaStreamDestroy(sl.stream);
    }
  }
  if (sv->alloc_stream) {
    cudaStreamSynchronize(sv->alloc_stream);
    cudaStreamDestroy(sv->alloc_stream);
  }
  for (auto& kv : sv->requests) delete kv.second;
  delete sv;
}

}  // extern "C"
