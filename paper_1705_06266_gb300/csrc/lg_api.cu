// extern "C" entry points of include/lg.h: argument checks, pointer-space
// detection, handle lifecycle, and the mapping of library errors to status
// codes. No entry point lets an exception or a CUDA error escape.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "lg_hier.h"

namespace lg {

thread_local std::string g_last_error;
std::atomic<uint64_t> g_launches{0};
static thread_local char g_launch_msg[256];

bool debug_sync() {
  static const bool on = [] {
    const char* v = std::getenv("LG_DEBUG_SYNC");
    return v && v[0] == '1';
  }();
  return on;
}

void check_launch(const char* file, int line) {
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && debug_sync()) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) return;
  const char* base = std::strrchr(file, '/');
  std::snprintf(g_launch_msg, sizeof(g_launch_msg), "kernel at %s:%d: %s", base ? base + 1 : file, line,
                cudaGetErrorName(e));
  fail(e == cudaErrorMemoryAllocation ? LG_ERR_NOMEM : LG_ERR_CUDA, g_launch_msg);
}

Hier::~Hier() {
  // every stream-ordered buffer goes back on the handle's stream before that
  // stream is destroyed
  ws.reset();
  wsb.reset();
  many.reset();
  mplans.reset();
  levels.clear();
  dev_err.release();
  perm.release();
  if (stream) cudaStreamSynchronize(stream);
  if (own_stream && stream) cudaStreamDestroy(stream);
}

static bool is_device_ptr(const void* p, int memory_space) {
  if (memory_space == LG_DEVICE) return true;
  if (memory_space == LG_HOST) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

__global__ void k_fill_value(double* __restrict__ a, double v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = v;
}

// n copies of v into a (device or host memory), ordered on stream s.
static void fill_value(double* a, double v, int64_t n, int memory_space, cudaStream_t s) {
  if (is_device_ptr(a, memory_space)) {
    k_fill_value<<<grid_for(n, 256, kSMs * 8), 256, 0, s>>>(a, v, n);
    LG_LAUNCH_CHECK();
  } else {
    LG_CUDA(cudaStreamSynchronize(s));
    std::fill_n(a, n, v);
  }
}

// One JSON line per setup and per solved right-hand side, appended to the
// file named by the environment variable LG_LOG (nothing when it is unset).
static std::mutex g_log_mu;

static bool log_on() {
  const char* p = std::getenv("LG_LOG");
  return p && *p;
}

static void log_line(const char* line) {
  const char* path = std::getenv("LG_LOG");
  if (!path || !*path) return;
  std::lock_guard<std::mutex> lk(g_log_mu);
  if (FILE* f = std::fopen(path, "a")) {
    std::fputs(line, f);
    std::fputc('\n', f);
    std::fclose(f);
  }
}

static void log_solve(const char* call, int index, const lg_info& inf) {
  char wda[40] = "null";  // work units per digit of residual reduction (Section 2.3.1)
  if (inf.relres > 0.0 && inf.relres < 1.0 && std::isfinite(inf.relres))
    std::snprintf(wda, sizeof(wda), "%.9g", inf.work_units / -std::log10(inf.relres));
  char line[640];
  std::snprintf(line, sizeof(line),
                "{\"call\": \"%s\", \"index\": %d, \"status\": %d, \"iterations\": %d, \"relres\": %.17g, "
                "\"solve_ms\": %.9g, \"setup_ms\": %.9g, \"work_units\": %.9g, \"wda\": %s, \"levels\": %d, "
                "\"nnz\": %lld, \"op_complexity\": %.9g}",
                call, index, inf.status, inf.iterations, std::isfinite(inf.relres) ? inf.relres : -1.0, inf.solve_ms,
                inf.setup_ms, inf.work_units, wda, inf.levels, (long long)inf.nnz, inf.op_complexity);
  log_line(line);
}

static int handle_error(const Error& e) {
  g_last_error = e.what ? e.what : "";
  cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) {
    g_last_error += ": ";
    g_last_error += cudaGetErrorName(ce);
  }
  return e.code;
}

}  // namespace lg

using lg::Error;

#define LG_API_BEGIN try {
#define LG_API_END                                              \
  }                                                             \
  catch (const lg::Error& e) { return lg::handle_error(e); }    \
  catch (const std::bad_alloc&) {                               \
    lg::g_last_error = "host allocation";                       \
    return LG_ERR_NOMEM;                                        \
  }                                                             \
  catch (...) {                                                 \
    lg::g_last_error = "unexpected exception";                  \
    return LG_ERR_CUDA;                                         \
  }

extern "C" {

const char* lg_last_error_detail(void) { return lg::g_last_error.c_str(); }

int lg_options_default(lg_options* o) {
  if (!o) return LG_ERR_INVALID;
  std::memset(o, 0, sizeof(*o));
  o->coarse_nnz = 1000.0;
  o->elim_min_frac = 0.05;
  o->jacobi_omega = 2.0 / 3.0;
  o->cheb_lo = 0.3;
  o->cheb_hi = 1.1;
  o->stagnation_frac = 0.95;
  o->seed = 0x5eed;
  o->stream = nullptr;
  o->precision = LG_FP64;
  o->max_levels = 64;
  o->max_iter = 500;
  o->elim_enable = 1;
  o->elim_max_degree = 4;
  o->agg_iters = 10;
  o->vote_threshold = 8;
  o->strength_vecs = 4;
  o->strength_sweeps = 3;
  o->cheb_degree = 2;
  o->eig_iters = 10;
  o->max_coarse_n = 4096;
  o->residual_replace = 50;
  o->memory_space = LG_AUTO;
  o->use_graphs = 1;
  o->autotune = 1;
  o->reorder = 1;
  o->kcycle = 0;
  o->elim_rounds = 1;
  o->lp_residual = 1;
  o->fp32_only = 0;
  o->const_weights = 1;
  o->row_sorts = 1;
  return LG_OK;
}

const char* lg_error_string(int status) {
  switch (status) {
    case LG_OK: return "ok";
    case LG_ERR_INVALID: return "invalid argument or graph";
    case LG_ERR_DISCONNECTED: return "graph is not connected";
    case LG_ERR_SETUP: return "coarsening failed to reach a small enough coarsest level";
    case LG_ERR_NOMEM: return "out of device memory or HBM budget";
    case LG_ERR_NOT_CONVERGED: return "not converged within max_iter";
    case LG_ERR_BREAKDOWN: return "CG breakdown (non-finite or non-positive scalar)";
    case LG_ERR_TIMEOUT: return "bounded wait or retry loop gave up";
    case LG_ERR_CUDA: return "CUDA runtime error";
    case LG_ERR_BUSY: return "server busy";
    default: return "unknown status";
  }
}

int lg_setup(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w, const lg_options* opts,
             lg_handle* out) {
  if (!out) return LG_ERR_INVALID;
  *out = nullptr;
  if (n < 1 || n >= (int64_t(1) << 31) || !rowptr || !col || !w) return LG_ERR_INVALID;
  lg::Hier* h = nullptr;
  LG_API_BEGIN
  h = new lg::Hier();
  lg::NvtxRange range("lg_setup");
  if (opts) h->opts = *opts; else lg_options_default(&h->opts);
  LG_CUDA(cudaGetDevice(&h->device));
  if (h->opts.stream) {
    h->stream = (cudaStream_t)h->opts.stream;
  } else {
    LG_CUDA(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    h->own_stream = true;
  }
  h->time_stages = lg::log_on();
  lg::setup_hierarchy(*h, n, rowptr, col, w);
  h->ws = lg::make_workspace(*h, 1, h->stream);
  LG_CUDA(cudaStreamSynchronize(h->stream));
  if (lg::log_on()) {
    std::string stages = "{";
    for (const auto& st : h->setup_stages) {
      char item[96];
      std::snprintf(item, sizeof(item), "%s\"%s\": %.6g", stages.size() > 1 ? ", " : "", st.first.c_str(), st.second);
      stages += item;
    }
    stages += "}";
    char head[256];
    std::snprintf(head, sizeof(head),
                  "{\"call\": \"lg_setup\", \"n\": %lld, \"nnz\": %lld, \"levels\": %d, \"setup_ms\": %.9g, "
                  "\"hierarchy_bytes\": %lld, \"stages_ms\": ",
                  (long long)n, (long long)h->nnz0, (int)h->levels.size(), h->setup_ms, (long long)h->bytes);
    lg::log_line((std::string(head) + stages + "}").c_str());
  }
  *out = reinterpret_cast<lg_handle>(h);
  h = nullptr;
  return LG_OK;
  }
  catch (const lg::Error& e) {
    delete h;
    return lg::handle_error(e);
  }
  catch (...) {
    delete h;
    lg::g_last_error = "unexpected exception";
    return LG_ERR_CUDA;
  }
}

int lg_save(lg_handle hh, const char* path) {
  if (!hh || !path) return LG_ERR_INVALID;
  if (reinterpret_cast<lg::Hier*>(hh)->fp32_only) {
    lg::g_last_error = "lg_save: an fp32_only hierarchy has released the FP64 arrays a file holds";
    return LG_ERR_INVALID;
  }
  LG_API_BEGIN
  lg::save_hierarchy(*reinterpret_cast<lg::Hier*>(hh), path);
  return LG_OK;
  LG_API_END
}

int lg_load(const char* path, const lg_options* opts, lg_handle* out) {
  if (!out) return LG_ERR_INVALID;
  *out = nullptr;
  if (!path) return LG_ERR_INVALID;
  lg::Hier* h = nullptr;
  try {
    h = new lg::Hier();
    lg::load_hierarchy(*h, path, opts);
    *out = reinterpret_cast<lg_handle>(h);
    return LG_OK;
  } catch (const lg::Error& e) {
    delete h;
    return lg::handle_error(e);
  } catch (const std::bad_alloc&) {
    delete h;
    lg::g_last_error = "host allocation";
    return LG_ERR_NOMEM;
  } catch (...) {
    delete h;
    lg::g_last_error = "unexpected exception";
    return LG_ERR_CUDA;
  }
}

void lg_destroy(lg_handle hh) {
  try {
    delete reinterpret_cast<lg::Hier*>(hh);
  } catch (...) {
  }
}

static lg::Hier* H(lg_handle h) { return reinterpret_cast<lg::Hier*>(h); }

int lg_set_precision(lg_handle hh, int32_t precision) {
  if (!hh || (precision != LG_FP64 && precision != LG_FP32_HIER)) return LG_ERR_INVALID;
  if (precision == LG_FP64 && H(hh)->fp32_only) {
    lg::g_last_error = "lg_set_precision: an fp32_only hierarchy serves FP32-hierarchy solves only";
    return LG_ERR_INVALID;
  }
  H(hh)->opts.precision = precision;
  return LG_OK;
}

int lg_solve(lg_handle hh, const double* b, double* x, double tol, lg_info* info) {
  if (!hh || !b || !x || !(tol > 0.0)) return LG_ERR_INVALID;
  LG_API_BEGIN
  lg::NvtxRange range("lg_solve");
  lg::Hier& h = *H(hh);
  cudaStream_t s = h.stream;
  const int64_t n = h.levels[0]->n;
  lg::DBuf<double> staged;
  const double* bd = b;
  if (!lg::is_device_ptr(b, h.opts.memory_space)) {
    staged.alloc(n, s);
    LG_CUDA(cudaMemcpyAsync(staged.get(), b, sizeof(double) * n, cudaMemcpyDefault, s));
    bd = staged.get();
  }
  lg_info inf{};
  int st = lg::pcg_solve(h, *h.ws, bd, x, tol, h.opts.precision, s, &inf);
  inf.op_complexity = 0.0;
  for (auto& L : h.levels) inf.op_complexity += (double)(L->nnz + L->n);
  inf.op_complexity /= (double)h.nnz0;
  if (info) *info = inf;
  if (lg::log_on()) lg::log_solve("lg_solve", 0, inf);
  return st;
  LG_API_END
}

int lg_solve_batch(lg_handle hh, int32_t k, const double* B, int64_t ldb, double* X, int64_t ldx, double tol,
                   lg_info* infos) {
  if (!hh || !B || !X || k < 1 || k > lg::kMaxCols || !(tol > 0.0)) return LG_ERR_INVALID;
  lg::Hier& h = *H(hh);
  const int64_t n = h.levels[0]->n;
  if (ldb < n || ldx < n) return LG_ERR_INVALID;
  LG_API_BEGIN
  lg::NvtxRange range("lg_solve_batch");
  cudaStream_t s = h.stream;
  lg::DBuf<double> Bd((size_t)n * k, s), Xd((size_t)n * k, s);
  for (int c = 0; c < k; ++c)
    LG_CUDA(cudaMemcpyAsync(Bd.get() + (size_t)c * n, B + (size_t)c * ldb, sizeof(double) * n, cudaMemcpyDefault, s));
  int kp = 1;
  while (kp < k) kp <<= 1;  // multi-column vectors are [n][k rounded up to a power of two]
  if (k > 1 && (!h.wsb || h.wsb->k < kp)) {
    h.wsb.reset();
    h.wsb = lg::make_workspace(h, kp, s);
  }
  std::vector<lg_info> own;
  lg_info* out = infos;
  if (!out && lg::log_on()) {
    own.resize((size_t)k);
    out = own.data();
  }
  int st = lg::pcg_solve_batch(h, k > 1 ? *h.wsb : *h.ws, k, Bd.get(), Xd.get(), tol, h.opts.precision, s, out);
  for (int c = 0; c < k; ++c)
    LG_CUDA(cudaMemcpyAsync(X + (size_t)c * ldx, Xd.get() + (size_t)c * n, sizeof(double) * n, cudaMemcpyDefault, s));
  LG_CUDA(cudaStreamSynchronize(s));
  if (out && lg::log_on())
    for (int c = 0; c < k; ++c) lg::log_solve("lg_solve_batch", c, out[c]);
  return st;
  LG_API_END
}

int lg_solve_many(int32_t count, const lg_handle* hs, const double* const* b, double* const* x, double tol,
                  lg_info* infos) {
  if (count < 1 || !hs || !b || !x || !(tol > 0.0)) return LG_ERR_INVALID;
  std::vector<lg::Hier*> v((size_t)count);
  for (int g = 0; g < count; ++g) {
    v[g] = H(hs[g]);
    if (!v[g] || !b[g] || !x[g]) return LG_ERR_INVALID;
    if (v[g]->nnz0 > lg::kManyMaxNnz || (int)v[g]->levels.size() > lg::kManyMaxLevels) return LG_ERR_INVALID;
  }
  {
    std::vector<lg::Hier*> sorted(v);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) return LG_ERR_INVALID;
  }
  {
    // the outputs x[g] (n_g doubles each) must not overlap one another nor
    // another graph's input b[g']: the packed kernel writes every x while
    // other blocks read their b. Inputs may share memory with each other
    // (they are only read), and a graph's own b may be its x.
    struct Span {
      uintptr_t beg, end;
      int g;
      bool operator<(const Span& o) const { return beg < o.beg; }
    };
    std::vector<Span> xs((size_t)count);
    for (int g = 0; g < count; ++g) {
      const uintptr_t a = reinterpret_cast<uintptr_t>(x[g]);
      xs[g] = Span{a, a + sizeof(double) * (uintptr_t)v[g]->levels[0]->n, g};
    }
    std::sort(xs.begin(), xs.end());
    for (int g = 1; g < count; ++g)
      if (xs[g].beg < xs[g - 1].end) return LG_ERR_INVALID;
    for (int g = 0; g < count; ++g) {
      const uintptr_t a = reinterpret_cast<uintptr_t>(b[g]);
      const uintptr_t e = a + sizeof(double) * (uintptr_t)v[g]->levels[0]->n;
      // x spans are disjoint and sorted, so their ends ascend too: walk the
      // ones that end after a and start before e
      auto it = std::upper_bound(xs.begin(), xs.end(), a, [](uintptr_t p, const Span& sp) { return p < sp.end; });
      for (; it != xs.end() && it->beg < e; ++it)
        if (it->g != g) return LG_ERR_INVALID;
    }
  }
  LG_API_BEGIN
  lg::NvtxRange range("lg_solve_many");
  int dev = 0;
  LG_CUDA(cudaGetDevice(&dev));
  std::unique_ptr<bool[]> bd(new bool[count]), xd(new bool[count]);
  for (int g = 0; g < count; ++g) {
    if (v[g]->device != dev) return LG_ERR_INVALID;
    bd[g] = lg::is_device_ptr(b[g], v[g]->opts.memory_space);
    xd[g] = lg::is_device_ptr(x[g], v[g]->opts.memory_space);
  }
  std::vector<lg_info> own;
  lg_info* out = infos;
  if (!out && lg::log_on()) {
    own.resize((size_t)count);
    out = own.data();
  }
  const int st = lg::solve_many(count, v.data(), b, x, bd.get(), xd.get(), tol, out);
  if (out && lg::log_on())
    for (int g = 0; g < count; ++g) lg::log_solve("lg_solve_many", g, out[g]);
  return st;
  LG_API_END
}

int lg_hier_info(lg_handle hh, lg_info* info) {
  if (!hh || !info) return LG_ERR_INVALID;
  lg::Hier& h = *H(hh);
  std::memset(info, 0, sizeof(*info));
  info->levels = (int)h.levels.size();
  info->setup_ms = h.setup_ms;
  info->nnz = h.nnz0;
  double oc = 0.0;
  for (auto& L : h.levels) oc += (double)(L->nnz + L->n);
  info->op_complexity = oc / (double)h.nnz0;
  return LG_OK;
}

int lg_hier_bytes(lg_handle hh, int64_t* hb, int64_t* wb) {
  if (!hh) return LG_ERR_INVALID;
  if (hb) *hb = H(hh)->bytes;
  if (wb) *wb = H(hh)->ws ? H(hh)->ws->bytes : 0;
  return LG_OK;
}

int lg_level_info(lg_handle hh, int32_t l, int32_t* kind, int64_t* n, int64_t* nnz, int64_t* nc, double* lambda) {
  if (!hh) return LG_ERR_INVALID;
  lg::Hier& h = *H(hh);
  if (l < 0 || l >= (int32_t)h.levels.size()) return LG_ERR_INVALID;
  const lg::Level& L = *h.levels[l];
  if (kind) *kind = L.kind;
  if (n) *n = L.n;
  if (nnz) *nnz = L.nnz;
  if (nc) *nc = L.kind == LG_LEVEL_COARSEST ? 0 : L.nc;
  if (lambda) *lambda = L.lambda;
  return LG_OK;
}

int lg_level_copy(lg_handle hh, int32_t l, int64_t* rowptr, int32_t* col, double* w, int32_t* map) {
  if (!hh) return LG_ERR_INVALID;
  lg::Hier& h = *H(hh);
  if (l < 0 || l >= (int32_t)h.levels.size()) return LG_ERR_INVALID;
  if (h.fp32_only && l > 0 && h.levels[l]->kind != LG_LEVEL_COARSEST) {
    lg::g_last_error = "lg_level_copy: an fp32_only hierarchy has released this level's FP64 operator";
    return LG_ERR_INVALID;
  }
  LG_API_BEGIN
  const lg::Level& L = *h.levels[l];
  cudaStream_t s = h.stream;
  if (rowptr) LG_CUDA(cudaMemcpyAsync(rowptr, L.rowptr.get(), sizeof(int64_t) * (L.n + 1), cudaMemcpyDefault, s));
  if (col && L.nnz) LG_CUDA(cudaMemcpyAsync(col, L.col.get(), sizeof(int32_t) * L.nnz, cudaMemcpyDefault, s));
  if (w && L.nnz) {
    if (L.wconst_on)
      lg::fill_value(w, L.wconst, L.nnz, h.opts.memory_space, s);
    else
      LG_CUDA(cudaMemcpyAsync(w, L.w.get(), sizeof(double) * L.nnz, cudaMemcpyDefault, s));
  }
  if (map) {
    if (L.kind == LG_LEVEL_AGG)
      LG_CUDA(cudaMemcpyAsync(map, L.agg.get(), sizeof(int32_t) * L.n, cudaMemcpyDefault, s));
    else if (L.kind == LG_LEVEL_ELIM)
      LG_CUDA(cudaMemcpyAsync(map, L.cmap.get(), sizeof(int32_t) * L.n, cudaMemcpyDefault, s));
  }
  LG_CUDA(cudaStreamSynchronize(s));
  return LG_OK;
  LG_API_END
}

int lg_permutation(lg_handle hh, int32_t* perm) {
  if (!hh || !perm) return LG_ERR_INVALID;
  LG_API_BEGIN
  lg::Hier& h = *H(hh);
  const int64_t n = h.levels[0]->n;
  LG_CUDA(cudaMemcpyAsync(perm, h.perm.get(), sizeof(int32_t) * n, cudaMemcpyDefault, h.stream));
  LG_CUDA(cudaStreamSynchronize(h.stream));
  return LG_OK;
  LG_API_END
}

int lg_coarsest_pinv(lg_handle hh, double* out) {
  if (!hh || !out) return LG_ERR_INVALID;
  LG_API_BEGIN
  lg::Hier& h = *H(hh);
  const lg::Level& L = *h.levels.back();
  LG_CUDA(cudaMemcpyAsync(out, L.pinv.get(), sizeof(double) * L.n * L.n, cudaMemcpyDefault, h.stream));
  LG_CUDA(cudaStreamSynchronize(h.stream));
  return LG_OK;
  LG_API_END
}

int lg_vcycle(lg_handle hh, const double* f, double* x, int32_t precision) {
  if (!hh || !f || !x || (precision != LG_FP64 && precision != LG_FP32_HIER)) return LG_ERR_INVALID;
  if (precision == LG_FP64 && H(hh)->fp32_only) return LG_ERR_INVALID;
  LG_API_BEGIN
  lg::Hier& h = *H(hh);
  cudaStream_t s = h.stream;
  const int64_t n = h.levels[0]->n;
  lg::DBuf<double> fd, xd;
  const double* fp = f;
  double* xp = x;
  const bool fdev = lg::is_device_ptr(f, h.opts.memory_space);
  const bool xdev = lg::is_device_ptr(x, h.opts.memory_space);
  if (!fdev) {
    fd.alloc(n, s);
    LG_CUDA(cudaMemcpyAsync(fd.get(), f, sizeof(double) * n, cudaMemcpyDefault, s));
    fp = fd.get();
  }
  if (!xdev) {
    xd.alloc(n, s);
    xp = xd.get();
  }
  lg::vcycle_apply(h, *h.ws, fp, xp, precision, s);
  if (!xdev) LG_CUDA(cudaMemcpyAsync(x, xp, sizeof(double) * n, cudaMemcpyDefault, s));
  LG_CUDA(cudaStreamSynchronize(s));
  return LG_OK;
  LG_API_END
}

int lg_level_apply(lg_handle hh, int32_t level, int32_t precision, const void* x, void* y) {
  if (!hh || !x || !y || (precision != LG_FP64 && precision != LG_FP32_HIER)) return LG_ERR_INVALID;
  lg::Hier& h = *H(hh);
  if (level < 0 || level >= (int)h.levels.size() || h.levels[level]->kind == LG_LEVEL_COARSEST) return LG_ERR_INVALID;
  const lg::Level& Lv = *h.levels[level];
  if (Lv.nnz > 0 && !Lv.wconst_on && (precision == LG_FP32_HIER ? !Lv.w32.get() : !Lv.w.get()))
    return LG_ERR_INVALID;
  if (h.fp32_only && level > 0 && h.levels[level]->kind == LG_LEVEL_ELIM) return LG_ERR_INVALID;  // rows released
  LG_API_BEGIN
  lg::NvtxRange range("lg_level_apply");
  lg::level_apply(h, level, precision, x, y, h.stream);
  LG_CUDA(cudaStreamSynchronize(h.stream));
  return LG_OK;
  LG_API_END
}

uint64_t lg_kernel_launches(void) { return lg::g_launches.load(); }

int lg_profile(lg_handle hh, int32_t enable) {
  if (!hh) return LG_ERR_INVALID;
  lg::Hier& h = *H(hh);
  if (!h.ws) return LG_ERR_INVALID;
  LG_API_BEGIN
  LG_CUDA(cudaStreamSynchronize(h.stream));
  h.ws->prof.collect();
  h.ws->prof.stats.clear();
  h.ws->prof.on = enable != 0;
  return LG_OK;
  LG_API_END
}

int lg_level_lp_nnz(lg_handle hh, int32_t l, int64_t* nnz) {
  if (!hh || !nnz) return LG_ERR_INVALID;
  lg::Hier& h = *H(hh);
  if (l < 0 || l >= (int32_t)h.levels.size()) return LG_ERR_INVALID;
  *nnz = h.levels[l]->lp_nnz;
  return LG_OK;
}

int lg_batch_plan(lg_handle hh, int32_t l, int64_t out[4]) {
  if (!hh || !out) return LG_ERR_INVALID;
  const lg::Hier& h = *H(hh);
  if (l < 0 || l >= (int32_t)h.levels.size()) return LG_ERR_INVALID;
  if (!lg::batch_plan_info(h, l, out)) {
    lg::g_last_error = "lg_batch_plan: no multi-column plans yet (they are built by the first multi-column solve)";
    return LG_ERR_INVALID;
  }
  return LG_OK;
}

int lg_level_plan(lg_handle hh, int32_t l, int64_t out[8]) {
  if (!hh || !out) return LG_ERR_INVALID;
  lg::Hier& h = *H(hh);
  if (l < 0 || l >= (int32_t)h.levels.size()) return LG_ERR_INVALID;
  const lg::RowPlan& p = h.levels[l]->plan.plan;
  out[0] = p.E;
  out[1] = p.cls_off[lg::kClasses - 1] - p.cls_off[0];  // rows served by groups of 1..16 lanes
  out[2] = p.cls_off[lg::kClasses] - p.cls_off[lg::kClasses - 1];  // rows served by a warp
  out[3] = p.nlong;
  out[4] = p.nchunks;
  out[5] = p.grid();
  out[6] = p.nseg_tiles;
  out[7] = h.levels[l]->wconst_on ? 1 : 0;
  return LG_OK;
}

int lg_profile_read(lg_handle hh, int32_t level, lg_kernel_profile* out) {
  if (!hh || !out) return LG_ERR_INVALID;
  LG_API_BEGIN
  lg::Hier& h = *H(hh);
  if (level < -1 || level >= 2 * (int32_t)h.levels.size()) return LG_ERR_INVALID;
  LG_CUDA(cudaStreamSynchronize(h.stream));
  lg::Prof& p = h.ws->prof;
  p.collect();
  std::memset(out, 0, sizeof(*out));
  for (size_t l = 0; l < p.stats.size(); ++l) {
    if (level >= 0 && (int32_t)l != level) continue;
    out->total_ms += p.stats[l].ms;
    out->bytes += p.stats[l].bytes;
    out->launches += p.stats[l].launches;
  }
  return LG_OK;
  LG_API_END
}

int lg_vcycle_batch(lg_handle hh, int32_t k, const double* F, int64_t ldf, double* X, int64_t ldx,
                    int32_t precision) {
  if (!hh || !F || !X || k < 1 || k > lg::kMaxCols || (precision != LG_FP64 && precision != LG_FP32_HIER))
    return LG_ERR_INVALID;
  lg::Hier& h = *H(hh);
  if (precision == LG_FP64 && h.fp32_only) return LG_ERR_INVALID;
  const int64_t n = h.levels[0]->n;
  if (ldf < n || ldx < n) return LG_ERR_INVALID;
  LG_API_BEGIN
  cudaStream_t s = h.stream;
  int kp = 2;
  while (kp < k) kp <<= 1;  // multi-column vectors are [n][k rounded up to a power of two]
  if (!h.wsb || h.wsb->k < kp) {
    h.wsb.reset();
    h.wsb = lg::make_workspace(h, kp, s);
  }
  lg::DBuf<double> Fd((size_t)n * k, s), Xd((size_t)n * k, s);
  for (int c = 0; c < k; ++c)
    LG_CUDA(cudaMemcpyAsync(Fd.get() + (size_t)c * n, F + (size_t)c * ldf, sizeof(double) * n, cudaMemcpyDefault, s));
  lg::vcycle_apply_batch(h, *h.wsb, k, Fd.get(), Xd.get(), precision, s);
  for (int c = 0; c < k; ++c)
    LG_CUDA(cudaMemcpyAsync(X + (size_t)c * ldx, Xd.get() + (size_t)c * n, sizeof(double) * n, cudaMemcpyDefault, s));
  LG_CUDA(cudaStreamSynchronize(s));
  return LG_OK;
  LG_API_END
}

int lg_laplacian_apply(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w, const double* x,
                       double* y, void* stream) {
  if (n < 1 || !rowptr || !col || !w || !x || !y) return LG_ERR_INVALID;
  LG_API_BEGIN
  lg::run_laplacian_apply(n, rowptr, col, w, x, y, (cudaStream_t)stream);
  return LG_OK;
  LG_API_END
}

int lg_elim_select(int64_t n, const int64_t* rowptr, const int32_t* col, int32_t max_degree, uint64_t seed,
                   uint8_t* is_f, int64_t* nf, void* stream) {
  if (n < 1 || !rowptr || !col || !is_f || max_degree < 0) return LG_ERR_INVALID;
  LG_API_BEGIN
  int64_t c = lg::run_elim_select(n, rowptr, col, max_degree, seed, is_f, (cudaStream_t)stream);
  if (nf) *nf = c;
  return LG_OK;
  LG_API_END
}

int lg_strength(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w, uint64_t seed, int32_t level,
                int32_t m, int32_t sweeps, double omega, double* S, void* stream) {
  if (n < 1 || !rowptr || !col || !w || !S || m < 1 || m > 8 || sweeps < 0) return LG_ERR_INVALID;
  LG_API_BEGIN
  lg::run_strength(n, rowptr, col, w, seed, level, m, sweeps, omega, S, (cudaStream_t)stream);
  return LG_OK;
  LG_API_END
}

int lg_aggregate(int64_t n, const int64_t* rowptr, const int32_t* col, const double* S, int32_t iters,
                 int32_t threshold, int32_t* agg, int64_t* nc, int8_t* state, int32_t* votes, void* stream) {
  if (n < 1 || !rowptr || !col || !S || !agg || iters < 0) return LG_ERR_INVALID;
  LG_API_BEGIN
  int64_t c = lg::run_aggregate(n, rowptr, col, S, iters, threshold, agg, state, votes, (cudaStream_t)stream);
  if (nc) *nc = c;
  return LG_OK;
  LG_API_END
}

}  // extern "C"
