// Save and load of a hierarchy (lg_save, lg_load): every level's arrays, the
// row-binning choice of each of its row plans, the Chebyshev constants, the
// vertex order and the setup options, in one flat binary file. A loaded
// hierarchy rebuilds its row plans with the saved binning, so every pass sums
// in the same order as on the saved one and solves return the same bits; the
// setup itself (elimination, strength, aggregation, Galerkin products,
// eigenvalue estimates, pseudo-inverse) does not run again.
//
// Layout: a header (magic, format version, sizeof(lg_options), the options,
// level count, n_0, nnz(L_0), setup time, first aggregation level), the
// vertex order, then per level its sizes and kind, whether its weights are
// one constant (and the constant; the weight arrays are then empty), its
// arrays (each a count
// followed by the values, counts checked against the sizes on load), its
// plans' binning and its Chebyshev constants. Host byte order; a file is
// meant to be read back on the machine (or the same architecture) that wrote
// it.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <vector>

#include "lg_hier.h"

namespace lg {

namespace {

constexpr char kMagic[8] = {'L', 'G', 'H', 'I', 'E', 'R', 'F', '1'};
constexpr uint32_t kVersion = 2;
constexpr size_t kStageBytes = size_t(64) << 20;  // host staging of one array at a time

struct File {
  FILE* f = nullptr;
  ~File() {
    if (f) std::fclose(f);
  }
};

struct Writer {
  FILE* f;
  void raw(const void* p, size_t bytes) {
    if (bytes && std::fwrite(p, 1, bytes, f) != bytes) fail(LG_ERR_INVALID, "hierarchy file: write failed");
  }
  template <typename T>
  void val(const T& v) {
    raw(&v, sizeof(T));
  }
  // count values of a device array, through a bounded host buffer
  template <typename T>
  void arr(const DBuf<T>& b, size_t count, cudaStream_t s) {
    val<uint64_t>(count);
    const size_t step = kStageBytes / sizeof(T);
    std::vector<T> h(count < step ? count : step);
    for (size_t at = 0; at < count; at += step) {
      const size_t m = count - at < step ? count - at : step;
      LG_CUDA(cudaMemcpyAsync(h.data(), b.get() + at, sizeof(T) * m, cudaMemcpyDeviceToHost, s));
      LG_CUDA(cudaStreamSynchronize(s));
      raw(h.data(), sizeof(T) * m);
    }
  }
};

struct Reader {
  FILE* f;
  void raw(void* p, size_t bytes) {
    if (bytes && std::fread(p, 1, bytes, f) != bytes) fail(LG_ERR_INVALID, "hierarchy file: truncated");
  }
  template <typename T>
  T val() {
    T v;
    raw(&v, sizeof(T));
    return v;
  }
  // a device array of exactly `expect` values (an empty one for 0), through
  // a bounded host buffer
  template <typename T>
  void arr(DBuf<T>& b, int64_t expect, cudaStream_t s, int64_t* counter) {
    const uint64_t count = val<uint64_t>();
    if (expect < 0 || count != (uint64_t)expect) fail(LG_ERR_INVALID, "hierarchy file: array size mismatch");
    if (!count) return;
    b.alloc(count, s, counter);
    const size_t step = kStageBytes / sizeof(T);
    std::vector<T> h(count < step ? count : step);
    for (size_t at = 0; at < count; at += step) {
      const size_t m = count - at < step ? count - at : step;
      raw(h.data(), sizeof(T) * m);
      LG_CUDA(cudaMemcpyAsync(b.get() + at, h.data(), sizeof(T) * m, cudaMemcpyHostToDevice, s));
      LG_CUDA(cudaStreamSynchronize(s));  // h is refilled next
    }
  }
};

// Range checks of what a file gives: a damaged or hostile file must be
// refused before any kernel indexes with its arrays. The checks compare
// values only (each thread reads its own element and the next pointer), so
// they cannot themselves reach outside the arrays.
#define LG_IO_STRIDE(i, n) \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

__global__ void k_io_check_ptr(int64_t rows, int64_t total, const int64_t* __restrict__ p, int* bad) {
  LG_IO_STRIDE(i, rows + 1) {
    const int64_t v = p[i];
    if (v < 0 || v > total || (i == 0 && v != 0) || (i == rows && v != total) || (i < rows && p[i + 1] < v))
      atomicOr(bad, 1);
  }
}

__global__ void k_io_check_range(int64_t count, const int32_t* __restrict__ a, int64_t lo, int64_t hi, int* bad) {
  LG_IO_STRIDE(i, count) {
    const int64_t v = a[i];
    if (v < lo || v >= hi) atomicOr(bad, 1);
  }
}

struct Checker {
  cudaStream_t s;
  DBuf<int> bad;
  explicit Checker(cudaStream_t st) : s(st), bad(1, st) {
    LG_CUDA(cudaMemsetAsync(bad.get(), 0, sizeof(int), s));
  }
  // rowptr of `rows` rows: 0 first, `total` last, non-decreasing
  void ptr(const DBuf<int64_t>& p, int64_t rows, int64_t total) {
    k_io_check_ptr<<<grid_for(rows + 1, 256, kSMs * 8), 256, 0, s>>>(rows, total, p.get(), bad.get());
    LG_LAUNCH_CHECK();
  }
  // every value in [lo, hi)
  void range(const DBuf<int32_t>& a, int64_t count, int64_t lo, int64_t hi) {
    if (count <= 0) return;
    k_io_check_range<<<grid_for(count, 256, kSMs * 8), 256, 0, s>>>(count, a.get(), lo, hi, bad.get());
    LG_LAUNCH_CHECK();
  }
  // fails with LG_ERR_INVALID if any check so far found a bad value
  void require(const char* what) {
    int v = 0;
    LG_CUDA(cudaMemcpyAsync(&v, bad.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    LG_CUDA(cudaStreamSynchronize(s));
    if (v) fail(LG_ERR_INVALID, what);
  }
};

// A plan over (rows, entries, rowptr) binned with E entries per lane, as the
// setup built it (build_row_plan bins with E = 4, the tuner may re-bin).
void plan_with(RowPlanStore& ps, int64_t rows, int64_t entries, const int64_t* rowptr, int E, cudaStream_t s,
               int64_t* counter, int64_t ncols = 0) {
  if (E != 2 && E != 4 && E != 8) fail(LG_ERR_INVALID, "hierarchy file: row binning");
  build_row_plan(ps, rows, entries, rowptr, s, counter, ncols);
  if (E != ps.plan.E) bin_rows(ps, rows, rowptr, E, s);
}

}  // namespace

void save_hierarchy(const Hier& h, const char* path) {
  cudaStream_t s = h.stream;
  File file;
  file.f = std::fopen(path, "wb");
  if (!file.f) fail(LG_ERR_INVALID, "hierarchy file: cannot open for writing");
  Writer w{file.f};
  w.raw(kMagic, sizeof(kMagic));
  w.val<uint32_t>(kVersion);
  w.val<uint32_t>((uint32_t)sizeof(lg_options));
  w.val(h.opts);
  const int32_t nl = (int32_t)h.levels.size();
  const int64_t n0 = h.levels[0]->n;
  w.val(nl);
  w.val(n0);
  w.val(h.nnz0);
  w.val(h.setup_ms);
  w.val<int32_t>(h.first_agg);
  w.arr(h.perm, (size_t)n0, s);
  for (int32_t l = 0; l < nl; ++l) {
    const Level& L = *h.levels[l];
    w.val<int32_t>(L.kind);
    w.val(L.n);
    w.val(L.nnz);
    w.val(L.nc);
    w.val(L.nf);
    w.val(L.lambda);
    w.val<int32_t>(L.plan.plan.E);
    w.val<int32_t>(L.wconst_on ? 1 : 0);
    w.val(L.wconst);
    w.arr(L.rowptr, (size_t)L.n + 1, s);
    w.arr(L.col, (size_t)L.nnz, s);
    w.arr(L.w, L.wconst_on ? 0 : (size_t)L.nnz, s);
    w.arr(L.d, L.d.size(), s);
    w.arr(L.dinv, L.dinv.size(), s);
    w.arr(L.w32, L.w32.size(), s);
    w.arr(L.dinv32, L.dinv32.size(), s);
    if (L.kind == LG_LEVEL_AGG) {
      w.arr(L.agg, (size_t)L.n, s);
      w.arr(L.mem_ptr, (size_t)L.nc + 1, s);
      w.arr(L.mem, (size_t)L.n, s);
      w.val<int32_t>(L.mem_plan.plan.E);
      const int64_t lpn = L.lp_nnz;
      w.val(lpn);
      if (lpn > 0) {
        w.arr(L.lp_ptr, (size_t)L.n + 1, s);
        w.arr(L.lp_col, (size_t)lpn, s);
        w.arr(L.lp_w, (size_t)lpn, s);
        w.arr(L.lp_w32, (size_t)lpn, s);
        w.arr(L.lp_d, (size_t)L.n, s);
        w.val<int32_t>(L.lp_plan.plan.E);
      }
    } else if (L.kind == LG_LEVEL_ELIM) {
      const int64_t npt = L.pt_f.size();
      w.arr(L.cmap, (size_t)L.n, s);
      w.arr(L.cfine, (size_t)L.nc, s);
      w.arr(L.pt_ptr, (size_t)L.nc + 1, s);
      w.val(npt);
      w.arr(L.pt_f, (size_t)npt, s);
      w.arr(L.pt_coef, (size_t)npt, s);
      w.arr(L.pt_coef32, L.pt_coef32.size(), s);
      w.val<int32_t>(L.pt_plan.plan.E);
    } else {
      w.arr(L.pinv, (size_t)L.n * (size_t)L.n, s);
    }
    w.val(h.cheb[l]);
  }
  if (std::fflush(file.f) != 0) fail(LG_ERR_INVALID, "hierarchy file: write failed");
}

void load_hierarchy(Hier& h, const char* path, const lg_options* call_opts) {
  File file;
  file.f = std::fopen(path, "rb");
  if (!file.f) fail(LG_ERR_INVALID, "hierarchy file: cannot open");
  Reader r{file.f};
  char magic[sizeof(kMagic)];
  r.raw(magic, sizeof(magic));
  if (std::memcmp(magic, kMagic, sizeof(kMagic)) != 0) fail(LG_ERR_INVALID, "hierarchy file: not a hierarchy");
  if (r.val<uint32_t>() != kVersion) fail(LG_ERR_INVALID, "hierarchy file: format version");
  if (r.val<uint32_t>() != (uint32_t)sizeof(lg_options)) fail(LG_ERR_INVALID, "hierarchy file: options layout");
  const lg_options saved = r.val<lg_options>();
  const int32_t nl = r.val<int32_t>();
  const int64_t n0 = r.val<int64_t>();
  const int64_t nnz0 = r.val<int64_t>();
  const double setup_ms = r.val<double>();
  const int32_t first_agg = r.val<int32_t>();
  if (nl < 1 || nl > 1024 || n0 < 1 || n0 >= (int64_t(1) << 31) || nnz0 < n0 || first_agg < -1 || first_agg >= nl)
    fail(LG_ERR_INVALID, "hierarchy file: header");
  // everything above is checked before the first CUDA call
  h.opts = saved;
  h.opts.stream = call_opts ? call_opts->stream : nullptr;
  h.opts.memory_space = call_opts ? call_opts->memory_space : LG_AUTO;
  LG_CUDA(cudaGetDevice(&h.device));
  if (h.opts.stream) {
    h.stream = (cudaStream_t)h.opts.stream;
  } else {
    LG_CUDA(cudaStreamCreateWithFlags(&h.stream, cudaStreamNonBlocking));
    h.own_stream = true;
  }
  cudaStream_t s = h.stream;
  int64_t* counter = &h.bytes;
  h.nnz0 = nnz0;
  h.setup_ms = setup_ms;
  h.first_agg = first_agg;
  h.dev_err.alloc(1, s);
  LG_CUDA(cudaMemsetAsync(h.dev_err.get(), 0, sizeof(int), s));
  r.arr(h.perm, n0, s, counter);
  Checker check(s);
  check.range(h.perm, n0, 0, n0);
  check.require("hierarchy file: vertex order out of range");
  h.cheb.assign((size_t)nl, Cheb{});
  int64_t expect_n = n0;
  for (int32_t l = 0; l < nl; ++l) {
    auto L = std::make_unique<Level>();
    L->kind = r.val<int32_t>();
    L->n = r.val<int64_t>();
    L->nnz = r.val<int64_t>();
    L->nc = r.val<int64_t>();
    L->nf = r.val<int64_t>();
    L->lambda = r.val<double>();
    const int E = r.val<int32_t>();
    const int32_t wconst_on = r.val<int32_t>();
    const double wconst = r.val<double>();
    const bool last = l == nl - 1;
    if (L->n != expect_n || L->nnz < 0 || L->nnz > L->n * (L->n - 1) ||
        (last != (L->kind == LG_LEVEL_COARSEST)) ||
        (L->kind != LG_LEVEL_AGG && L->kind != LG_LEVEL_ELIM && L->kind != LG_LEVEL_COARSEST) ||
        (!last && (L->nc < 1 || L->nc > L->n)))
      fail(LG_ERR_INVALID, "hierarchy file: level sizes");
    if (wconst_on != 0 && (wconst_on != 1 || l != 0 || !(wconst > 0.0) || !std::isfinite(wconst)))
      fail(LG_ERR_INVALID, "hierarchy file: constant weight");
    L->wconst_on = wconst_on == 1;
    L->wconst = L->wconst_on ? wconst : 0.0;
    const int64_t nw = L->wconst_on ? 0 : L->nnz;
    r.arr(L->rowptr, L->n + 1, s, counter);
    r.arr(L->col, L->nnz, s, counter);
    r.arr(L->w, nw, s, counter);
    r.arr(L->d, L->n, s, counter);
    r.arr(L->dinv, L->n, s, counter);
    r.arr(L->w32, nw, s, counter);
    r.arr(L->dinv32, L->n, s, counter);
    check.ptr(L->rowptr, L->n, L->nnz);
    check.range(L->col, L->nnz, 0, L->n);
    check.require("hierarchy file: operator row pointer or column out of range");
    plan_with(L->plan, L->n, L->nnz, L->rowptr.get(), E, s, counter, L->n);
    if (L->kind == LG_LEVEL_AGG) {
      r.arr(L->agg, L->n, s, counter);
      r.arr(L->mem_ptr, L->nc + 1, s, counter);
      r.arr(L->mem, L->n, s, counter);
      check.range(L->agg, L->n, 0, L->nc);
      check.ptr(L->mem_ptr, L->nc, L->n);
      check.range(L->mem, L->n, 0, L->n);
      check.require("hierarchy file: aggregates or member lists out of range");
      plan_with(L->mem_plan, L->nc, L->n, L->mem_ptr.get(), r.val<int32_t>(), s, counter);
      const int64_t lpn = r.val<int64_t>();
      if (lpn < 0 || lpn > L->nnz) fail(LG_ERR_INVALID, "hierarchy file: W size");
      if (lpn > 0) {
        L->lp_nnz = lpn;
        r.arr(L->lp_ptr, L->n + 1, s, counter);
        r.arr(L->lp_col, lpn, s, counter);
        r.arr(L->lp_w, lpn, s, counter);
        r.arr(L->lp_w32, lpn, s, counter);
        r.arr(L->lp_d, L->n, s, counter);
        check.ptr(L->lp_ptr, L->n, lpn);
        check.range(L->lp_col, lpn, 0, L->nc);
        check.require("hierarchy file: W row pointer or aggregate id out of range");
        plan_with(L->lp_plan, L->n, lpn, L->lp_ptr.get(), r.val<int32_t>(), s, counter, L->nc);
      }
    } else if (L->kind == LG_LEVEL_ELIM) {
      r.arr(L->cmap, L->n, s, counter);
      r.arr(L->cfine, L->nc, s, counter);
      r.arr(L->pt_ptr, L->nc + 1, s, counter);
      const int64_t npt = r.val<int64_t>();
      if (npt < 0 || npt > L->nnz) fail(LG_ERR_INVALID, "hierarchy file: elimination rows");
      r.arr(L->pt_f, npt, s, counter);
      r.arr(L->pt_coef, npt, s, counter);
      r.arr(L->pt_coef32, npt, s, counter);
      check.range(L->cmap, L->n, -1, L->nc);
      check.range(L->cfine, L->nc, 0, L->n);
      check.ptr(L->pt_ptr, L->nc, npt);
      check.range(L->pt_f, npt, 0, L->n);
      check.require("hierarchy file: elimination maps out of range");
      plan_with(L->pt_plan, L->nc, npt, L->pt_ptr.get(), r.val<int32_t>(), s, counter);
    } else {
      if (L->n > h.opts.max_coarse_n && L->n > 4096) fail(LG_ERR_INVALID, "hierarchy file: coarsest size");
      r.arr(L->pinv, L->n * L->n, s, counter);
    }
    h.cheb[l] = r.val<Cheb>();
    expect_n = L->nc;
    h.levels.push_back(std::move(L));
  }
  char extra;
  if (std::fread(&extra, 1, 1, file.f) != 0) fail(LG_ERR_INVALID, "hierarchy file: trailing bytes");
  h.ws = make_workspace(h, 1, h.stream);
  LG_CUDA(cudaStreamSynchronize(h.stream));
}

}  // namespace lg
