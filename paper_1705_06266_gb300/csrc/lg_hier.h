// The multigrid hierarchy as it lives in device memory, and the host-side
// entry points of setup, cycle and PCG.
//
// Level layout (all device arrays, one hierarchy = one set of allocations):
//  - operator L_l: CSR of the off-diagonal weights (rowptr int64, col int32,
//    w double + float copy) and 1/diag (double + float). The diagonal is the
//    row sum of w (Section 2.1), so L 1 = 0 holds in the difference form.
//  - AGG level: agg[n] (vertex -> aggregate) and the member CSR of R
//    (mem_ptr[nc+1], mem[n], members in ascending vertex order) for a
//    deterministic restriction r_c = R r; with lp_residual also W = L P off
//    the own aggregate (lp_ptr[n+1], lp_col = aggregate ids, lp_w, and the
//    row sums lp_d), so that (L P x_c)_i = sum_a W_ia (x_c[agg_i] - x_c[a]).
//  - ELIM level: cmap[n] (kept vertex -> coarse id, eliminated -> -1),
//    cfine[nc] (coarse id -> kept vertex) and the transpose of the
//    elimination prolongation's F rows per kept vertex (pt_ptr, pt_f,
//    pt_coef = w_cf / d_f), for (P^T f)_c = f_c + sum_f pt_coef f_f.
//  - COARSEST: the dense FP64 pseudo-inverse, n x n row-major.
#pragma once

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "lg_prims.h"

namespace lg {

// A named NVTX range for the life of the object: the phases of a setup or a
// solve on a profiler's timeline (nothing happens without a profiler).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

template <typename T>
struct OpView {
  int64_t n = 0, nnz = 0;
  const int64_t* rowptr = nullptr;
  const int32_t* col = nullptr;
  const T* w = nullptr;
  const T* dinv = nullptr;
  const double* d = nullptr;  // FP64 row sums (used by the FP64 passes)
  RowPlan plan;
  T wc = T(0);                // every weight, when w is null (a constant-weight operator)
};

struct Level {
  int kind = 0;
  int64_t n = 0, nnz = 0, nc = 0;
  DBuf<int64_t> rowptr;
  DBuf<int32_t> col;
  DBuf<double> w, d, dinv;
  DBuf<float> w32, dinv32;
  RowPlanStore plan;
  double lambda = 0.0;
  // A finest operator whose weights are all equal (an unweighted graph) keeps
  // that value instead of its weight arrays (w and w32 released after setup).
  bool wconst_on = false;
  double wconst = 0.0;
  // aggregation
  DBuf<int32_t> agg, mem;
  DBuf<int64_t> mem_ptr;
  RowPlanStore mem_plan;
  int64_t lp_nnz = 0;  // W = L P (0: not built)
  DBuf<int64_t> lp_ptr;
  DBuf<int32_t> lp_col;
  DBuf<double> lp_w, lp_d;
  DBuf<float> lp_w32;
  RowPlanStore lp_plan;
  // elimination
  int64_t nf = 0;
  DBuf<int32_t> cmap, cfine, pt_f;
  DBuf<int64_t> pt_ptr;
  DBuf<double> pt_coef;
  DBuf<float> pt_coef32;
  RowPlanStore pt_plan;
  // coarsest
  DBuf<double> pinv;

  template <typename T> OpView<T> op() const;
  template <typename T> OpView<T> lp() const;
};

template <> inline OpView<double> Level::op<double>() const {
  return OpView<double>{n, nnz, rowptr.get(), col.get(), w.get(), dinv.get(), d.get(), plan.plan, wconst};
}
template <> inline OpView<float> Level::op<float>() const {
  return OpView<float>{n, nnz, rowptr.get(), col.get(), w32.get(), dinv32.get(), d.get(), plan.plan, (float)wconst};
}
// W = L P as an operator view: its rows' entries, and lp_d in place of d.
template <> inline OpView<double> Level::lp<double>() const {
  return OpView<double>{n, lp_nnz, lp_ptr.get(), lp_col.get(), lp_w.get(), dinv.get(), lp_d.get(), lp_plan.plan};
}
template <> inline OpView<float> Level::lp<float>() const {
  return OpView<float>{n, lp_nnz, lp_ptr.get(), lp_col.get(), lp_w32.get(), dinv32.get(), lp_d.get(), lp_plan.plan};
}

// Chebyshev constants of one aggregation level (Section 3.6): the interval
// [lo, hi] * lambda, theta / delta its centre / half-width, and for step s
// (1-based) c1[s] = rho_s rho_{s-1}, c2[s] = 2 rho_s / delta.
struct Cheb {
  double inv_theta = 0.0;
  double c1[8] = {0}, c2[8] = {0};
};

// Per-level vectors of a solve workspace, for one precision and k columns.
template <typename T>
struct LevelVecs {
  DBuf<T> f, x, r, dA, dB;
  DBuf<T> kc1, kv1, kv2;  // K-cycle levels: the first FCG direction, L c1, L c2
};

// K-cycle scalars of one level (ws.kscal, kKScal per level).
enum KScal : int { kRho1 = 0, kA1, kT1, kOk1, kG, kB2, kA2, kU1, kU2, kKScal = 10 };

// Long-row scratch (chunk partials, per-row tickets) of one row plan, owned by
// a workspace so that concurrent solves on one hierarchy never share it.
struct PlanScratch {
  DBuf<double> partial;
  DBuf<unsigned> ticket;
  void make(const RowPlan& p, int k, cudaStream_t s, int64_t* counter) {
    partial.alloc((size_t)(p.nchunks > 0 ? p.nchunks : 1) * k, s, counter);
    ticket.alloc(p.nlong > 0 ? p.nlong : 1, s, counter);
    check_cuda(cudaMemsetAsync(ticket.get(), 0, sizeof(unsigned) * (p.nlong > 0 ? p.nlong : 1), s), "memset");
  }
  RowPlan bind(RowPlan p) const {
    p.partial = partial.get();
    p.ticket = ticket.get();
    return p;
  }
};

struct LevelScratch {
  PlanScratch op, mem, pt, lp;
};

struct Hier;

// Event timing of the operator passes (Laplacian row passes) of one
// workspace, per level.
struct Prof {
  struct Stat {
    double ms = 0.0, bytes = 0.0;
    int64_t launches = 0;
  };
  struct Pending {
    int level;
    double bytes;
  };
  bool on = false;
  std::vector<cudaEvent_t> ev;  // pairs
  std::vector<Pending> pending;
  std::vector<Stat> stats;      // indexed by level
  void begin(cudaStream_t s);
  void end(cudaStream_t s, int level, double bytes);
  void collect();  // after the stream has been synchronised
  ~Prof();
};

// Workspace of one concurrent solve: per-level cycle vectors in both
// precisions, the FP64 Krylov vectors, reduction scratch and device scalars.
struct Workspace {
  int k = 1;
  cudaStream_t alloc_stream = nullptr;  // the stream its memory is allocated and freed on
  std::vector<LevelVecs<double>> v64;
  std::vector<LevelVecs<float>> v32;
  std::vector<LevelScratch> scratch;
  DBuf<double> bm, x, r, ro, z, p, q;   // FP64 Krylov vectors, n * k (level-0 numbering)
  DBuf<double> io;                     // input / output in the caller's numbering
  DBuf<double> partials;               // grid reduction partials
  DBuf<unsigned> tickets;              // grid reduction tickets (zero between launches)
  DBuf<double> scal;                   // device scalars of the PCG (see lg_cycle.cu)
  DBuf<double> kscal;                  // K-cycle scalars, kKScal per level
  double* host_scal = nullptr;         // pinned mirror of the scalars read by the host
  int64_t bytes = 0;
  Prof prof;
  std::shared_ptr<void> batch;          // SpMM plans of multi-column solves (lg_batch.cu)
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // captured preconditioned iteration per precision
  ~Workspace();
};

// Device time of the setup's stages, for the solve log: events recorded on
// the setup stream at stage boundaries (only while `on`), each interval
// charged to the stage named by its closing mark and summed over levels.
struct StageClock {
  bool on = false;
  cudaStream_t s = nullptr;
  std::vector<std::pair<const char*, cudaEvent_t>> marks;
  void mark(const char* name) {
    if (!on) return;
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess || cudaEventRecord(e, s) != cudaSuccess) {
      cudaGetLastError();
      if (e) cudaEventDestroy(e);
      return;
    }
    marks.emplace_back(name, e);
  }
  // after the stream has been synchronised: (stage, ms) in first-seen order
  std::vector<std::pair<std::string, double>> collect() {
    std::vector<std::pair<std::string, double>> out;
    for (size_t i = 1; i < marks.size(); ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, marks[i - 1].second, marks[i].second) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      auto it = std::find_if(out.begin(), out.end(), [&](const auto& p) { return p.first == marks[i].first; });
      if (it == out.end()) out.emplace_back(marks[i].first, (double)ms);
      else it->second += ms;
    }
    return out;
  }
  ~StageClock() {
    for (auto& m : marks) cudaEventDestroy(m.second);
  }
};

struct Hier {
  lg_options opts;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  int64_t bytes = 0;
  int64_t nnz0 = 0;
  double setup_ms = 0.0;
  std::vector<std::unique_ptr<Level>> levels;
  std::vector<Cheb> cheb;               // per level (aggregation levels only)
  std::unique_ptr<Workspace> ws;        // default workspace of lg_solve
  std::unique_ptr<Workspace> wsb;       // workspace of lg_solve_batch (widest batch so far)
  DBuf<int> dev_err;                    // device error word
  DBuf<int32_t> perm;                   // level-0 vertex i is the caller's vertex perm[i]
  int first_agg = -1;                   // first aggregation level (-1: none)
  std::shared_ptr<void> many;           // device views of the levels for lg_solve_many (lg_many.cu)
  std::shared_ptr<void> mplans;         // SpMM plans of multi-column solves, read by every workspace (lg_batch.cu);
                                        // released before the handle's stream, with the workspaces' own state
  bool fp32_only = false;               // FP64 copies released (option fp32_only): FP32 solves only
  bool time_stages = false;             // record setup_stages (set before the setup)
  std::vector<std::pair<std::string, double>> setup_stages;  // device ms per setup stage
  ~Hier();
};

// ---- setup (lg_setup.cu) ----
void setup_hierarchy(Hier& h, int64_t n, const int64_t* rowptr, const int32_t* col, const double* w);

// step kernels usable on caller data
void run_laplacian_apply(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w,
                         const double* x, double* y, cudaStream_t s);
int64_t run_elim_select(int64_t n, const int64_t* rowptr, const int32_t* col, int max_degree,
                        uint64_t seed, uint8_t* is_f, cudaStream_t s);
// bins / dinv: the level's own (setup), or null to derive them from the CSR.
void run_strength(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w, uint64_t seed,
                  int level, int m, int sweeps, double omega, double* S, cudaStream_t s,
                  const RowBins* bins = nullptr, const double* dinv = nullptr);
int64_t run_aggregate(int64_t n, const int64_t* rowptr, const int32_t* col, const double* S, int iters,
                      int threshold, int32_t* agg, int8_t* state, int32_t* votes, cudaStream_t s,
                      const RowBins* bins = nullptr);

// ---- solve (lg_cycle.cu) ----
std::unique_ptr<Workspace> make_workspace(Hier& h, int k, cudaStream_t s);
// y = L_l x on level l with the cycle's row plan (T = double for LG_FP64,
// float for LG_FP32_HIER; device vectors in the level's numbering).
void level_apply(Hier& h, int l, int precision, const void* x, void* y, cudaStream_t s);
// x = M f on the device (FP64 in and out), starting from x = 0.
void vcycle_apply(Hier& h, Workspace& ws, const double* f, double* x, int precision, cudaStream_t s);
// PCG on device vectors b, x (n doubles each, column c of a k-wide block
// uses stride-1 columns of length n). Fills info.
int pcg_solve(Hier& h, Workspace& ws, const double* b, double* x, double tol, int precision,
              cudaStream_t s, lg_info* info);
void vcycle_apply_batch(Hier& h, Workspace& ws, int k, const double* F, double* X, int precision, cudaStream_t s);
// Work of one PCG iteration in finest-residual units (lg_info.work_units / iterations).
double iteration_work(const Hier& h);
int pcg_solve_batch(Hier& h, Workspace& ws, int k, const double* B, double* X, double tol, int precision,
                    cudaStream_t s, lg_info* infos);
// Build (and tune, timing passes at width kp) the multi-column plans of h now
// rather than at its first multi-column solve.
void prepare_columns(Hier& h, int kp, int precision);
// Level l's multi-column schedule (stretch length and virtual rows of its
// operator and W plans); false until the plans are built.
bool batch_plan_info(const Hier& h, int level, int64_t out[4]);
// Capture ws's multi-column solve loops (every width up to ws.k) on stream s
// now rather than at their first solves.
void prepare_column_graphs(Hier& h, Workspace& ws, int precision, cudaStream_t s);
// The multi-column path for every k (k = 1 included), whose per-column
// results do not depend on the batch (the server's solves).
int pcg_solve_columns(Hier& h, Workspace& ws, int k, const double* B, double* X, double tol, int precision,
                      cudaStream_t s, lg_info* infos);

// ---- save and load (lg_io.cu) ----
void save_hierarchy(const Hier& h, const char* path);
// Fills a fresh Hier from a file written by save_hierarchy; opts (may be
// null) gives the stream and memory space. The header is checked before any
// CUDA call.
void load_hierarchy(Hier& h, const char* path, const lg_options* opts);

// ---- many small solves in one launch (lg_many.cu) ----
// Build h's device views for the packed solver now (else at its first packed solve).
void prepare_many(Hier& h);
constexpr int64_t kManyMaxNnz = int64_t(1) << 22;  // largest nnz(L_0) one block solves
constexpr int kManyMaxLevels = 64;
// hs: distinct handles on one device; b / x: each graph's vectors in the
// caller's numbering, device memory where b_dev / x_dev say so, else host.
// precision: LG_FP64 / LG_FP32_HIER for every graph, or -1 for each handle's own.
int solve_many(int count, Hier* const* hs, const double* const* b, double* const* x, const bool* b_dev,
               const bool* x_dev, double tol, lg_info* infos, int precision = -1);

}  // namespace lg
