// V-cycle and preconditioned conjugate gradients (Sections 2.3, 3.6, 4).
//
// The cycle runs in FP32 or FP64 (template T) over per-level vectors of a
// workspace; the outer CG is FP64 throughout, with the mean projection and
// the coarsest dense solve in FP64 too. Every SpMV of the cycle is one
// lg::k_rows pass whose epilogue applies the Chebyshev vector updates, so a
// degree-2 smoother costs two passes over the level's operator (the second
// pre-smoothing pass also yields the residual that is restricted).
#include <algorithm>
#include <cmath>

#include "lg_hier.h"
#include "lg_rows.cuh"

namespace lg {

constexpr int kVT = 256;

// Scalars of the FP64 PCG (device array ws.scal).
enum Scal : int {
  kBB = 0,     // ||b_m||^2
  kRZ = 1,     // r^T z (projected z)
  kPQ = 2,     // p^T L p
  kAlpha = 3,
  kBeta = 4,
  kMeanZ = 5,
  kRR = 6,     // ||r||^2
  kSumB = 7,
  kBreak = 8,  // 1 after a breakdown
  kZ0 = 9,     // 5 sums of the z reduction (9..13)
  kTmp = 14,   // 2 scratch totals (14..15)
  kIter = 16,  // iterations done
  kDone = 17,  // 1 once the true residual met the tolerance
  kTol2BB = 18,  // tol^2 ||b_m||^2
  kMaxit = 19,
  kEvery = 20,   // true-residual replacement period
  kNeedTrue = 21,  // 1 when this iteration recomputes the true residual
  kNScal = 24
};

#define LG_GRID_STRIDE(i, n) \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

static inline int vblocks(int64_t n) { return grid_for(n, kVT, kSMs * 8); }

void Prof::begin(cudaStream_t s) {
  const size_t i = pending.size();
  while (ev.size() < 2 * i + 2) {
    cudaEvent_t e;
    LG_CUDA(cudaEventCreate(&e));
    ev.push_back(e);
  }
  LG_CUDA(cudaEventRecord(ev[2 * i], s));
}

void Prof::end(cudaStream_t s, int level, double bytes) {
  const size_t i = pending.size();
  LG_CUDA(cudaEventRecord(ev[2 * i + 1], s));
  pending.push_back(Pending{level, bytes});
}

void Prof::collect() {
  for (size_t i = 0; i < pending.size(); ++i) {
    float ms = 0.f;
    LG_CUDA(cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]));
    const int l = pending[i].level;
    if ((int)stats.size() <= l) stats.resize(l + 1);
    stats[l].ms += ms;
    stats[l].bytes += pending[i].bytes;
    stats[l].launches += 1;
  }
  pending.clear();
}

Prof::~Prof() {
  for (auto e : ev) cudaEventDestroy(e);
}

// ---------------------------------------------------------------------------
// Epilogues of the cycle's row passes.
// ---------------------------------------------------------------------------

// One Chebyshev step on D^-1 L (Section 3.6), given s = (L g)_i for the
// gathered vector g = d_{s-1}:
//   r_s = r_{s-1} - L d_{s-1},  d_s = c1 d_{s-1} + c2 D^-1 r_s,
//   x  (mode 1) = d_{s-1} [+ d_s]   or  (mode 2) x += d_{s-1} [+ d_s].
// With c1 = 0 and c2 = 1/theta it is the first step d_0 = D^-1 r_0 / theta.
template <typename T>
struct EpiCheb {
  const T* g;
  const T* rin;
  T* rout;
  const T* dinv;
  T* dout;
  T* x;
  int x_mode;
  int add_d;
  T c1, c2;
  struct Pre {
    T rin, g, dinv, x;
  };
  __device__ __forceinline__ Pre pre(int64_t i) const {
    return Pre{rin[i], g[i], dout ? dinv[i] : T(0), (x && x_mode == 2) ? x[i] : T(0)};
  }
  __device__ __forceinline__ void operator()(int64_t i, T s, const Pre& p, double*) const {
    const T r = p.rin - s;
    rout[i] = r;
    T d = T(0);
    if (dout) {
      d = c1 * p.g + c2 * p.dinv * r;
      dout[i] = d;
    }
    if (x) x[i] = p.x + p.g + (add_d ? d : T(0));
  }
  __device__ void finish(const double*) const {}
};

// Aggregation restriction r_c = R r (Section 3.5); also the next level's
// first Chebyshev direction d_0 = D^-1 f_c / theta when it smooths.
template <typename T>
struct EpiRestrict {
  T* fc;
  T* d0;
  const T* dinvc;
  T inv_theta;
  __device__ __forceinline__ T pre(int64_t I) const { return d0 ? dinvc[I] : T(0); }
  __device__ __forceinline__ void operator()(int64_t I, T s, T dv, double*) const {
    fc[I] = s;
    if (d0) d0[I] = s * dv * inv_theta;
  }
  __device__ void finish(const double*) const {}
};

// Elimination restriction (P^T f)_c = f_c + sum_f (w_fc / d_f) f_f (Section 3.4).
template <typename T>
struct EpiElimRestrict {
  const T* f;
  const int32_t* cfine;
  T* fc;
  T* d0;
  const T* dinvc;
  T inv_theta;
  struct Pre {
    T f, dv;
  };
  __device__ __forceinline__ Pre pre(int64_t c) const { return Pre{f[cfine[c]], d0 ? dinvc[c] : T(0)}; }
  __device__ __forceinline__ void operator()(int64_t c, T s, const Pre& p, double*) const {
    const T v = p.f + s;
    fc[c] = v;
    if (d0) d0[c] = v * p.dv * inv_theta;
  }
  __device__ void finish(const double*) const {}
};

// (L P x_c)_i over W = L P off the own aggregate (Level::lp):
// sum_a W_ia (x_c[agg_i] - x_c[a]). FP32 in that difference form, as LapTerm;
// FP64 as d^W_i x_c[agg_i] - sum_a W_ia x_c[a], d^W the row sums of W. The
// gathered x_c is the coarse level's, short enough to stay in L1.
template <typename T>
struct LpTerm;

template <>
struct LpTerm<float> {
  const float* __restrict__ w;
  const float* __restrict__ xc;
  const int32_t* __restrict__ agg;
  __device__ __forceinline__ float row(int64_t i) const { return ld_keep(&xc[__ldg(&agg[i])]); }
  __device__ __forceinline__ float acc(float s, int64_t k, int32_t a, float xa) const {
    return fmaf(ld_stream(&w[k]), xa - ld_keep(&xc[a]), s);
  }
  __device__ __forceinline__ const float* src() const { return xc; }
  __device__ __forceinline__ float wload(int64_t k) const { return ld_stream(&w[k]); }
  __device__ __forceinline__ float accw(float s, float wk, float xj, float xa) const { return fmaf(wk, xa - xj, s); }
  __device__ __forceinline__ float finish(int64_t, float, float s) const { return s; }
};

template <>
struct LpTerm<double> {
  const double* __restrict__ w;
  const double* __restrict__ xc;
  const int32_t* __restrict__ agg;
  const double* __restrict__ d;
  __device__ __forceinline__ double row(int64_t) const { return 0.0; }
  __device__ __forceinline__ double acc(double s, int64_t k, int32_t a, double) const {
    return fma(ld_stream(&w[k]), ld_keep(&xc[a]), s);
  }
  __device__ __forceinline__ const double* src() const { return xc; }
  __device__ __forceinline__ double wload(int64_t k) const { return ld_stream(&w[k]); }
  __device__ __forceinline__ double accw(double s, double wk, double xj, double) const { return fma(wk, xj, s); }
  __device__ __forceinline__ double finish(int64_t i, double, double s) const {
    return fma(__ldg(&d[i]), ld_keep(&xc[__ldg(&agg[i])]), -s);
  }
};

template <typename T>
static LpTerm<T> lp_term(const OpView<T>& w, const T* xc, const int32_t* agg);
template <>
LpTerm<float> lp_term<float>(const OpView<float>& w, const float* xc, const int32_t* agg) {
  return LpTerm<float>{w.w, xc, agg};
}
template <>
LpTerm<double> lp_term<double>(const OpView<double>& w, const double* xc, const int32_t* agg) {
  return LpTerm<double>{w.w, xc, agg, w.d};
}

// Start of post-smoothing after the coarse correction (Section 3.6), in one
// pass over W given s = (L P x_c)_i: x += P x_c; r_0 = r_pre - s (r_pre, the
// pre-smoothing residual f - L x, is still in r); d_0 = D^-1 r_0 / theta.
template <typename T>
struct EpiPost {
  T* r;
  T* x;
  const T* xc;
  const int32_t* agg;
  const T* dinv;
  T* d0;
  T inv_theta;
  struct Pre {
    T r, x, xa, dv;
  };
  __device__ __forceinline__ Pre pre(int64_t i) const { return Pre{r[i], x[i], xc[agg[i]], dinv[i]}; }
  __device__ __forceinline__ void operator()(int64_t i, T s, const Pre& p, double*) const {
    const T r0 = p.r - s;
    r[i] = r0;
    d0[i] = inv_theta * p.dv * r0;
    x[i] = p.x + p.xa;
  }
  __device__ void finish(const double*) const {}
};

// Algorithmic bytes of one row pass over an operator with elements of size t:
// the CSR arrays once, the gathered vector once, and `streams` further
// length-n vector streams (reads or writes) of the epilogue.
// Algorithmic bytes of one pass: the CSR stream (the weights only when the
// operator stores them), the row pointers, the gathered vector once, and the
// epilogue's vector streams.
static double pass_bytes(int64_t n, int64_t nnz, int t, int streams, bool weights = true) {
  return (double)nnz * (4.0 + (weights ? t : 0)) + (double)(n + 1) * 8.0 + (double)n * t * (1 + streams);
}

template <typename T>
static int cheb_streams(const EpiCheb<T>& e) {
  return 2 + (e.dout ? 2 : 0) + (e.x ? (e.x_mode == 2 ? 2 : 1) : 0);
}

// A row pass over level `level`'s operator, timed when the workspace profiles.
template <typename T, int NRED, class Term, class Epi>
static void op_pass(Workspace& ws, int level, const OpView<T>& op, const Term& term, const Epi& epi, int streams,
                    cudaStream_t s, double* rp = nullptr, unsigned* rt = nullptr, double* ro = nullptr,
                    const double* gate = nullptr) {
  const bool timed = ws.prof.on && gate == nullptr;  // a gated pass may do nothing: not timed
  if (timed) ws.prof.begin(s);
  launch_rows<T, NRED>(op.n, op.rowptr, op.col, term, op.plan, epi, s, rp, rt, ro, gate);
  if (timed) ws.prof.end(s, level, pass_bytes(op.n, op.nnz, (int)sizeof(T), streams, op.w != nullptr));
}

// The PCG's reduction over the preconditioned residual z (see k_z_reduce),
// when the kernel that produces z computes it on the way.
struct ZSums {
  const double* r = nullptr;   // null: no reduction
  const double* ro = nullptr;
  double* scal = nullptr;
  double* partials = nullptr;
  unsigned* ticket = nullptr;
};
__device__ void z_sums_finish(int64_t n, double* scal, int first);

// x = P x_c + Fsmooth(f) at an elimination level: kept vertices take their
// coarse value; an eliminated f takes (f_f + sum_c w_fc x_c) / d_f. At level 0
// of a PCG iteration the same kernel also forms the sums over z = x (zs).
template <typename T, bool kZ>
__global__ void k_elim_prolong(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                               const T* __restrict__ w, T wc, const T* __restrict__ dinv,
                               const int32_t* __restrict__ cmap,
                               const T* __restrict__ f, const T* __restrict__ xc, T* __restrict__ x, ZSums zs) {
  int first = 0;
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if constexpr (kZ) first = zs.scal[kIter] == 0.0;
  LG_GRID_STRIDE(i, n) {
    const int32_t c = cmap[i];
    T v;
    if (c >= 0) {
      v = xc[c];
    } else {
      T s = f[i];
      for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) s += (w ? w[k] : wc) * xc[cmap[col[k]]];
      v = s * dinv[i];
    }
    x[i] = v;
    if constexpr (kZ) {
      const double zi = (double)v, ri = zs.r[i], roi = first ? 0.0 : zs.ro[i];
      acc[0] += zi;
      acc[1] += zi * ri;
      acc[2] += zi * roi;
      acc[3] += ri;
      acc[4] += roi;
    }
  }
  if constexpr (kZ) {
    if (grid_sum<kVT, 5>(acc, zs.partials, zs.ticket, zs.scal + kZ0)) z_sums_finish(n, zs.scal, first);
  }
}

// x += P x_c at an aggregation level (P = R^T).
template <typename T>
__global__ void k_agg_prolong(int64_t n, const int32_t* __restrict__ agg, const T* __restrict__ xc, T* __restrict__ x) {
  LG_GRID_STRIDE(i, n) x[i] += xc[agg[i]];
}

template <typename T>
__global__ void k_axpy1(int64_t n, const T* __restrict__ d, T* __restrict__ x) {
  LG_GRID_STRIDE(i, n) x[i] += d[i];
}

// Coarsest level: x = L_c^+ f with the FP64 pseudo-inverse, one warp per row.
template <typename T>
__global__ void k_coarse_apply(int64_t n, const double* __restrict__ pinv, const T* __restrict__ f, T* __restrict__ x) {
  const int lane = threadIdx.x & 31;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n;
       i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    double s = 0.0;
    for (int64_t j = lane; j < n; j += 32) s += pinv[i * n + j] * (double)f[j];
    s = group_sum<32>(s, 0xffffffffu);
    if (lane == 0) x[i] = (T)s;
  }
}

// Level-0 input of the cycle: f = (T) r; d_0 = D^-1 f / theta when level 0 smooths.
template <typename T>
__global__ void k_cycle_in(int64_t n, const double* __restrict__ r, T* __restrict__ f, T* __restrict__ d0,
                           const T* __restrict__ dinv, T inv_theta) {
  LG_GRID_STRIDE(i, n) {
    const T v = (T)r[i];
    f[i] = v;
    if (d0) d0[i] = v * dinv[i] * inv_theta;
  }
}

template <typename T>
__global__ void k_cycle_out(int64_t n, const T* __restrict__ x, double* __restrict__ out) {
  LG_GRID_STRIDE(i, n) out[i] = (double)x[i];
}

// ---------------------------------------------------------------------------
// V-cycle driver (Algorithm 1, gamma = 1, x = 0 on entry).
// ---------------------------------------------------------------------------
template <typename T> std::vector<LevelVecs<T>>& vecs(Workspace& ws);
template <> std::vector<LevelVecs<double>>& vecs<double>(Workspace& ws) { return ws.v64; }
template <> std::vector<LevelVecs<float>>& vecs<float>(Workspace& ws) { return ws.v32; }

template <typename T> const T* pt_coef_of(const Level& L);
template <> const double* pt_coef_of<double>(const Level& L) { return L.pt_coef.get(); }
template <> const float* pt_coef_of<float>(const Level& L) { return L.pt_coef32.get(); }

// ---------------------------------------------------------------------------
// K-cycle (Section 3.7): two FCG iterations at an aggregation level, the
// level's own cycle as the preconditioner (see kcycle_level). Sums in FP64.
// ---------------------------------------------------------------------------
template <typename T>
struct EpiKStore {  // y = L c
  T* y;
  __device__ __forceinline__ NoPre pre(int64_t) const { return NoPre{}; }
  __device__ __forceinline__ void operator()(int64_t i, T s, NoPre, double*) const { y[i] = s; }
  __device__ void finish(const double*) const {}
};

// c1 = x (kept), rho1 = c1.v1, c1.f; the last block: t1 = c1.f / rho1 (0 and
// the flag cleared when rho1 is not positive).
template <typename T>
__global__ void k_kfirst(int64_t n, const T* __restrict__ x, const T* __restrict__ v1, const T* __restrict__ f,
                         T* __restrict__ c1, double* ks, double* partials, unsigned* ticket) {
  double acc[2] = {0.0, 0.0};
  LG_GRID_STRIDE(i, n) {
    const T xi = x[i];
    c1[i] = xi;
    acc[0] += (double)xi * (double)v1[i];
    acc[1] += (double)xi * (double)f[i];
  }
  if (grid_sum<kVT, 2>(acc, partials, ticket, ks + kRho1)) {
    const bool ok = ks[kRho1] > 0.0 && isfinite(ks[kRho1]);
    ks[kOk1] = ok ? 1.0 : 0.0;
    ks[kT1] = ok ? ks[kA1] / ks[kRho1] : 0.0;
  }
}

// r1 = f - t1 v1 in place of f, and its first Chebyshev direction
// d_0 = D^-1 r1 / theta: the input of the level's second cycle.
template <typename T>
__global__ void k_kres(int64_t n, T* __restrict__ f, const T* __restrict__ v1, const T* __restrict__ dinv,
                       T inv_theta, T* __restrict__ d0, const double* ks) {
  const T t1 = (T)ks[kT1];
  LG_GRID_STRIDE(i, n) {
    const T r = f[i] - t1 * v1[i];
    f[i] = r;
    d0[i] = r * dinv[i] * inv_theta;
  }
}

// With x = c2: g = c2.v1, c2.v2, c2.r1; the last block forms the weights of
// x = u1 c1 + u2 c2 (rho2 = c2.v2 - g^2 / rho1; u1 = t1 - g (c2.r1) / (rho1
// rho2), u2 = (c2.r1) / rho2; x = c1 when rho1 was not positive, x = t1 c1
// when rho2 is not).
template <typename T>
__global__ void k_ksecond(int64_t n, const T* __restrict__ x, const T* __restrict__ v1, const T* __restrict__ v2,
                          const T* __restrict__ r1, double* ks, double* partials, unsigned* ticket) {
  double acc[3] = {0.0, 0.0, 0.0};
  LG_GRID_STRIDE(i, n) {
    const double xi = (double)x[i];
    acc[0] += xi * (double)v1[i];
    acc[1] += xi * (double)v2[i];
    acc[2] += xi * (double)r1[i];
  }
  if (grid_sum<kVT, 3>(acc, partials, ticket, ks + kG)) {
    double u1 = 1.0, u2 = 0.0;
    if (ks[kOk1] != 0.0) {
      const double rho1 = ks[kRho1], t1 = ks[kT1], g = ks[kG], a2 = ks[kA2];
      const double rho2 = ks[kB2] - g * g / rho1;
      if (rho2 > 0.0 && isfinite(rho2)) {
        u1 = t1 - g * a2 / (rho1 * rho2);
        u2 = a2 / rho2;
      } else {
        u1 = t1;
      }
    }
    ks[kU1] = u1;
    ks[kU2] = u2;
  }
}

template <typename T>
__global__ void k_kcombine(int64_t n, const T* __restrict__ c1, T* __restrict__ x, const double* ks) {
  const double u1 = ks[kU1], u2 = ks[kU2];
  LG_GRID_STRIDE(i, n) x[i] = (T)(u1 * (double)c1[i] + u2 * (double)x[i]);
}

// Next level's d_0 target, when that level smooths.
template <typename T>
static void next_dir(Hier& h, Workspace& ws, int l, T** d0, const T** dinv, T* inv_theta) {
  const Level& N = *h.levels[l + 1];
  if (N.kind == LG_LEVEL_AGG) {
    *d0 = vecs<T>(ws)[l + 1].dA.get();
    *dinv = N.op<T>().dinv;
    *inv_theta = (T)h.cheb[l + 1].inv_theta;
  } else {
    *d0 = nullptr;
    *dinv = nullptr;
    *inv_theta = T(0);
  }
}

// Precondition: level l's f (and d_0 = dA when l smooths) hold the input.
// Postcondition: level l's x holds the cycle's result.
template <typename T>
static void kcycle_level(Hier& h, Workspace& ws, int l, cudaStream_t s);

template <typename T>
static void cycle_level(Hier& h, Workspace& ws, int l, cudaStream_t s, const ZSums& zs = ZSums{},
                        bool body = false) {
  const Level& L = *h.levels[l];
  if (!body && h.opts.kcycle && L.kind == LG_LEVEL_AGG && l != h.first_agg) {
    kcycle_level<T>(h, ws, l, s);
    return;
  }
  LevelVecs<T>& V = vecs<T>(ws)[l];
  const int64_t n = L.n;
  if (L.kind == LG_LEVEL_COARSEST) {
    k_coarse_apply<T><<<grid_for(n * 32, kVT, kSMs * 8), kVT, 0, s>>>(n, L.pinv.get(), V.f.get(), V.x.get());
    LG_LAUNCH_CHECK();
    return;
  }
  const LevelScratch& sc = ws.scratch[l];
  LevelVecs<T>& C = vecs<T>(ws)[l + 1];
  T* d0n;
  const T* dinvn;
  T itn;
  next_dir<T>(h, ws, l, &d0n, &dinvn, &itn);
  if (L.kind == LG_LEVEL_ELIM) {
    launch_rows<T, 0>(L.nc, L.pt_ptr.get(), L.pt_f.get(), WGatherTerm<T>{pt_coef_of<T>(L), V.f.get()},
                      sc.pt.bind(L.pt_plan.plan),
                      EpiElimRestrict<T>{V.f.get(), L.cfine.get(), C.f.get(), d0n, dinvn, itn}, s);
    cycle_level<T>(h, ws, l + 1, s);
    const OpView<T> op = L.op<T>();
    if (zs.r)
      k_elim_prolong<T, true><<<vblocks(n), kVT, 0, s>>>(n, op.rowptr, op.col, op.w, op.wc, op.dinv, L.cmap.get(),
                                                        V.f.get(), C.x.get(), V.x.get(), zs);
    else
      k_elim_prolong<T, false><<<vblocks(n), kVT, 0, s>>>(n, op.rowptr, op.col, op.w, op.wc, op.dinv, L.cmap.get(),
                                                         V.f.get(), C.x.get(), V.x.get(), zs);
    LG_LAUNCH_CHECK();
    return;
  }
  // aggregation level
  OpView<T> op = L.op<T>();
  op.plan = sc.op.bind(op.plan);
  const Cheb& ch = h.cheb[l];
  const int deg = h.opts.cheb_degree;
  T* g = V.dA.get();
  T* gn = V.dB.get();
  const T* rin = V.f.get();
  for (int st = 1; st < deg; ++st) {  // pre-smoothing from x = 0
    const EpiCheb<T> e{g, rin, V.r.get(), op.dinv, gn, V.x.get(), st == 1 ? 1 : 2, st == deg - 1,
                       (T)ch.c1[st], (T)ch.c2[st]};
    op_pass<T, 0>(ws, l, op, lap_term<T>(op, g), e, cheb_streams(e), s);
    rin = V.r.get();
    std::swap(g, gn);
  }
  {  // residual r = f - L x of the pre-smoothed x (for degree 1 also x = d_0)
    const EpiCheb<T> e{g, rin, V.r.get(), op.dinv, nullptr, deg == 1 ? V.x.get() : nullptr, 1, 0, T(0), T(0)};
    op_pass<T, 0>(ws, l, op, lap_term<T>(op, g), e, cheb_streams(e), s);
  }
  // r_c = R r, then the coarse cycle
  launch_rows<T, 0>(L.nc, L.mem_ptr.get(), L.mem.get(), GatherTerm<T>{V.r.get()}, sc.mem.bind(L.mem_plan.plan),
                    EpiRestrict<T>{C.f.get(), d0n, dinvn, itn}, s);
  cycle_level<T>(h, ws, l + 1, s);
  if (L.lp_nnz > 0) {
    // x += P x_c, r_0 = r_pre - L P x_c, d_0 = D^-1 r_0 / theta: one pass over W
    OpView<T> lp = L.lp<T>();
    lp.plan = sc.lp.bind(lp.plan);
    op_pass<T, 0>(ws, (int)h.levels.size() + l, lp, lp_term<T>(lp, C.x.get(), L.agg.get()),
                  EpiPost<T>{V.r.get(), V.x.get(), C.x.get(), L.agg.get(), op.dinv, V.dA.get(), (T)ch.inv_theta}, 7,
                  s);
  } else {
    k_agg_prolong<T><<<vblocks(n), kVT, 0, s>>>(n, L.agg.get(), C.x.get(), V.x.get());
    LG_LAUNCH_CHECK();
    // post-smoothing from x: r_0 = f - L x, d_0 = D^-1 r_0 / theta
    const EpiCheb<T> e{V.x.get(), V.f.get(), V.r.get(), op.dinv, V.dA.get(), nullptr, 0, 0, T(0), (T)ch.inv_theta};
    op_pass<T, 0>(ws, l, op, lap_term<T>(op, V.x.get()), e, cheb_streams(e), s);
  }
  g = V.dA.get();
  gn = V.dB.get();
  for (int st = 1; st < deg; ++st) {
    const EpiCheb<T> e{g, V.r.get(), V.r.get(), op.dinv, gn, V.x.get(), 2, st == deg - 1, (T)ch.c1[st],
                       (T)ch.c2[st]};
    op_pass<T, 0>(ws, l, op, lap_term<T>(op, g), e, cheb_streams(e), s);
    std::swap(g, gn);
  }
  if (deg == 1) {
    k_axpy1<T><<<vblocks(n), kVT, 0, s>>>(n, V.dA.get(), V.x.get());
    LG_LAUNCH_CHECK();
  }
}

// K-cycle at aggregation level l (Section 3.7; Notay and Vassilevski's two
// inner iterations): the level's system L_l x = f solved by two FCG
// iterations from x = 0, preconditioned by the level's cycle body (which
// recurses with the K-cycle below):
//   c1 = B f, v1 = L c1, t1 = c1.f / c1.v1, r1 = f - t1 v1,
//   c2 = B r1, v2 = L c2, x = u1 c1 + u2 c2 (k_ksecond).
// Same pre/postconditions as cycle_level; f is overwritten by r1.
template <typename T>
static void kcycle_level(Hier& h, Workspace& ws, int l, cudaStream_t s) {
  const Level& L = *h.levels[l];
  LevelVecs<T>& V = vecs<T>(ws)[l];
  const int64_t n = L.n;
  OpView<T> op = L.op<T>();
  op.plan = ws.scratch[l].op.bind(op.plan);
  double* ks = ws.kscal.get() + (size_t)kKScal * l;
  const int vb = vblocks(n);
  cycle_level<T>(h, ws, l, s, ZSums{}, true);  // c1 in V.x
  op_pass<T, 0>(ws, l, op, lap_term<T>(op, V.x.get()), EpiKStore<T>{V.kv1.get()}, 1, s);
  k_kfirst<T><<<vb, kVT, 0, s>>>(n, V.x.get(), V.kv1.get(), V.f.get(), V.kc1.get(), ks, ws.partials.get(),
                                 ws.tickets.get());
  LG_LAUNCH_CHECK();
  k_kres<T><<<vb, kVT, 0, s>>>(n, V.f.get(), V.kv1.get(), op.dinv, (T)h.cheb[l].inv_theta, V.dA.get(), ks);
  LG_LAUNCH_CHECK();
  cycle_level<T>(h, ws, l, s, ZSums{}, true);  // c2 in V.x
  op_pass<T, 0>(ws, l, op, lap_term<T>(op, V.x.get()), EpiKStore<T>{V.kv2.get()}, 1, s);
  k_ksecond<T><<<vb, kVT, 0, s>>>(n, V.x.get(), V.kv1.get(), V.kv2.get(), V.f.get(), ks, ws.partials.get(),
                                  ws.tickets.get());
  LG_LAUNCH_CHECK();
  k_kcombine<T><<<vb, kVT, 0, s>>>(n, V.kc1.get(), V.x.get(), ks);
  LG_LAUNCH_CHECK();
}

// Level-0 cycle from an FP64 vector r0; result in level 0's x (precision T).
// zs: the PCG's sums over that result, formed by the cycle's last kernel
// when level 0 is an elimination level (returns whether it did).
template <typename T>
static bool cycle_from(Hier& h, Workspace& ws, const double* r0, cudaStream_t s, const ZSums& zs = ZSums{}) {
  const Level& L0 = *h.levels[0];
  LevelVecs<T>& V = vecs<T>(ws)[0];
  T* d0 = nullptr;
  const T* dinv = nullptr;
  T it = T(0);
  if (L0.kind == LG_LEVEL_AGG) {
    d0 = V.dA.get();
    dinv = L0.op<T>().dinv;
    it = (T)h.cheb[0].inv_theta;
  }
  k_cycle_in<T><<<vblocks(L0.n), kVT, 0, s>>>(L0.n, r0, V.f.get(), d0, dinv, it);
  LG_LAUNCH_CHECK();
  const bool fused = L0.kind == LG_LEVEL_ELIM && zs.r != nullptr;
  cycle_level<T>(h, ws, 0, s, fused ? zs : ZSums{});
  return fused;
}

__global__ void k_gather_perm(int64_t n, const int32_t* __restrict__ perm, const double* __restrict__ src,
                              double* __restrict__ dst) {
  LG_GRID_STRIDE(i, n) dst[i] = src[perm[i]];
}

__global__ void k_scatter_perm(int64_t n, const int32_t* __restrict__ perm, const double* __restrict__ src,
                               double* __restrict__ dst) {
  LG_GRID_STRIDE(i, n) dst[perm[i]] = src[i];
}

// y = L_l x on level l's operator, with the row plan the cycle uses (the
// tuned binning, the default workspace's long-row scratch); x and y are
// device vectors of the level's n values in its own numbering.
template <typename T>
struct EpiY {
  T* y;
  __device__ __forceinline__ NoPre pre(int64_t) const { return NoPre{}; }
  __device__ __forceinline__ void operator()(int64_t i, T s, NoPre, double*) const { y[i] = s; }
  __device__ void finish(const double*) const {}
};

template <typename T>
static void level_apply_t(Hier& h, int l, const T* x, T* y, cudaStream_t s) {
  const Level& L = *h.levels[l];
  OpView<T> op = L.op<T>();
  op.plan = h.ws->scratch[l].op.bind(op.plan);
  launch_rows<T, 0>(op.n, op.rowptr, op.col, lap_term<T>(op, x), op.plan, EpiY<T>{y}, s);
}

void level_apply(Hier& h, int l, int precision, const void* x, void* y, cudaStream_t s) {
  if (precision == LG_FP32_HIER)
    level_apply_t<float>(h, l, static_cast<const float*>(x), static_cast<float*>(y), s);
  else
    level_apply_t<double>(h, l, static_cast<const double*>(x), static_cast<double*>(y), s);
}

void vcycle_apply(Hier& h, Workspace& ws, const double* f, double* x, int precision, cudaStream_t s) {
  const int64_t n = h.levels[0]->n;
  k_gather_perm<<<vblocks(n), kVT, 0, s>>>(n, h.perm.get(), f, ws.z.get());
  LG_LAUNCH_CHECK();
  if (precision == LG_FP32_HIER) {
    cycle_from<float>(h, ws, ws.z.get(), s);
    k_cycle_out<float><<<vblocks(n), kVT, 0, s>>>(n, ws.v32[0].x.get(), ws.io.get());
  } else {
    cycle_from<double>(h, ws, ws.z.get(), s);
    k_cycle_out<double><<<vblocks(n), kVT, 0, s>>>(n, ws.v64[0].x.get(), ws.io.get());
  }
  LG_LAUNCH_CHECK();
  k_scatter_perm<<<vblocks(n), kVT, 0, s>>>(n, h.perm.get(), ws.io.get(), x);
  LG_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// FP64 preconditioned CG (Sections 2.3, 4). Scalars live on the device so the
// iteration needs no host round trip except the convergence test.
// ---------------------------------------------------------------------------

__global__ void k_sum1(int64_t n, const double* __restrict__ v, double* partials, unsigned* ticket, double* out) {
  double acc[1] = {0.0};
  LG_GRID_STRIDE(i, n) acc[0] += v[i];
  grid_sum<kVT, 1>(acc, partials, ticket, out);
}

// b_m = b - mean(b) (b in the caller's numbering, gathered into level-0
// order); x = 0; r = b_m; p = 0 (the first update takes beta = 0, and 0 times
// whatever a reused buffer held could be NaN); ||b_m||^2; loop control scalars.
__global__ void k_pcg_init(int64_t n, const double* __restrict__ b, const int32_t* __restrict__ perm,
                           double* __restrict__ bm, double* __restrict__ x, double* __restrict__ r,
                           double* __restrict__ p, double* scal, double* partials, unsigned* ticket, double tol,
                           int maxit, int every) {
  const double mean = scal[kSumB] / (double)n;
  double acc[1] = {0.0};
  LG_GRID_STRIDE(i, n) {
    const double v = b[perm[i]] - mean;
    bm[i] = v;
    r[i] = v;
    x[i] = 0.0;
    p[i] = 0.0;
    acc[0] += v * v;
  }
  if (grid_sum<kVT, 1>(acc, partials, ticket, scal + kBB)) {
    scal[kBreak] = 0.0;
    scal[kRR] = scal[kBB];
    scal[kIter] = 0.0;
    scal[kDone] = 0.0;
    scal[kTol2BB] = tol * tol * scal[kBB];
    scal[kMaxit] = (double)maxit;
    scal[kEvery] = (double)every;
    scal[kNeedTrue] = 0.0;
  }
}

// Sums over the preconditioned residual z (precision T, mean not yet
// removed): sum z, z.r, z.r_old, sum r, sum r_old. The last block derives the
// projected products (z - mean(z)).v = z.v - mean(z) sum v, the Polak-Ribiere
// beta = z^T (r - r_old) / (z_old^T r_old) (0 on the first iteration), and
// stores r^T z for the next alpha.
template <typename T>
__global__ void k_z_reduce(int64_t n, const T* __restrict__ z, const double* __restrict__ r,
                           const double* __restrict__ ro, double* scal, double* partials, unsigned* ticket) {
  const int first = scal[kIter] == 0.0;
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  LG_GRID_STRIDE(i, n) {
    const double zi = (double)z[i], ri = r[i], roi = first ? 0.0 : ro[i];
    acc[0] += zi;
    acc[1] += zi * ri;
    acc[2] += zi * roi;
    acc[3] += ri;
    acc[4] += roi;
  }
  if (grid_sum<kVT, 5>(acc, partials, ticket, scal + kZ0)) z_sums_finish(n, scal, first);
}

// From the five sums: the mean of z, the projected r^T z and the
// Polak-Ribiere beta (0 on the first iteration); breakdown on r^T z <= 0.
__device__ void z_sums_finish(int64_t n, double* scal, int first) {
  const double m = scal[kZ0] / (double)n;
  const double zr = scal[kZ0 + 1] - m * scal[kZ0 + 3];
  const double zro = scal[kZ0 + 2] - m * scal[kZ0 + 4];
  scal[kMeanZ] = m;
  if (first) {
    scal[kBeta] = 0.0;
  } else {
    scal[kBeta] = (zr - zro) / scal[kRZ];
  }
  if (!(zr > 0.0) || !isfinite(zr)) scal[kBreak] = 1.0;
  scal[kRZ] = zr;
}

// p = (z - mean z) + beta p.
template <typename T>
__global__ void k_p_update(int64_t n, const T* __restrict__ z, double* __restrict__ p, const double* scal) {
  const double m = scal[kMeanZ], beta = scal[kBeta];
  LG_GRID_STRIDE(i, n) p[i] = ((double)z[i] - m) + beta * p[i];
}

// q = L p.
struct EpiQ {
  double* q;
  __device__ __forceinline__ NoPre pre(int64_t) const { return NoPre{}; }
  __device__ __forceinline__ void operator()(int64_t i, double s, NoPre, double*) const { q[i] = s; }
  __device__ void finish(const double*) const {}
};

// p^T q; the last block sets alpha = r^T z / p^T q (0 after a breakdown). A
// separate kernel: summing inside the q pass would put a grid-wide ticket on
// every one of its many small blocks.
__global__ void k_pq_dot(int64_t n, const double* __restrict__ p, const double* __restrict__ q, double* scal,
                         double* partials, unsigned* ticket) {
  double acc[1] = {0.0};
  LG_GRID_STRIDE(i, n) acc[0] += p[i] * q[i];
  if (grid_sum<kVT, 1>(acc, partials, ticket, scal + kTmp)) {
    const double pq = scal[kTmp];
    scal[kPQ] = pq;
    if (!(pq > 0.0) || !isfinite(pq) || scal[kBreak] != 0.0) {
      scal[kBreak] = 1.0;
      scal[kAlpha] = 0.0;
    } else {
      scal[kAlpha] = scal[kRZ] / pq;
    }
  }
}

// r_old = r; x += alpha p; r -= alpha q; ||r||^2. The last block counts the
// iteration and asks for the true residual on replacement iterations or when
// the recurrence residual meets the tolerance; without that request it also
// sets the loop condition (inside the graph): go on unless broken down or at
// max_iter.
__global__ void k_xr_update(int64_t n, double* __restrict__ x, double* __restrict__ r, double* __restrict__ ro,
                            const double* __restrict__ p, const double* __restrict__ q, double* scal,
                            double* partials, unsigned* ticket, cudaGraphConditionalHandle handle, int in_graph) {
  const double a = scal[kAlpha];
  double acc[1] = {0.0};
  LG_GRID_STRIDE(i, n) {
    const double ri = r[i];
    ro[i] = ri;
    x[i] += a * p[i];
    const double rn = ri - a * q[i];
    r[i] = rn;
    acc[0] += rn * rn;
  }
  if (grid_sum<kVT, 1>(acc, partials, ticket, scal + kRR)) {
    const double it = scal[kIter] + 1.0;
    scal[kIter] = it;
    const bool need = fmod(it, scal[kEvery]) == 0.0 || scal[kRR] <= scal[kTol2BB];
    scal[kNeedTrue] = need ? 1.0 : 0.0;
    if (!need && in_graph) cudaGraphSetConditional(handle, scal[kBreak] == 0.0 && it < scal[kMaxit] ? 1u : 0u);
  }
}

// r = b_m - L x (true residual).
struct EpiTrueRes {
  const double* bm;
  double* r;
  __device__ __forceinline__ double pre(int64_t i) const { return bm[i]; }
  __device__ __forceinline__ void operator()(int64_t i, double s, double b, double*) const { r[i] = b - s; }
  __device__ void finish(const double*) const {}
};

// ||r||^2 into scal[kRR]; skipped like the pass before it when gated off.
// Inside the PCG loop (loop = 1) the last block also ends the iteration:
// converged once this true residual meets the tolerance; the loop condition
// (inside the graph) is to go on unless converged, broken down or at max_iter.
__global__ void k_rr(int64_t n, const double* __restrict__ r, double* scal, double* partials, unsigned* ticket,
                     const double* gate, int loop, cudaGraphConditionalHandle handle, int in_graph) {
  if (gate && *gate == 0.0) return;
  double acc[1] = {0.0};
  LG_GRID_STRIDE(i, n) acc[0] += r[i] * r[i];
  if (grid_sum<kVT, 1>(acc, partials, ticket, scal + kRR) && loop) {
    const bool conv = scal[kRR] <= scal[kTol2BB];
    if (conv) scal[kDone] = 1.0;
    const bool cont = !conv && scal[kBreak] == 0.0 && scal[kIter] < scal[kMaxit];
    if (in_graph) cudaGraphSetConditional(handle, cont ? 1u : 0u);
  }
}

// out[perm[i]] = x[i] - mean(x): back to the caller's numbering, mean removed.
__global__ void k_sub_mean_out(int64_t n, const double* __restrict__ x, const int32_t* __restrict__ perm,
                               const double* scal_sum, double* __restrict__ out) {
  const double m = scal_sum[0] / (double)n;
  LG_GRID_STRIDE(i, n) out[perm[i]] = x[i] - m;
}

Workspace::~Workspace() {
  for (auto& g : graph)
    if (g) cudaGraphExecDestroy(g);
  if (host_scal) cudaFreeHost(host_scal);
}

std::unique_ptr<Workspace> make_workspace(Hier& h, int k, cudaStream_t s) {
  auto ws = std::make_unique<Workspace>();
  ws->k = k;
  ws->alloc_stream = s;
  int64_t* c = &ws->bytes;
  const size_t L = h.levels.size();
  ws->v64.resize(L);
  ws->v32.resize(L);
  ws->scratch.resize(L);
  int64_t max_grid = 1;
  for (size_t l = 0; l < L; ++l) {
    const Level& lv = *h.levels[l];
    const size_t n = (size_t)lv.n * k;
    const bool smooth = lv.kind == LG_LEVEL_AGG;
    for (int prec = 0; prec < 2; ++prec) {
      if (prec == 0 && h.fp32_only) continue;  // FP32-hierarchy solves only: no FP64 cycle vectors
      const bool kc = h.opts.kcycle && smooth && (int)l != h.first_agg;
      auto alloc = [&](auto& V) {
        V.f.alloc(n, s, c);
        V.x.alloc(n, s, c);
        if (smooth) {
          V.r.alloc(n, s, c);
          V.dA.alloc(n, s, c);
          V.dB.alloc(n, s, c);
        }
        if (kc) {
          V.kc1.alloc(n, s, c);
          V.kv1.alloc(n, s, c);
          V.kv2.alloc(n, s, c);
        }
      };
      if (prec == 0) alloc(ws->v64[l]); else alloc(ws->v32[l]);
    }
    max_grid = std::max<int64_t>(max_grid, lv.plan.plan.grid());
    ws->scratch[l].op.make(lv.plan.plan, k, s, c);
    if (lv.kind == LG_LEVEL_AGG) ws->scratch[l].mem.make(lv.mem_plan.plan, k, s, c);
    if (lv.lp_nnz > 0) ws->scratch[l].lp.make(lv.lp_plan.plan, k, s, c);
    if (lv.kind == LG_LEVEL_ELIM) ws->scratch[l].pt.make(lv.pt_plan.plan, k, s, c);
  }
  const size_t n0 = (size_t)h.levels[0]->n * k;
  ws->bm.alloc(n0, s, c);
  ws->x.alloc(n0, s, c);
  ws->r.alloc(n0, s, c);
  ws->ro.alloc(n0, s, c);
  ws->z.alloc(n0, s, c);
  ws->p.alloc(n0, s, c);
  ws->q.alloc(n0, s, c);
  ws->io.alloc(n0, s, c);
  max_grid = std::max<int64_t>(max_grid, kSMs * 8);
  ws->partials.alloc((size_t)max_grid * (k > 1 ? 5 * kMaxCols : 8), s, c);
  ws->tickets.alloc(4, s, c);
  LG_CUDA(cudaMemsetAsync(ws->tickets.get(), 0, 4 * sizeof(unsigned), s));
  ws->kscal.alloc((size_t)kKScal * L, s, c);
  LG_CUDA(cudaMemsetAsync(ws->kscal.get(), 0, sizeof(double) * kKScal * L, s));
  ws->scal.alloc((size_t)kNScal * k, s, c);
  LG_CUDA(cudaMemsetAsync(ws->scal.get(), 0, sizeof(double) * kNScal * k, s));
  LG_CUDA(cudaMallocHost(&ws->host_scal, sizeof(double) * kNScal * k));
  return ws;
}

// One PCG iteration: z = M r (cycle in T) with its sums, beta, p; q = L p;
// p^T q and alpha; x, r with the true-residual request; the requested true
// residual, which decides convergence. The loop condition is set by the
// update kernel, or by the true residual's when it runs.
static void true_residual(Hier& h, Workspace& ws, cudaStream_t s, const double* gate, int loop,
                          cudaGraphConditionalHandle handle, int in_graph);

template <typename T>
static void pcg_body(Hier& h, Workspace& ws, cudaStream_t s, cudaGraphConditionalHandle handle, int in_graph) {
  const Level& L0 = *h.levels[0];
  const int64_t n = L0.n;
  double* scal = ws.scal.get();
  const ZSums zs{ws.r.get(), ws.ro.get(), scal, ws.partials.get(), ws.tickets.get()};
  const T* z = vecs<T>(ws)[0].x.get();
  if (!cycle_from<T>(h, ws, ws.r.get(), s, zs)) {
    k_z_reduce<T><<<vblocks(n), kVT, 0, s>>>(n, z, ws.r.get(), ws.ro.get(), scal, ws.partials.get(),
                                             ws.tickets.get());
    LG_LAUNCH_CHECK();
  }
  k_p_update<T><<<vblocks(n), kVT, 0, s>>>(n, z, ws.p.get(), scal);
  LG_LAUNCH_CHECK();
  OpView<double> op = L0.op<double>();
  op.plan = ws.scratch[0].op.bind(op.plan);
  op_pass<double, 0>(ws, 0, op, lap_term<double>(op, ws.p.get()), EpiQ{ws.q.get()}, 1, s);
  k_pq_dot<<<vblocks(n), kVT, 0, s>>>(n, ws.p.get(), ws.q.get(), scal, ws.partials.get(), ws.tickets.get());
  LG_LAUNCH_CHECK();
  k_xr_update<<<vblocks(n), kVT, 0, s>>>(n, ws.x.get(), ws.r.get(), ws.ro.get(), ws.p.get(), ws.q.get(), scal,
                                        ws.partials.get(), ws.tickets.get(), handle, in_graph);
  LG_LAUNCH_CHECK();
  true_residual(h, ws, s, scal + kNeedTrue, 1, handle, in_graph);
}

static void true_residual(Hier& h, Workspace& ws, cudaStream_t s, const double* gate, int loop,
                          cudaGraphConditionalHandle handle, int in_graph) {
  const Level& L0 = *h.levels[0];
  OpView<double> op = L0.op<double>();
  op.plan = ws.scratch[0].op.bind(op.plan);
  double* scal = ws.scal.get();
  op_pass<double, 0>(ws, 0, op, lap_term<double>(op, ws.x.get()), EpiTrueRes{ws.bm.get(), ws.r.get()}, 2, s,
                     nullptr, nullptr, nullptr, gate);
  k_rr<<<vblocks(L0.n), kVT, 0, s>>>(L0.n, ws.r.get(), scal, ws.partials.get(), ws.tickets.get(), gate, loop, handle,
                                     in_graph);
  LG_LAUNCH_CHECK();
}

static void read_scal(Workspace& ws, cudaStream_t s) {
  LG_CUDA(cudaMemcpyAsync(ws.host_scal, ws.scal.get(), sizeof(double) * kNScal, cudaMemcpyDeviceToHost, s));
  LG_CUDA(cudaStreamSynchronize(s));
  if (ws.prof.on) ws.prof.collect();
}

// The whole PCG loop as one graph: a WHILE node whose body is one iteration
// (captured once per workspace and precision) and whose condition the
// iteration's last kernel sets.
template <typename T>
static cudaGraphExec_t pcg_graph(Hier& h, Workspace& ws, cudaStream_t s) {
  const int slot = sizeof(T) == 4 ? 1 : 0;
  if (ws.graph[slot]) return ws.graph[slot];
  cudaGraph_t g = nullptr;
  LG_CUDA(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle handle;
  LG_CUDA(cudaGraphConditionalHandleCreate(&handle, g, 1u, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = handle;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  LG_CUDA(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  LG_CUDA(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  try {
    pcg_body<T>(h, ws, s, handle, 1);
  } catch (...) {
    cudaGraph_t dummy;
    cudaStreamEndCapture(s, &dummy);
    cudaGraphDestroy(g);
    throw;
  }
  LG_CUDA(cudaStreamEndCapture(s, &body));
  cudaGraphExec_t exec = nullptr;
  LG_CUDA(cudaGraphInstantiate(&exec, g, 0));
  cudaGraphDestroy(g);
  ws.graph[slot] = exec;
  return exec;
}

// Work of one PCG iteration in finest-residual units (Section 2.3.1: work =
// flops / flops of a finest residual, approximated by operator nonzeros). An
// operator application on level l costs A_l = nnz_off + n. Per iteration:
// A_0 for q = L p, plus the cycle from level 0, where an aggregation body costs
// 2 deg A_l (pre- and post-smoothing passes; where the level has W = L P, one
// of them costs nnz(W) + n_l instead) + 2 n_l (restriction, prolongation) + its
// coarse solve; a K-cycle level two bodies + 2 A_l; an elimination level
// 2 nnz_F + n_c + n_l (restriction and prolongation through the F rows'
// entries) + its coarse solve; the coarsest level n_c^2.
static double solve_work(const Hier& h, int l) {
  const Level& L = *h.levels[l];
  const double A = (double)(L.nnz + L.n);
  if (L.kind == LG_LEVEL_COARSEST) return (double)L.n * (double)L.n;
  if (L.kind == LG_LEVEL_ELIM)
    return 2.0 * (double)L.pt_f.size() + (double)L.nc + (double)L.n + solve_work(h, l + 1);
  double body = 2.0 * h.opts.cheb_degree * A + 2.0 * (double)L.n + solve_work(h, l + 1);
  if (L.lp_nnz > 0) body += (double)(L.lp_nnz + L.n) - A;
  if (h.opts.kcycle && l != h.first_agg) return 2.0 * body + 2.0 * A;
  return body;
}

double iteration_work(const Hier& h) {
  const Level& L0 = *h.levels[0];
  const double A0 = (double)(L0.nnz + L0.n);
  return (A0 + solve_work(h, 0)) / A0;
}

int pcg_solve(Hier& h, Workspace& ws, const double* b, double* x, double tol, int precision, cudaStream_t s,
              lg_info* info) {
  const Level& L0 = *h.levels[0];
  const int64_t n = L0.n;
  double* scal = ws.scal.get();
  cudaEvent_t e0, e1;
  LG_CUDA(cudaEventCreate(&e0));
  LG_CUDA(cudaEventCreate(&e1));
  LG_CUDA(cudaEventRecord(e0, s));
  const int maxit = h.opts.max_iter;
  const int every = h.opts.residual_replace > 0 ? h.opts.residual_replace : 1 << 30;
  k_sum1<<<vblocks(n), kVT, 0, s>>>(n, b, ws.partials.get(), ws.tickets.get(), scal + kSumB);
  LG_LAUNCH_CHECK();
  k_pcg_init<<<vblocks(n), kVT, 0, s>>>(n, b, h.perm.get(), ws.bm.get(), ws.x.get(), ws.r.get(), ws.p.get(), scal,
                                        ws.partials.get(), ws.tickets.get(), tol, maxit, every);
  LG_LAUNCH_CHECK();
  read_scal(ws, s);
  const double bb = ws.host_scal[kBB];
  const bool fp32 = precision == LG_FP32_HIER;
  if (bb > 0.0 && maxit > 0) {
    if (h.opts.use_graphs && !ws.prof.on && !debug_sync()) {
      cudaGraphExec_t ge = fp32 ? pcg_graph<float>(h, ws, s) : pcg_graph<double>(h, ws, s);
      LG_CUDA(cudaGraphLaunch(ge, s));
    } else {
      for (int it = 0; it < maxit; ++it) {
        if (fp32) pcg_body<float>(h, ws, s, cudaGraphConditionalHandle{}, 0);
        else pcg_body<double>(h, ws, s, cudaGraphConditionalHandle{}, 0);
        read_scal(ws, s);
        const double* hs = ws.host_scal;
        const bool conv = hs[kDone] != 0.0;
        if (conv || hs[kBreak] != 0.0 || hs[kIter] >= hs[kMaxit]) break;
      }
    }
    read_scal(ws, s);
  }
  const double* hs = ws.host_scal;
  int status = LG_OK, it = 0;
  double rel = 0.0;
  if (bb > 0.0) {
    it = (int)hs[kIter];
    status = hs[kDone] != 0.0 ? LG_OK : hs[kBreak] != 0.0 ? LG_ERR_BREAKDOWN : LG_ERR_NOT_CONVERGED;
    rel = std::sqrt(hs[kRR] / bb);
  }
  if (status != LG_OK && bb > 0.0) {
    true_residual(h, ws, s, nullptr, 0, cudaGraphConditionalHandle{}, 0);
    read_scal(ws, s);
    rel = std::sqrt(ws.host_scal[kRR] / bb);
  }
  // x with its mean removed, in the caller's numbering, copied out
  k_sum1<<<vblocks(n), kVT, 0, s>>>(n, ws.x.get(), ws.partials.get(), ws.tickets.get(), scal + kTmp);
  LG_LAUNCH_CHECK();
  k_sub_mean_out<<<vblocks(n), kVT, 0, s>>>(n, ws.x.get(), h.perm.get(), scal + kTmp, ws.io.get());
  LG_LAUNCH_CHECK();
  LG_CUDA(cudaMemcpyAsync(x, ws.io.get(), sizeof(double) * n, cudaMemcpyDefault, s));
  LG_CUDA(cudaEventRecord(e1, s));
  LG_CUDA(cudaStreamSynchronize(s));
  float ms = 0.f;
  LG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (info) {
    info->status = status;
    info->iterations = it;
    info->relres = rel;
    info->solve_ms = ms;
    info->work_units = it * iteration_work(h);
    info->levels = (int)h.levels.size();
    info->setup_ms = h.setup_ms;
    info->nnz = h.nnz0;
  }
  return status;
}

}  // namespace lg
