// Multi-right-hand-side solve: the V-cycle and the FP64 outer CG on k
// columns at once (k <= 32), vectors stored row-major [n][KP] with KP = k
// rounded up to a power of two (the padding columns carry zeros), so that the
// values of one vertex are one aligned, contiguous stretch.
//
// Every SpMV of the cycle becomes an SpMM pass. The rows of an operator are
// cut into virtual rows (a whole row of at most ch entries, or a stretch of
// ch entries of a longer row; ch is chosen per level shape by timing) and a
// virtual row goes to a slice of KP / VEC lanes, each lane holding VEC
// consecutive columns (VEC = 4 floats or 2 doubles, as one vector load). A
// warp thus has several virtual rows in flight, each entry's columns are one
// coalesced access, and every matrix entry is read once for all columns.
//
// A column's arithmetic does not depend on the batch: every virtual row adds
// its entries in entry order, the stretches of a long row are added in order
// by the last of them to finish, and every per-column dot product is summed
// in an order fixed by n alone (see col_reduce). The CG scalars are per
// column; a column whose true residual meets the tolerance is frozen while
// the others go on, and a column's residual is replaced by its true residual
// only on its own schedule. So a right-hand side gives the same bits whether
// it is solved alone or with other columns, whatever their number: the
// server merges requests on one hierarchy into one batch on that basis.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>

#include "lg_hier.h"
#include "lg_rows.cuh"

namespace lg {
namespace {  // internals of this file

constexpr int kBT = 256;

#define LG_GRID_STRIDE(i, n) \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

static inline int bblocks(int64_t n) { return grid_for(n, kBT, kSMs * 8); }

static int pow2_at_least(int k) {
  int p = 1;
  while (p < k) p <<= 1;
  return p;
}

// ---------------------------------------------------------------------------
// Plans of the SpMM passes: virtual rows, longest first.
// ---------------------------------------------------------------------------
struct MPlan {
  int64_t nv = 0;                    // virtual rows
  const int32_t* vrow = nullptr;     // the row of each
  const int64_t* vbeg = nullptr;     // its entries [vbeg, vend)
  const int64_t* vend = nullptr;
  const int32_t* vlong = nullptr;    // the index of its long row, or -1 (a whole row)
  const int32_t* vslot = nullptr;    // its partial-sum slot (long rows: slots of a row consecutive, in entry order)
  const int32_t* lfirst = nullptr;   // per long row: first slot
  const int32_t* lcount = nullptr;   // per long row: stretches
  int64_t nlong = 0, nslots = 0;
  int ch = 256;                      // entries per stretch of a long row
  double* partial = nullptr;         // nslots * kMaxCols (a workspace's)
  unsigned* ticket = nullptr;        // nlong (a workspace's; zero between launches)
};

__global__ void k_mp_count(int64_t n, const int64_t* __restrict__ rowptr, int ch, int64_t* __restrict__ parts,
                           uint8_t* __restrict__ islong) {
  LG_GRID_STRIDE(i, n) {
    const int64_t deg = rowptr[i + 1] - rowptr[i];
    const bool l = deg > ch;
    islong[i] = l;
    parts[i] = l ? (deg + ch - 1) / ch : 1;
  }
}

// Virtual rows in row order, with a sort key that puts the longest first
// (ties in row order: the sort is stable).
__global__ void k_mp_fill(int64_t n, const int64_t* __restrict__ rowptr, int ch, const int64_t* __restrict__ voff,
                          const uint8_t* __restrict__ islong, const int64_t* __restrict__ lidx,
                          const int64_t* __restrict__ sidx, int32_t* __restrict__ vrow, int64_t* __restrict__ vbeg,
                          int64_t* __restrict__ vend, int32_t* __restrict__ vlong, int32_t* __restrict__ vslot,
                          int32_t* __restrict__ lfirst, int32_t* __restrict__ lcount, uint64_t* __restrict__ key,
                          uint64_t* __restrict__ val) {
  LG_GRID_STRIDE(i, n) {
    const int64_t b = rowptr[i], e = rowptr[i + 1], o = voff[i], parts = voff[i + 1] - o;
    const bool l = islong[i];
    if (l) {
      lfirst[lidx[i]] = (int32_t)sidx[i];
      lcount[lidx[i]] = (int32_t)parts;
    }
    for (int64_t q = 0; q < parts; ++q) {
      const int64_t vb = b + q * ch, ve = l ? (vb + ch < e ? vb + ch : e) : e;
      vrow[o + q] = (int32_t)i;
      vbeg[o + q] = vb;
      vend[o + q] = ve;
      vlong[o + q] = l ? (int32_t)lidx[i] : -1;
      vslot[o + q] = l ? (int32_t)(sidx[i] + q) : -1;
      key[o + q] = (uint64_t)(ch - (ve - vb));  // at most ch entries: longer first
      val[o + q] = (uint64_t)(o + q);
    }
  }
}

template <typename A>
__global__ void k_mp_permute(int64_t nv, const uint64_t* __restrict__ order, const A* __restrict__ in,
                             A* __restrict__ out) {
  LG_GRID_STRIDE(v, nv) out[v] = in[order[v]];
}

__global__ void k_mp_slots(int64_t n, const int64_t* __restrict__ parts, const uint8_t* __restrict__ islong,
                           int64_t* __restrict__ slots) {
  LG_GRID_STRIDE(i, n) slots[i] = islong[i] ? parts[i] : 0;
}

struct MPlanStore {
  MPlan plan;
  DBuf<int32_t> vrow, vlong, vslot, lfirst, lcount;
  DBuf<int64_t> vbeg, vend;
  void build(int64_t n, const int64_t* rowptr, int ch, cudaStream_t s, int64_t* counter) {
    plan = MPlan{};
    plan.ch = ch;
    if (n <= 0) return;
    DBuf<int64_t> parts(n + 1, s), lidx(n + 1, s), sidx(n + 1, s), lslots(n + 1, s);
    DBuf<uint8_t> islong(n, s);
    const int g = grid_for(n, 256, kSMs * 16);
    k_mp_count<<<g, 256, 0, s>>>(n, rowptr, ch, parts.get(), islong.get());
    LG_LAUNCH_CHECK();
    k_mp_slots<<<g, 256, 0, s>>>(n, parts.get(), islong.get(), lslots.get());
    LG_LAUNCH_CHECK();
    exclusive_scan(lslots.get(), sidx.get(), n, s);
    exclusive_scan(parts.get(), parts.get(), n, s);
    exclusive_scan_flags(islong.get(), lidx.get(), n, s);
    int64_t tot[3];
    LG_CUDA(cudaMemcpyAsync(&tot[0], parts.get() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    LG_CUDA(cudaMemcpyAsync(&tot[1], lidx.get() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    LG_CUDA(cudaMemcpyAsync(&tot[2], sidx.get() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    LG_CUDA(cudaStreamSynchronize(s));
    const int64_t nv = tot[0];
    plan.nv = nv;
    plan.nlong = tot[1];
    plan.nslots = tot[2];
    DBuf<int32_t> r0(nv, s), l0(nv, s), s0(nv, s);
    DBuf<int64_t> b0(nv, s), e0(nv, s);
    DBuf<uint64_t> key(nv, s), val(nv, s);
    lfirst.alloc(plan.nlong, s, counter);
    lcount.alloc(plan.nlong, s, counter);
    k_mp_fill<<<g, 256, 0, s>>>(n, rowptr, ch, parts.get(), islong.get(), lidx.get(), sidx.get(), r0.get(), b0.get(),
                                e0.get(), l0.get(), s0.get(), lfirst.get(), lcount.get(), key.get(), val.get());
    LG_LAUNCH_CHECK();
    radix_sort_pairs(key.get(), val.get(), nv, bits_for((int64_t)ch + 1), s);
    vrow.alloc(nv, s, counter);
    vlong.alloc(nv, s, counter);
    vslot.alloc(nv, s, counter);
    vbeg.alloc(nv, s, counter);
    vend.alloc(nv, s, counter);
    const int gv = grid_for(nv, 256, kSMs * 16);
    k_mp_permute<<<gv, 256, 0, s>>>(nv, val.get(), r0.get(), vrow.get());
    k_mp_permute<<<gv, 256, 0, s>>>(nv, val.get(), l0.get(), vlong.get());
    k_mp_permute<<<gv, 256, 0, s>>>(nv, val.get(), s0.get(), vslot.get());
    k_mp_permute<<<gv, 256, 0, s>>>(nv, val.get(), b0.get(), vbeg.get());
    k_mp_permute<<<gv, 256, 0, s>>>(nv, val.get(), e0.get(), vend.get());
    LG_LAUNCH_CHECK();
    LG_CUDA(cudaStreamSynchronize(s));  // the temporaries are released on return
    plan.vrow = vrow.get();
    plan.vbeg = vbeg.get();
    plan.vend = vend.get();
    plan.vlong = vlong.get();
    plan.vslot = vslot.get();
    plan.lfirst = lfirst.get();
    plan.lcount = lcount.get();
  }
};

// ---------------------------------------------------------------------------
// Terms of an SpMM pass over one column c of [n][KP] vectors. Each gives
// src() (the gathered vector), coef(e) (entry e's coefficient), rowv(i, c)
// (a per-row value the entries need), step(s, w, xj, xi) (s plus one entry's
// contribution) and finish(i, c, xi, s) (the row's result).
// ---------------------------------------------------------------------------
template <typename T>
struct MLap;

template <>
struct MLap<float> {  // difference form, as the single-vector FP32 pass (null w: every weight wc)
  const float* __restrict__ w;
  const float* __restrict__ x;
  int ld;
  float wc;
  __device__ __forceinline__ const float* src() const { return x; }
  __device__ __forceinline__ float coef(int64_t e) const { return w ? ld_stream(&w[e]) : wc; }
  __device__ __forceinline__ float rowv(int64_t i, int c) const { return x[i * ld + c]; }
  __device__ __forceinline__ float step(float s, float wk, float xj, float xi) const { return fmaf(wk, xi - xj, s); }
  __device__ __forceinline__ float finish(int64_t, int, float, float s) const { return s; }
};

template <>
struct MLap<double> {  // d_i x_i - sum_j w_ij x_j, as the single-vector FP64 pass (null w: every weight wc)
  const double* __restrict__ w;
  const double* __restrict__ x;
  const double* __restrict__ d;
  int ld;
  double wc;
  __device__ __forceinline__ const double* src() const { return x; }
  __device__ __forceinline__ double coef(int64_t e) const { return w ? ld_stream(&w[e]) : wc; }
  __device__ __forceinline__ double rowv(int64_t, int) const { return 0.0; }
  __device__ __forceinline__ double step(double s, double wk, double xj, double) const { return fma(wk, xj, s); }
  __device__ __forceinline__ double finish(int64_t i, int c, double, double s) const {
    return fma(d[i], x[i * ld + c], -s);
  }
};

template <typename T>
struct MGather {  // restriction by member lists: sum v[j][c]
  const T* __restrict__ v;
  __device__ __forceinline__ const T* src() const { return v; }
  __device__ __forceinline__ T coef(int64_t) const { return T(1); }
  __device__ __forceinline__ T rowv(int64_t, int) const { return T(0); }
  __device__ __forceinline__ T step(T s, T, T xj, T) const { return s + xj; }
  __device__ __forceinline__ T finish(int64_t, int, T, T s) const { return s; }
};

// (L P x_c)[i][c] over W = L P off the own aggregate (Level::lp; see LpTerm
// in lg_cycle.cu): FP32 sum_a W_ia (x_c[agg_i][c] - x_c[a][c]); FP64
// d^W_i x_c[agg_i][c] - sum_a W_ia x_c[a][c].
template <typename T>
struct MLp;

template <>
struct MLp<float> {
  const float* __restrict__ w;
  const float* __restrict__ xc;
  const int32_t* __restrict__ agg;
  int ld;
  __device__ __forceinline__ const float* src() const { return xc; }
  __device__ __forceinline__ float coef(int64_t e) const { return ld_stream(&w[e]); }
  __device__ __forceinline__ float rowv(int64_t i, int c) const { return xc[(int64_t)agg[i] * ld + c]; }
  __device__ __forceinline__ float step(float s, float wk, float xj, float xa) const { return fmaf(wk, xa - xj, s); }
  __device__ __forceinline__ float finish(int64_t, int, float, float s) const { return s; }
};

template <>
struct MLp<double> {
  const double* __restrict__ w;
  const double* __restrict__ xc;
  const int32_t* __restrict__ agg;
  const double* __restrict__ d;
  int ld;
  __device__ __forceinline__ const double* src() const { return xc; }
  __device__ __forceinline__ double coef(int64_t e) const { return ld_stream(&w[e]); }
  __device__ __forceinline__ double rowv(int64_t, int) const { return 0.0; }
  __device__ __forceinline__ double step(double s, double wk, double xj, double) const { return fma(wk, xj, s); }
  __device__ __forceinline__ double finish(int64_t i, int c, double, double s) const {
    return fma(d[i], xc[(int64_t)agg[i] * ld + c], -s);
  }
};

template <typename T>
struct MWGather {  // elimination restriction: sum coef_e v[j][c]
  const T* __restrict__ coefs;
  const T* __restrict__ v;
  __device__ __forceinline__ const T* src() const { return v; }
  __device__ __forceinline__ T coef(int64_t e) const { return ld_stream(&coefs[e]); }
  __device__ __forceinline__ T rowv(int64_t, int) const { return T(0); }
  __device__ __forceinline__ T step(T s, T wk, T xj, T) const { return fma(wk, xj, s); }
  __device__ __forceinline__ T finish(int64_t, int, T, T s) const { return s; }
};

// VEC consecutive values of one row of an [n][KP] vector, one aligned load.
template <typename T, int VEC>
struct VecLoad;
template <typename T>
struct VecLoad<T, 1> {
  static __device__ __forceinline__ void load(const T* p, T (&v)[1]) { v[0] = __ldg(p); }
};
template <>
struct VecLoad<float, 2> {
  static __device__ __forceinline__ void load(const float* p, float (&v)[2]) {
    const float2 t = __ldg(reinterpret_cast<const float2*>(p));
    v[0] = t.x;
    v[1] = t.y;
  }
};
template <>
struct VecLoad<float, 4> {
  static __device__ __forceinline__ void load(const float* p, float (&v)[4]) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
  }
};
template <>
struct VecLoad<double, 2> {
  static __device__ __forceinline__ void load(const double* p, double (&v)[2]) {
    const double2 t = __ldg(reinterpret_cast<const double2*>(p));
    v[0] = t.x;
    v[1] = t.y;
  }
};

template <typename T, int KP>
struct MShape {
  static constexpr int VEC = sizeof(T) == 4 ? (KP < 4 ? KP : 4) : (KP < 2 ? KP : 2);
  static constexpr int LS = KP / VEC;  // lanes of a slice
  static constexpr int S = 32 / LS;    // slices (virtual rows in flight) per warp
};

// ---------------------------------------------------------------------------
// The SpMM pass: one virtual row per slice, entries in order, four entries'
// loads issued together; a stretch of a long row leaves its partial sums and
// the last stretch to finish (a per-row ticket) adds them in order.
// ---------------------------------------------------------------------------
template <typename T, int KP, class Term, class Epi>
__global__ void __launch_bounds__(kBT)
k_mrows(const int32_t* __restrict__ col, Term term, MPlan plan, Epi epi, const double* gate) {
  if (gate && *gate == 0.0) return;  // a pass gated off does nothing (every block reads the same flag)
  using Sh = MShape<T, KP>;
  constexpr int VEC = Sh::VEC, LS = Sh::LS, S = Sh::S;
  const int lane = threadIdx.x & 31, slice = lane / LS, sl = lane % LS;
  const int c0 = sl * VEC;
  const int64_t v = ((int64_t)blockIdx.x * (kBT / 32) + (threadIdx.x >> 5)) * S + slice;
  if (v >= plan.nv) return;  // the whole slice leaves together
  const int64_t row = plan.vrow[v], beg = plan.vbeg[v], end = plan.vend[v];
  const T* src = term.src();
  T xi[VEC], acc[VEC];
#pragma unroll
  for (int q = 0; q < VEC; ++q) {
    xi[q] = term.rowv(row, c0 + q);
    acc[q] = T(0);
  }
  int64_t e = beg;
  for (; e + 4 <= end; e += 4) {
    int32_t j[4];
    T wk[4], xv[4][VEC];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      j[u] = ld_stream(&col[e + u]);
      wk[u] = term.coef(e + u);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) VecLoad<T, VEC>::load(src + (int64_t)j[u] * KP + c0, xv[u]);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int q = 0; q < VEC; ++q) acc[q] = term.step(acc[q], wk[u], xv[u][q], xi[q]);
  }
  for (; e < end; ++e) {
    const int32_t j = ld_stream(&col[e]);
    const T wk = term.coef(e);
    T xv[VEC];
    VecLoad<T, VEC>::load(src + (int64_t)j * KP + c0, xv);
#pragma unroll
    for (int q = 0; q < VEC; ++q) acc[q] = term.step(acc[q], wk, xv[q], xi[q]);
  }
  const int32_t lr = plan.vlong[v];
  if (lr < 0) {
#pragma unroll
    for (int q = 0; q < VEC; ++q) epi(row, c0 + q, term.finish(row, c0 + q, xi[q], acc[q]));
    return;
  }
  // a stretch of a long row: partial sums out, then the row's ticket
  const unsigned smask = LS == 32 ? 0xffffffffu : (((1u << LS) - 1u) << (slice * LS));
  const int64_t slot = plan.vslot[v];
#pragma unroll
  for (int q = 0; q < VEC; ++q) plan.partial[slot * kMaxCols + c0 + q] = (double)acc[q];
  __threadfence();
  __syncwarp(smask);
  unsigned last = 0;
  if (sl == 0) {
    const unsigned tk = atomicAdd(&plan.ticket[lr], 1u);
    last = tk == (unsigned)plan.lcount[lr] - 1u;
    if (last) plan.ticket[lr] = 0u;
  }
  last = __shfl_sync(smask, last, slice * LS);
  if (!last) return;
  __threadfence();
  const int32_t f0 = plan.lfirst[lr], cnt = plan.lcount[lr];
#pragma unroll
  for (int q = 0; q < VEC; ++q) {
    double tot = 0.0;
    for (int32_t p = 0; p < cnt; ++p) tot += __ldcg(&plan.partial[(int64_t)(f0 + p) * kMaxCols + c0 + q]);
    epi(row, c0 + q, term.finish(row, c0 + q, xi[q], (T)tot));
  }
}

template <typename T, class Term, class Epi>
static void launch_mrows(int kp, const int32_t* col, const Term& term, const MPlan& plan, const Epi& epi,
                         cudaStream_t s, const double* gate = nullptr) {
  if (plan.nv <= 0) return;
#define LG_MR_CASE(KK)                                                                              \
  case KK: {                                                                                        \
    constexpr int64_t per_block = (kBT / 32) * MShape<T, KK>::S;                                    \
    const int64_t grid = (plan.nv + per_block - 1) / per_block;                                     \
    k_mrows<T, KK><<<(unsigned)grid, kBT, 0, s>>>(col, term, plan, epi, gate);                      \
  } break;
  switch (kp) {
    LG_MR_CASE(1)
    LG_MR_CASE(2)
    LG_MR_CASE(4)
    LG_MR_CASE(8)
    LG_MR_CASE(16)
    LG_MR_CASE(32)
    default: fail(LG_ERR_INVALID, "column block width");
  }
#undef LG_MR_CASE
  LG_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// Epilogues over (row i, column c), vectors [n][ld].
// ---------------------------------------------------------------------------
template <typename T>
struct MEpiCheb {  // one Chebyshev step (see lg_cycle.cu, EpiCheb)
  const T* g;
  const T* rin;
  T* rout;
  const T* dinv;
  T* dout;
  T* x;
  int x_mode, add_d, ld;
  T c1, c2;
  __device__ __forceinline__ void operator()(int64_t i, int c, T s) const {
    const int64_t e = i * ld + c;
    const T r = rin[e] - s;
    rout[e] = r;
    T d = T(0);
    if (dout) {
      d = c1 * g[e] + c2 * dinv[i] * r;
      dout[e] = d;
    }
    if (x) x[e] = (x_mode == 2 ? x[e] : T(0)) + g[e] + (add_d ? d : T(0));
  }
};

template <typename T>
struct MEpiRestrict {
  T* fc;
  T* d0;
  const T* dinvc;
  T inv_theta;
  int ld;
  __device__ __forceinline__ void operator()(int64_t I, int c, T s) const {
    fc[I * ld + c] = s;
    if (d0) d0[I * ld + c] = s * dinvc[I] * inv_theta;
  }
};

template <typename T>
struct MEpiElimRestrict {
  const T* f;
  const int32_t* cfine;
  T* fc;
  T* d0;
  const T* dinvc;
  T inv_theta;
  int ld;
  __device__ __forceinline__ void operator()(int64_t cr, int c, T s) const {
    const T v = f[(int64_t)cfine[cr] * ld + c] + s;
    fc[cr * ld + c] = v;
    if (d0) d0[cr * ld + c] = v * dinvc[cr] * inv_theta;
  }
};

// Start of post-smoothing over W (see EpiPost in lg_cycle.cu): x += P x_c,
// r_0 = r_pre - (L P x_c), d_0 = D^-1 r_0 / theta.
template <typename T>
struct MEpiPost {
  T* r;
  T* x;
  const T* xc;
  const int32_t* agg;
  const T* dinv;
  T* d0;
  T inv_theta;
  int ld;
  __device__ __forceinline__ void operator()(int64_t i, int c, T s) const {
    const int64_t e = i * ld + c;
    const T r0 = r[e] - s;
    r[e] = r0;
    d0[e] = inv_theta * dinv[i] * r0;
    x[e] = x[e] + xc[(int64_t)agg[i] * ld + c];
  }
};

struct MEpiStore {
  double* y;
  int ld;
  __device__ __forceinline__ void operator()(int64_t i, int c, double s) const { y[i * ld + c] = s; }
};

// Per-column scalars, column c at scal[c * kMS + field].
enum MScal : int {
  mBB = 0, mRZ, mPQ, mAlpha, mBeta, mMeanZ, mRR, mSumB, mBreak, mDone, mIter, mTol2BB, mNeedTrue, mActive, mConv,
  kMS = 16
};
// Loop scalars after the k column blocks (scal + k kMS).
enum MGlob : int { gIter = 0, gNeed, gMaxit, gEvery, kMG = 4 };

// r = b_m - L x for the columns whose true residual is due (mNeedTrue, or
// every column at the final check); the others keep their residual.
struct MEpiTrueRes {
  const double* bm;
  double* r;
  const double* scal;
  int k, ld, all;
  __device__ __forceinline__ void operator()(int64_t i, int c, double s) const {
    if (c < k && (all || scal[c * kMS + mNeedTrue] != 0.0)) r[i * ld + c] = bm[i * ld + c] - s;
  }
};

// ---------------------------------------------------------------------------
// Element-wise kernels over [n][KP] (the padding columns included).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_m_elim_prolong(int64_t n, int ld, const int64_t* __restrict__ rowptr,
                                 const int32_t* __restrict__ col, const T* __restrict__ w, T wc,
                                 const T* __restrict__ dinv,
                                 const int32_t* __restrict__ cmap, const T* __restrict__ f, const T* __restrict__ xc,
                                 T* __restrict__ x) {
  LG_GRID_STRIDE(e, n * ld) {
    const int64_t i = e / ld;
    const int c = (int)(e - i * ld);
    const int32_t cm = cmap[i];
    if (cm >= 0) {
      x[e] = xc[(int64_t)cm * ld + c];
    } else {
      T s = f[e];
      for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q) s += (w ? w[q] : wc) * xc[(int64_t)cmap[col[q]] * ld + c];
      x[e] = s * dinv[i];
    }
  }
}

template <typename T>
__global__ void k_m_agg_prolong(int64_t n, int ld, const int32_t* __restrict__ agg, const T* __restrict__ xc,
                                T* __restrict__ x) {
  LG_GRID_STRIDE(e, n * ld) {
    const int64_t i = e / ld;
    x[e] += xc[(int64_t)agg[i] * ld + (e - i * ld)];
  }
}

template <typename T>
__global__ void k_m_axpy1(int64_t m, const T* __restrict__ d, T* __restrict__ x) {
  LG_GRID_STRIDE(e, m) x[e] += d[e];
}

// x = L_c^+ f on the columns: one warp per coarse row, a lane per column,
// the dense row taken in order.
template <typename T>
__global__ void k_m_coarse_apply(int64_t n, int ld, const double* __restrict__ pinv, const T* __restrict__ f,
                                 T* __restrict__ x) {
  const int lane = threadIdx.x & 31;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n;
       i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    for (int c = lane; c < ld; c += 32) {
      double s = 0.0;
      for (int64_t j = 0; j < n; ++j) s += pinv[i * n + j] * (double)f[j * ld + c];
      x[i * ld + c] = (T)s;
    }
  }
}

// Level-0 input: f = (T) r (column block), d_0 = D^-1 f / theta.
template <typename T>
__global__ void k_m_cycle_in(int64_t n, int ld, const double* __restrict__ r, T* __restrict__ f, T* __restrict__ d0,
                             const T* __restrict__ dinv, T inv_theta) {
  LG_GRID_STRIDE(e, n * ld) {
    const T v = (T)r[e];
    f[e] = v;
    if (d0) d0[e] = v * dinv[e / ld] * inv_theta;
  }
}

// ---------------------------------------------------------------------------
// Per-column sums in an order fixed by n alone, so that a column's sums do
// not depend on the batch it is in. The launch has kRG blocks of kBT
// threads; rows are taken in tiles of 256 (32 groups of 8 consecutive rows),
// tile t by block t mod kRG in tile order. Thread pairs (group g, column c)
// keep one running sum per (g, c), row by row; a block adds its 32 group
// sums of a column by a fixed tree and stores one partial per column; the
// last block (a ticket) adds a column's partials as 8 running sums (blocks
// b = j mod 8, in block order) taken in order. f(i, c, acc) adds row i's
// terms of column c (c < KP; it may also update the row) into acc[0..NV).
// Returns true in thread 0 of the last block, after out[q * KP + c].
// ---------------------------------------------------------------------------
constexpr int kRG = kSMs * 8;
constexpr int kRTile = 256;

template <int KP, int NV, class F>
__device__ __forceinline__ bool col_reduce(int64_t n, const F& f, double* partials, unsigned* ticket, double* out) {
  constexpr int kPairs = 32 * KP;
  constexpr int kPer = (kPairs + kBT - 1) / kBT;
  __shared__ double sm[NV][32][KP];
  __shared__ bool am_last;
  double acc[kPer][NV];
#pragma unroll
  for (int p = 0; p < kPer; ++p)
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[p][q] = 0.0;
  const int64_t ntiles = (n + kRTile - 1) / kRTile;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
#pragma unroll
    for (int p = 0; p < kPer; ++p) {
      const int pr = threadIdx.x + p * kBT;
      if (pr < kPairs) {
        const int g = pr / KP, c = pr % KP;
        const int64_t r0 = t * kRTile + g * 8;
        for (int q = 0; q < 8; ++q)
          if (r0 + q < n) f(r0 + q, c, acc[p]);
      }
    }
  }
#pragma unroll
  for (int p = 0; p < kPer; ++p) {
    const int pr = threadIdx.x + p * kBT;
    if (pr < kPairs)
#pragma unroll
      for (int q = 0; q < NV; ++q) sm[q][pr / KP][pr % KP] = acc[p][q];
  }
  __syncthreads();
  for (int h = 16; h >= 1; h >>= 1) {
    for (int pr = threadIdx.x; pr < h * KP; pr += kBT) {
      const int g = pr / KP, c = pr % KP;
#pragma unroll
      for (int q = 0; q < NV; ++q) sm[q][g][c] += sm[q][g + h][c];
    }
    __syncthreads();
  }
  if (threadIdx.x < KP)
#pragma unroll
    for (int q = 0; q < NV; ++q) partials[((int64_t)blockIdx.x * NV + q) * KP + threadIdx.x] = sm[q][0][threadIdx.x];
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    am_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  // the block's own partials are stored: sm holds the 8 running sums per column now
  auto fin = reinterpret_cast<double(*)[8][KP]>(&sm[0][0][0]);
  if (threadIdx.x < 8 * KP) {
    const int j = threadIdx.x / KP, c = threadIdx.x % KP;
    double t[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) t[q] = 0.0;
    for (unsigned b = j; b < gridDim.x; b += 8)
#pragma unroll
      for (int q = 0; q < NV; ++q) t[q] += __ldcg(&partials[((int64_t)b * NV + q) * KP + c]);
#pragma unroll
    for (int q = 0; q < NV; ++q) fin[q][j][c] = t[q];
  }
  __syncthreads();
  if (threadIdx.x < KP) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double u = 0.0;
      for (int j = 0; j < 8; ++j) u += fin[q][j][threadIdx.x];
      out[q * KP + threadIdx.x] = u;
    }
  }
  __syncthreads();
  if (threadIdx.x != 0) return false;
  *ticket = 0u;
  return true;  // one thread of the last block, which alone updates the column scalars
}

// column sums of [n][KP] (the caller's b or the final x)
template <int KP>
__global__ void __launch_bounds__(kBT) k_m_colsum(int64_t n, const double* __restrict__ v, double* partials,
                                                  unsigned* ticket, double* out) {
  col_reduce<KP, 1>(n, [&](int64_t i, int c, double(&a)[1]) { a[0] += v[i * KP + c]; }, partials, ticket, out);
}

// b_m = b - mean(b) per column (b in the caller's numbering, gathered);
// x = 0; r = b_m; p = 0; column scalars initialised. Padding columns are 0.
template <int KP>
__global__ void __launch_bounds__(kBT) k_m_init(int64_t n, int k, const double* __restrict__ b,
                                                const int32_t* __restrict__ perm, const double* __restrict__ colsum,
                                                double* __restrict__ bm, double* __restrict__ x, double* __restrict__ r,
                                                double* __restrict__ p, double* scal, double* partials,
                                                unsigned* ticket, double* tmp, double tol, int maxit, int every) {
  auto f = [&](int64_t i, int c, double(&a)[1]) {
    const int64_t e = i * KP + c;
    const double v = c < k ? b[(int64_t)perm[i] * KP + c] - colsum[c] / (double)n : 0.0;
    bm[e] = v;
    r[e] = v;
    x[e] = 0.0;
    p[e] = 0.0;
    a[0] += v * v;
  };
  if (col_reduce<KP, 1>(n, f, partials, ticket, tmp)) {
    for (int q = 0; q < k; ++q) {
      double* sc = scal + q * kMS;
      sc[mBB] = tmp[q];
      sc[mRR] = tmp[q];
      sc[mBreak] = 0.0;
      sc[mDone] = 0.0;
      sc[mIter] = 0.0;
      sc[mTol2BB] = tol * tol * tmp[q];
      sc[mNeedTrue] = 0.0;
      sc[mActive] = tmp[q] > 0.0 ? 1.0 : 0.0;
      sc[mConv] = 0.0;
    }
    double* gl = scal + k * kMS;
    gl[gIter] = 0.0;
    gl[gNeed] = 0.0;
    gl[gMaxit] = (double)maxit;
    gl[gEvery] = (double)every;
  }
}

// Sums over z per column (as k_z_reduce in lg_cycle.cu), then beta and r^T z.
template <typename T, int KP>
__global__ void __launch_bounds__(kBT) k_m_z_reduce(int64_t n, int k, const T* __restrict__ z,
                                                    const double* __restrict__ r, const double* __restrict__ ro,
                                                    double* scal, double* partials, unsigned* ticket, double* tmp) {
  const int first = scal[k * kMS + gIter] == 0.0;
  auto f = [&](int64_t i, int c, double(&a)[5]) {
    const int64_t e = i * KP + c;
    const double zi = (double)z[e], ri = r[e], roi = first ? 0.0 : ro[e];
    a[0] += zi;
    a[1] += zi * ri;
    a[2] += zi * roi;
    a[3] += ri;
    a[4] += roi;
  };
  if (col_reduce<KP, 5>(n, f, partials, ticket, tmp)) {
    for (int q = 0; q < k; ++q) {
      double* sc = scal + q * kMS;
      const double m = tmp[0 * KP + q] / (double)n;
      const double zr = tmp[1 * KP + q] - m * tmp[3 * KP + q];
      const double zro = tmp[2 * KP + q] - m * tmp[4 * KP + q];
      sc[mMeanZ] = m;
      sc[mBeta] = first ? 0.0 : (zr - zro) / sc[mRZ];
      if (sc[mActive] != 0.0 && (!(zr > 0.0) || !isfinite(zr))) {
        sc[mBreak] = 1.0;
        sc[mActive] = 0.0;
      }
      sc[mRZ] = zr;
    }
  }
}

template <typename T, int KP>
__global__ void k_m_p_update(int64_t n, int k, const T* __restrict__ z, double* __restrict__ p, const double* scal) {
  LG_GRID_STRIDE(e, n * KP) {
    const int c = (int)(e % KP);
    // a frozen (or padding) column keeps p = 0 (its scalars may be 0/0)
    if (c < k && scal[c * kMS + mActive] != 0.0) {
      const double* sc = scal + c * kMS;
      p[e] = ((double)z[e] - sc[mMeanZ]) + sc[mBeta] * p[e];
    } else {
      p[e] = 0.0;
    }
  }
}

template <int KP>
__global__ void __launch_bounds__(kBT) k_m_pq(int64_t n, int k, const double* __restrict__ p,
                                              const double* __restrict__ q, double* scal, double* partials,
                                              unsigned* ticket, double* tmp) {
  auto f = [&](int64_t i, int c, double(&a)[1]) { a[0] += p[i * KP + c] * q[i * KP + c]; };
  if (col_reduce<KP, 1>(n, f, partials, ticket, tmp)) {
    for (int cc = 0; cc < k; ++cc) {
      double* sc = scal + cc * kMS;
      const double pq = tmp[cc];
      sc[mPQ] = pq;
      if (sc[mActive] == 0.0 || !(pq > 0.0) || !isfinite(pq)) {
        if (sc[mActive] != 0.0) sc[mBreak] = 1.0;
        sc[mActive] = 0.0;
        sc[mAlpha] = 0.0;
      } else {
        sc[mAlpha] = sc[mRZ] / pq;
      }
    }
  }
}

// r_old = r; x += alpha p; r -= alpha q (frozen columns keep x and r); ||r||^2.
// The last block counts the iteration and marks the columns whose true
// residual is due: every column on replacement iterations, else each live
// column whose recurrence residual meets its tolerance (as the single-column
// solve does), so no column's residual changes on another's account.
template <int KP>
__global__ void __launch_bounds__(kBT) k_m_xr(int64_t n, int k, double* __restrict__ x, double* __restrict__ r,
                                              double* __restrict__ ro, const double* __restrict__ p,
                                              const double* __restrict__ q, double* scal, double* partials,
                                              unsigned* ticket, double* tmp, cudaGraphConditionalHandle handle,
                                              int in_graph) {
  auto f = [&](int64_t i, int c, double(&a)[1]) {
    const int64_t e = i * KP + c;
    const double ri = r[e];
    ro[e] = ri;
    double rn = ri;
    if (c < k && scal[c * kMS + mActive] != 0.0) {
      x[e] += scal[c * kMS + mAlpha] * p[e];
      rn = ri - scal[c * kMS + mAlpha] * q[e];
      r[e] = rn;
    }
    a[0] += rn * rn;
  };
  if (col_reduce<KP, 1>(n, f, partials, ticket, tmp)) {
    double* gl = scal + k * kMS;
    const double it = gl[gIter] + 1.0;
    gl[gIter] = it;
    const bool periodic = fmod(it, gl[gEvery]) == 0.0;
    bool need = false, any = false;
    for (int cc = 0; cc < k; ++cc) {
      double* sc = scal + cc * kMS;
      sc[mRR] = tmp[cc];
      sc[mNeedTrue] = 0.0;
      if (sc[mActive] != 0.0) {
        sc[mIter] += 1.0;
        any = true;
        if (periodic || sc[mRR] <= sc[mTol2BB]) {
          sc[mNeedTrue] = 1.0;
          need = true;
        }
      }
    }
    gl[gNeed] = need ? 1.0 : 0.0;
    if (!need && in_graph) cudaGraphSetConditional(handle, any && it < gl[gMaxit] ? 1u : 0u);
  }
}

// ||r||^2 per column after a true residual: the replaced columns take the new
// norm. Inside the loop (loop = 1, gated by the request) the last block also
// freezes every replaced live column whose true residual meets the
// tolerance and sets the loop condition: go on while a column is live and the
// iteration bound allows. At the end (loop = 0) every column was replaced.
template <int KP>
__global__ void __launch_bounds__(kBT) k_m_rr(int64_t n, int k, const double* __restrict__ r, double* scal,
                                              double* partials, unsigned* ticket, double* tmp, const double* gate,
                                              int loop, cudaGraphConditionalHandle handle, int in_graph) {
  if (gate && *gate == 0.0) return;
  auto f = [&](int64_t i, int c, double(&a)[1]) { a[0] += r[i * KP + c] * r[i * KP + c]; };
  if (col_reduce<KP, 1>(n, f, partials, ticket, tmp)) {
    for (int cc = 0; cc < k; ++cc)
      if (!loop || scal[cc * kMS + mNeedTrue] != 0.0) scal[cc * kMS + mRR] = tmp[cc];
    if (loop) {
      double* gl = scal + k * kMS;
      const double it = gl[gIter];
      bool any = false;
      for (int cc = 0; cc < k; ++cc) {
        double* sc = scal + cc * kMS;
        if (sc[mNeedTrue] != 0.0 && sc[mActive] != 0.0 && sc[mRR] <= sc[mTol2BB]) {
          sc[mActive] = 0.0;
          sc[mDone] = 1.0;
          sc[mConv] = it;
        }
        sc[mNeedTrue] = 0.0;
        if (sc[mActive] != 0.0) any = true;
      }
      if (in_graph) cudaGraphSetConditional(handle, any && it < gl[gMaxit] ? 1u : 0u);
    }
  }
}

// x columns back to the caller's numbering, column mean removed.
template <int KP>
__global__ void k_m_out(int64_t n, const double* __restrict__ x, const int32_t* __restrict__ perm,
                        const double* __restrict__ colsum, double* __restrict__ out) {
  LG_GRID_STRIDE(e, n * KP) {
    const int64_t i = e / KP;
    const int c = (int)(e - i * KP);
    out[(int64_t)perm[i] * KP + c] = x[e] - colsum[c] / (double)n;
  }
}

// ---------------------------------------------------------------------------
// Host side: plans (shared by every workspace of a hierarchy, their virtual
// row length tuned per level shape), the multi-column cycle and PCG loop.
// ---------------------------------------------------------------------------
struct HierPlans {
  std::vector<std::unique_ptr<MPlanStore>> op, mem, pt, lp;  // per level
  std::vector<int> tuned;                                    // per level: virtual row length of op and lp
};

// Per workspace: the long-row scratch of every plan, reduction scratch,
// totals, and the captured loops.
struct PlanScratchM {
  DBuf<double> partial;
  DBuf<unsigned> ticket;
  void make(const MPlan& p, cudaStream_t s, int64_t* counter) {
    partial.alloc((size_t)(p.nslots > 0 ? p.nslots : 1) * kMaxCols, s, counter);
    ticket.alloc(p.nlong > 0 ? p.nlong : 1, s, counter);
    LG_CUDA(cudaMemsetAsync(ticket.get(), 0, sizeof(unsigned) * (p.nlong > 0 ? p.nlong : 1), s));
  }
  MPlan bind(MPlan p) const {
    p.partial = partial.get();
    p.ticket = ticket.get();
    return p;
  }
};

struct BatchState {
  const HierPlans* plans = nullptr;  // owned by the hierarchy, which outlives its workspaces' use
  std::vector<PlanScratchM> op, mem, pt, lp;  // per level
  DBuf<double> tmp, colsum, partials;         // reduction totals and partials of the column kernels
  DBuf<unsigned> tickets;
  std::map<std::pair<int, int>, cudaGraphExec_t> graphs;  // captured loop per (FP32?, k)
  ~BatchState() {
    for (auto& g : graphs)
      if (g.second) cudaGraphExecDestroy(g.second);
  }
  MPlan op_plan(int l) const { return op[l].bind(plans->op[l]->plan); }
  MPlan mem_plan(int l) const { return mem[l].bind(plans->mem[l]->plan); }
  MPlan pt_plan(int l) const { return pt[l].bind(plans->pt[l]->plan); }
  MPlan lp_plan(int l) const { return lp[l].bind(plans->lp[l]->plan); }
};

template <typename T> static std::vector<LevelVecs<T>>& mvecs(Workspace& ws);
template <> std::vector<LevelVecs<double>>& mvecs<double>(Workspace& ws) { return ws.v64; }
template <> std::vector<LevelVecs<float>>& mvecs<float>(Workspace& ws) { return ws.v32; }
template <typename T> static const T* mpt_coef(const Level& L);
template <> const double* mpt_coef<double>(const Level& L) { return L.pt_coef.get(); }
template <> const float* mpt_coef<float>(const Level& L) { return L.pt_coef32.get(); }

template <typename T>
static MLap<T> mlap(const OpView<T>& op, const T* x, int ld);
template <>
MLap<float> mlap<float>(const OpView<float>& op, const float* x, int ld) {
  return MLap<float>{op.w, x, ld, op.wc};
}
template <>
MLap<double> mlap<double>(const OpView<double>& op, const double* x, int ld) {
  return MLap<double>{op.w, x, op.d, ld, op.wc};
}

template <typename T>
static MLp<T> mlp_term(const OpView<T>& w, const T* xc, const int32_t* agg, int ld);
template <>
MLp<float> mlp_term<float>(const OpView<float>& w, const float* xc, const int32_t* agg, int ld) {
  return MLp<float>{w.w, xc, agg, ld};
}
template <>
MLp<double> mlp_term<double>(const OpView<double>& w, const double* xc, const int32_t* agg, int ld) {
  return MLp<double>{w.w, xc, agg, w.d, ld};
}

template <typename T>
static void mcycle(Hier& h, Workspace& ws, BatchState& bs, int l, int kp, cudaStream_t s) {
  const Level& L = *h.levels[l];
  LevelVecs<T>& V = mvecs<T>(ws)[l];
  const int64_t n = L.n;
  if (L.kind == LG_LEVEL_COARSEST) {
    k_m_coarse_apply<T><<<grid_for(n * 32, kBT, kSMs * 8), kBT, 0, s>>>(n, kp, L.pinv.get(), V.f.get(), V.x.get());
    LG_LAUNCH_CHECK();
    return;
  }
  LevelVecs<T>& C = mvecs<T>(ws)[l + 1];
  const Level& N = *h.levels[l + 1];
  T* d0n = nullptr;
  const T* dinvn = nullptr;
  T itn = T(0);
  if (N.kind == LG_LEVEL_AGG) {
    d0n = C.dA.get();
    dinvn = N.op<T>().dinv;
    itn = (T)h.cheb[l + 1].inv_theta;
  }
  if (L.kind == LG_LEVEL_ELIM) {
    launch_mrows<T>(kp, L.pt_f.get(), MWGather<T>{mpt_coef<T>(L), V.f.get()}, bs.pt_plan(l),
                    MEpiElimRestrict<T>{V.f.get(), L.cfine.get(), C.f.get(), d0n, dinvn, itn, kp}, s);
    mcycle<T>(h, ws, bs, l + 1, kp, s);
    const OpView<T> op = L.op<T>();
    k_m_elim_prolong<T><<<bblocks(n * kp), kBT, 0, s>>>(n, kp, op.rowptr, op.col, op.w, op.wc, op.dinv, L.cmap.get(),
                                                        V.f.get(), C.x.get(), V.x.get());
    LG_LAUNCH_CHECK();
    return;
  }
  const OpView<T> op = L.op<T>();
  const MPlan P = bs.op_plan(l);
  const Cheb& ch = h.cheb[l];
  const int deg = h.opts.cheb_degree;
  T* g = V.dA.get();
  T* gn = V.dB.get();
  const T* rin = V.f.get();
  for (int st = 1; st < deg; ++st) {
    launch_mrows<T>(kp, op.col, mlap<T>(op, g, kp), P,
                    MEpiCheb<T>{g, rin, V.r.get(), op.dinv, gn, V.x.get(), st == 1 ? 1 : 2, st == deg - 1, kp,
                                (T)ch.c1[st], (T)ch.c2[st]},
                    s);
    rin = V.r.get();
    std::swap(g, gn);
  }
  launch_mrows<T>(kp, op.col, mlap<T>(op, g, kp), P,
                  MEpiCheb<T>{g, rin, V.r.get(), op.dinv, nullptr, deg == 1 ? V.x.get() : nullptr, 1, 0, kp, T(0),
                              T(0)},
                  s);
  launch_mrows<T>(kp, L.mem.get(), MGather<T>{V.r.get()}, bs.mem_plan(l), MEpiRestrict<T>{C.f.get(), d0n, dinvn, itn, kp},
                  s);
  mcycle<T>(h, ws, bs, l + 1, kp, s);
  if (L.lp_nnz > 0) {  // x += P x_c, r_0 = r_pre - L P x_c, d_0: one pass over W
    const OpView<T> lp = L.lp<T>();
    launch_mrows<T>(kp, lp.col, mlp_term<T>(lp, C.x.get(), L.agg.get(), kp), bs.lp_plan(l),
                    MEpiPost<T>{V.r.get(), V.x.get(), C.x.get(), L.agg.get(), op.dinv, V.dA.get(), (T)ch.inv_theta,
                                kp},
                    s);
  } else {
    k_m_agg_prolong<T><<<bblocks(n * kp), kBT, 0, s>>>(n, kp, L.agg.get(), C.x.get(), V.x.get());
    LG_LAUNCH_CHECK();
    launch_mrows<T>(kp, op.col, mlap<T>(op, V.x.get(), kp), P,
                    MEpiCheb<T>{V.x.get(), V.f.get(), V.r.get(), op.dinv, V.dA.get(), nullptr, 0, 0, kp, T(0),
                                (T)ch.inv_theta},
                    s);
  }
  g = V.dA.get();
  gn = V.dB.get();
  for (int st = 1; st < deg; ++st) {
    launch_mrows<T>(kp, op.col, mlap<T>(op, g, kp), P,
                    MEpiCheb<T>{g, V.r.get(), V.r.get(), op.dinv, gn, V.x.get(), 2, st == deg - 1, kp, (T)ch.c1[st],
                                (T)ch.c2[st]},
                    s);
    std::swap(g, gn);
  }
  if (deg == 1) {
    k_m_axpy1<T><<<bblocks(n * kp), kBT, 0, s>>>(n * kp, V.dA.get(), V.x.get());
    LG_LAUNCH_CHECK();
  }
}

// One multi-column PCG iteration (as pcg_body in lg_cycle.cu): z = M r, the
// per-column sums, beta and p; q = L p; alpha; x, r and the true-residual
// requests; the requested true residuals, which freeze converged columns.
template <int KP>
static void mtrue_res(Hier& h, Workspace& ws, BatchState& bs, int k, cudaStream_t s, const double* gate, int loop,
                      cudaGraphConditionalHandle handle, int in_graph);

template <typename T, int KP>
static void mbody(Hier& h, Workspace& ws, BatchState& bs, int k, cudaStream_t s, cudaGraphConditionalHandle handle,
                  int in_graph) {
  const Level& L0 = *h.levels[0];
  const int64_t n = L0.n;
  double* scal = ws.scal.get();
  double* tmp = bs.tmp.get();
  LevelVecs<T>& V = mvecs<T>(ws)[0];
  T* d0 = nullptr;
  const T* dinv = nullptr;
  T it = T(0);
  if (L0.kind == LG_LEVEL_AGG) {
    d0 = V.dA.get();
    dinv = L0.op<T>().dinv;
    it = (T)h.cheb[0].inv_theta;
  }
  k_m_cycle_in<T><<<bblocks(n * KP), kBT, 0, s>>>(n, KP, ws.r.get(), V.f.get(), d0, dinv, it);
  LG_LAUNCH_CHECK();
  mcycle<T>(h, ws, bs, 0, KP, s);
  const T* z = V.x.get();
  k_m_z_reduce<T, KP><<<kRG, kBT, 0, s>>>(n, k, z, ws.r.get(), ws.ro.get(), scal, bs.partials.get(),
                                          bs.tickets.get(), tmp);
  LG_LAUNCH_CHECK();
  k_m_p_update<T, KP><<<bblocks(n * KP), kBT, 0, s>>>(n, k, z, ws.p.get(), scal);
  LG_LAUNCH_CHECK();
  const OpView<double> op = L0.op<double>();
  launch_mrows<double>(KP, op.col, mlap<double>(op, ws.p.get(), KP), bs.op_plan(0), MEpiStore{ws.q.get(), KP}, s);
  k_m_pq<KP><<<kRG, kBT, 0, s>>>(n, k, ws.p.get(), ws.q.get(), scal, bs.partials.get(), bs.tickets.get(), tmp);
  LG_LAUNCH_CHECK();
  k_m_xr<KP><<<kRG, kBT, 0, s>>>(n, k, ws.x.get(), ws.r.get(), ws.ro.get(), ws.p.get(), ws.q.get(), scal,
                                 bs.partials.get(), bs.tickets.get(), tmp, handle, in_graph);
  LG_LAUNCH_CHECK();
  mtrue_res<KP>(h, ws, bs, k, s, scal + k * kMS + gNeed, 1, handle, in_graph);
}

template <int KP>
static void mtrue_res(Hier& h, Workspace& ws, BatchState& bs, int k, cudaStream_t s, const double* gate, int loop,
                      cudaGraphConditionalHandle handle, int in_graph) {
  const Level& L0 = *h.levels[0];
  const int64_t n = L0.n;
  const OpView<double> op = L0.op<double>();
  launch_mrows<double>(KP, op.col, mlap<double>(op, ws.x.get(), KP), bs.op_plan(0),
                       MEpiTrueRes{ws.bm.get(), ws.r.get(), ws.scal.get(), k, KP, loop ? 0 : 1}, s, gate);
  k_m_rr<KP><<<kRG, kBT, 0, s>>>(n, k, ws.r.get(), ws.scal.get(), bs.partials.get(), bs.tickets.get(), bs.tmp.get(),
                                 gate, loop, handle, in_graph);
  LG_LAUNCH_CHECK();
}

static BatchState& batch_state(Hier& h, Workspace& ws, int kp, cudaStream_t s);

// The whole multi-column loop as one graph: a WHILE node whose body is one
// iteration, captured once per workspace, precision and width.
template <typename T, int KP>
static cudaGraphExec_t mgraph(Hier& h, Workspace& ws, BatchState& bs, int k, cudaStream_t s) {
  const auto key = std::make_pair(sizeof(T) == 4 ? 1 : 0, k);
  auto found = bs.graphs.find(key);
  if (found != bs.graphs.end()) return found->second;
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
    mbody<T, KP>(h, ws, bs, k, s, handle, 1);
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
  bs.graphs[key] = exec;
  return exec;
}

// B: device [n][KP] in the caller's numbering (columns past k zero); the
// result lands in ws.io, [n][KP] in the caller's numbering.
template <typename T, int KP>
static int msolve(Hier& h, Workspace& ws, int k, const double* B, double tol, cudaStream_t s, lg_info* infos) {
  const Level& L0 = *h.levels[0];
  const int64_t n = L0.n;
  BatchState& bs = batch_state(h, ws, KP, s);
  double* scal = ws.scal.get();
  double* tmp = bs.tmp.get();
  double* colsum = bs.colsum.get();
  const int maxit = h.opts.max_iter;
  const int every = h.opts.residual_replace > 0 ? h.opts.residual_replace : 1 << 30;
  cudaEvent_t e0, e1;
  LG_CUDA(cudaEventCreate(&e0));
  LG_CUDA(cudaEventCreate(&e1));
  struct EvGuard {
    cudaEvent_t a, b;
    ~EvGuard() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } guard{e0, e1};
  LG_CUDA(cudaEventRecord(e0, s));
  k_m_colsum<KP><<<kRG, kBT, 0, s>>>(n, B, bs.partials.get(), bs.tickets.get(), colsum);
  LG_LAUNCH_CHECK();
  k_m_init<KP><<<kRG, kBT, 0, s>>>(n, k, B, h.perm.get(), colsum, ws.bm.get(), ws.x.get(), ws.r.get(), ws.p.get(),
                                   scal, bs.partials.get(), bs.tickets.get(), tmp, tol, maxit, every);
  LG_LAUNCH_CHECK();
  const size_t nscal = (size_t)k * kMS + kMG;
  std::vector<double> hs(nscal);
  auto read = [&]() {
    LG_CUDA(cudaMemcpyAsync(hs.data(), scal, sizeof(double) * nscal, cudaMemcpyDeviceToHost, s));
    LG_CUDA(cudaStreamSynchronize(s));
  };
  auto any_active = [&]() {
    for (int c = 0; c < k; ++c)
      if (hs[c * kMS + mActive] != 0.0) return true;
    return false;
  };
  read();
  if (any_active() && maxit > 0) {
    if (h.opts.use_graphs && !debug_sync()) {
      LG_CUDA(cudaGraphLaunch(mgraph<T, KP>(h, ws, bs, k, s), s));
      read();
    } else {
      for (;;) {
        mbody<T, KP>(h, ws, bs, k, s, cudaGraphConditionalHandle{}, 0);
        read();
        if (!any_active() || hs[k * kMS + gIter] >= maxit) break;
      }
    }
  }
  const int it = (int)hs[k * kMS + gIter];
  // results in the caller's numbering, mean removed
  k_m_colsum<KP><<<kRG, kBT, 0, s>>>(n, ws.x.get(), bs.partials.get(), bs.tickets.get(), colsum);
  LG_LAUNCH_CHECK();
  bool all_done = true;
  for (int c = 0; c < k; ++c)
    if (hs[c * kMS + mDone] == 0.0 && hs[c * kMS + mBB] != 0.0) all_done = false;
  if (!all_done) {
    mtrue_res<KP>(h, ws, bs, k, s, nullptr, 0, cudaGraphConditionalHandle{}, 0);
    read();
  }
  k_m_out<KP><<<bblocks(n * KP), kBT, 0, s>>>(n, ws.x.get(), h.perm.get(), colsum, ws.io.get());
  LG_LAUNCH_CHECK();
  LG_CUDA(cudaEventRecord(e1, s));
  LG_CUDA(cudaStreamSynchronize(s));
  float ms = 0.f;
  LG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  int worst = LG_OK;
  for (int c = 0; c < k; ++c) {
    const double* sc = &hs[c * kMS];
    const int st = sc[mBB] == 0.0 || sc[mDone] != 0.0 ? LG_OK : sc[mBreak] != 0.0 ? LG_ERR_BREAKDOWN
                                                                                   : LG_ERR_NOT_CONVERGED;
    if (st != LG_OK && worst == LG_OK) worst = st;
    if (infos) {
      lg_info& inf = infos[c];
      inf = lg_info{};
      inf.status = st;
      inf.iterations = sc[mBB] == 0.0 ? 0 : (sc[mDone] != 0.0 ? (int)sc[mConv] : it);
      inf.relres = sc[mBB] > 0.0 ? std::sqrt(sc[mRR] / sc[mBB]) : 0.0;
      inf.solve_ms = ms;
      inf.work_units = inf.iterations * iteration_work(h);
      inf.levels = (int)h.levels.size();
      inf.setup_ms = h.setup_ms;
      inf.nnz = h.nnz0;
    }
  }
  return worst;
}

// ---------------------------------------------------------------------------
// The virtual row length of each level, chosen by timing: one SpMM pass of
// the level's operator (and of W) at the width of the first batch for each
// candidate, the fastest kept. Cached per (rows, entries) for the life of the
// process, so every batch on a hierarchy (and every hierarchy of that shape)
// uses the same plan. Option autotune = 0 keeps 256.
// ---------------------------------------------------------------------------
constexpr int kChDefault = 256;
static std::mutex g_mtune_mu;
static std::map<std::tuple<int64_t, int64_t, int>, int> g_mtune;

template <typename T>
struct MEpiNull {
  T* y;
  int ld;
  __device__ __forceinline__ void operator()(int64_t i, int c, T s) const { y[i * ld + c] = s; }
};

template <typename T>
static float time_mpass(const Level& L, bool w_op, const MPlan& p, int kp, const T* x, T* y, cudaStream_t s,
                        cudaEvent_t e0, cudaEvent_t e1) {
  float best = 0.f;
  for (int rep = 0; rep < 3; ++rep) {
    LG_CUDA(cudaEventRecord(e0, s));
    if (w_op) {
      const OpView<T> lp = L.lp<T>();
      launch_mrows<T>(kp, lp.col, mlp_term<T>(lp, x, L.agg.get(), kp), p, MEpiNull<T>{y, kp}, s);
    } else {
      const OpView<T> op = L.op<T>();
      launch_mrows<T>(kp, op.col, mlap<T>(op, x, kp), p, MEpiNull<T>{y, kp}, s);
    }
    LG_CUDA(cudaEventRecord(e1, s));
    LG_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    LG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (rep == 0 || ms < best) best = ms;
  }
  return best;
}

static int tune_ch(const Level& L, bool w_op, int kp, bool fp32, cudaStream_t s) {
  const int64_t rows = L.n, entries = w_op ? L.lp_nnz : L.nnz;
  const int64_t xlen = w_op ? L.nc : L.n;
  const auto key = std::make_tuple(rows, entries, w_op ? 1 : 0);
  {
    std::lock_guard<std::mutex> lk(g_mtune_mu);
    auto it = g_mtune.find(key);
    if (it != g_mtune.end()) return it->second;
  }
  int best = kChDefault;
  if (entries >= (int64_t(1) << 22)) {  // smaller levels are launch-bound: any length serves
    const int64_t* rowptr = w_op ? L.lp_ptr.get() : L.rowptr.get();
    const size_t tb = fp32 ? 4 : 8;
    DBuf<unsigned char> xb((size_t)xlen * kp * tb, s), yb((size_t)rows * kp * tb, s);
    LG_CUDA(cudaMemsetAsync(xb.get(), 0, (size_t)xlen * kp * tb, s));
    cudaEvent_t e0, e1;
    LG_CUDA(cudaEventCreate(&e0));
    LG_CUDA(cudaEventCreate(&e1));
    float best_ms = 0.f;
    for (int ch : {64, 256, 1024}) {
      MPlanStore ps;
      ps.build(rows, rowptr, ch, s, nullptr);
      PlanScratchM sc;
      sc.make(ps.plan, s, nullptr);
      const MPlan p = sc.bind(ps.plan);
      const float ms = fp32 ? time_mpass<float>(L, w_op, p, kp, reinterpret_cast<const float*>(xb.get()),
                                                reinterpret_cast<float*>(yb.get()), s, e0, e1)
                            : time_mpass<double>(L, w_op, p, kp, reinterpret_cast<const double*>(xb.get()),
                                                 reinterpret_cast<double*>(yb.get()), s, e0, e1);
      if (ch == 64 || ms < best_ms) {
        best = ch;
        best_ms = ms;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  std::lock_guard<std::mutex> lk(g_mtune_mu);
  return g_mtune.emplace(key, best).first->second;
}

static std::mutex g_plans_mu;

// Built (and tuned) on the handle's own stream, whose life bounds theirs: a
// solve on another stream (a server slot's) may come first.
static const HierPlans* hier_plans(Hier& h, int kp, bool fp32) {
  std::lock_guard<std::mutex> lk(g_plans_mu);
  if (h.mplans) return static_cast<const HierPlans*>(h.mplans.get());
  cudaStream_t s = h.stream;
  auto hp = std::make_shared<HierPlans>();
  const size_t nl = h.levels.size();
  hp->op.resize(nl);
  hp->mem.resize(nl);
  hp->pt.resize(nl);
  hp->lp.resize(nl);
  for (size_t l = 0; l < nl; ++l) {
    const Level& L = *h.levels[l];
    const bool tune = h.opts.autotune && L.kind != LG_LEVEL_COARSEST;
    hp->op[l] = std::make_unique<MPlanStore>();
    // an elimination level below the finest applies no operator pass: an empty plan
    if (L.kind == LG_LEVEL_AGG || l == 0)
      hp->op[l]->build(L.n, L.rowptr.get(), tune ? tune_ch(L, false, kp, fp32, s) : kChDefault, s, &h.bytes);
    if (L.kind == LG_LEVEL_AGG) {
      hp->mem[l] = std::make_unique<MPlanStore>();
      hp->mem[l]->build(L.nc, L.mem_ptr.get(), kChDefault, s, &h.bytes);
    }
    if (L.kind == LG_LEVEL_ELIM) {
      hp->pt[l] = std::make_unique<MPlanStore>();
      hp->pt[l]->build(L.nc, L.pt_ptr.get(), kChDefault, s, &h.bytes);
    }
    if (L.lp_nnz > 0) {
      hp->lp[l] = std::make_unique<MPlanStore>();
      hp->lp[l]->build(L.n, L.lp_ptr.get(), tune ? tune_ch(L, true, kp, fp32, s) : kChDefault, s, &h.bytes);
    }
  }
  LG_CUDA(cudaStreamSynchronize(s));
  h.mplans = hp;
  return hp.get();
}

// The state lives in the workspace's memory: allocated (and later freed) on
// the stream the workspace was made on, which a solve on another stream
// waits for.
static BatchState& batch_state(Hier& h, Workspace& ws, int kp, cudaStream_t run) {
  if (!ws.batch) {
    cudaStream_t s = ws.alloc_stream ? ws.alloc_stream : run;
    auto st = std::make_shared<BatchState>();
    st->plans = hier_plans(h, kp, h.opts.precision == LG_FP32_HIER);
    const size_t nl = h.levels.size();
    st->op.resize(nl);
    st->mem.resize(nl);
    st->pt.resize(nl);
    st->lp.resize(nl);
    for (size_t l = 0; l < nl; ++l) {
      st->op[l].make(st->plans->op[l]->plan, s, &ws.bytes);
      if (st->plans->mem[l]) st->mem[l].make(st->plans->mem[l]->plan, s, &ws.bytes);
      if (st->plans->pt[l]) st->pt[l].make(st->plans->pt[l]->plan, s, &ws.bytes);
      if (st->plans->lp[l]) st->lp[l].make(st->plans->lp[l]->plan, s, &ws.bytes);
    }
    st->tmp.alloc(5 * kMaxCols, s, &ws.bytes);
    st->colsum.alloc(kMaxCols, s, &ws.bytes);
    st->partials.alloc((size_t)kRG * 5 * kMaxCols, s, &ws.bytes);
    st->tickets.alloc(1, s, &ws.bytes);
    LG_CUDA(cudaMemsetAsync(st->tickets.get(), 0, sizeof(unsigned), s));
    if (s != run) LG_CUDA(cudaStreamSynchronize(s));
    ws.batch = st;
  }
  return *static_cast<BatchState*>(ws.batch.get());
}

// Column-major (ld = n, k columns) <-> row-major [n][KP] (padding columns zero).
__global__ void k_cm_to_rm(int64_t n, int k, int kp, const double* __restrict__ cm, double* __restrict__ rm) {
  LG_GRID_STRIDE(e, n * kp) {
    const int64_t i = e / kp;
    const int c = (int)(e - i * kp);
    rm[e] = c < k ? cm[(int64_t)c * n + i] : 0.0;
  }
}

__global__ void k_rm_to_cm(int64_t n, int k, int kp, const double* __restrict__ rm, double* __restrict__ cm) {
  LG_GRID_STRIDE(e, n * k) {
    const int64_t c = e / n, i = e - c * n;
    cm[e] = rm[i * kp + c];
  }
}

}  // namespace

// B, X: device, column-major n x k with leading dimension n. Every width runs
// the multi-column path, k = 1 included (its result is then the same as in
// any batch).
int pcg_solve_columns(Hier& h, Workspace& ws, int k, const double* B, double* X, double tol, int precision,
                      cudaStream_t s, lg_info* infos) {
  const int kp = pow2_at_least(k);
  if (ws.k < kp) fail(LG_ERR_INVALID, "workspace narrower than the batch");
  if (precision == LG_FP64 && h.fp32_only) fail(LG_ERR_INVALID, "an fp32_only hierarchy serves FP32 solves only");
  const int64_t n = h.levels[0]->n;
  if (h.opts.kcycle) {  // the SpMM cycle is the V-cycle: K-cycle columns run one at a time
    int worst = LG_OK;
    for (int c = 0; c < k; ++c) {
      const int st = pcg_solve(h, ws, B + (size_t)c * n, X + (size_t)c * n, tol, precision, s,
                               infos ? infos + c : nullptr);
      if (st != LG_OK && worst == LG_OK) worst = st;
    }
    return worst;
  }
  const bool f32 = precision == LG_FP32_HIER;
  k_cm_to_rm<<<bblocks(n * kp), kBT, 0, s>>>(n, k, kp, B, ws.z.get());
  LG_LAUNCH_CHECK();
  // The solve runs all kp columns: the padding columns have b = 0, so they
  // are inactive from the start and change nothing in the others; one
  // captured loop then serves every k of a width.
  int st = LG_OK;
  std::vector<lg_info> all((size_t)kp);
#define LG_MS_CASE(KK)                                                             \
  case KK:                                                                         \
    st = f32 ? msolve<float, KK>(h, ws, KK, ws.z.get(), tol, s, all.data())        \
             : msolve<double, KK>(h, ws, KK, ws.z.get(), tol, s, all.data());      \
    break;
  switch (kp) {
    LG_MS_CASE(1)
    LG_MS_CASE(2)
    LG_MS_CASE(4)
    LG_MS_CASE(8)
    LG_MS_CASE(16)
    LG_MS_CASE(32)
    default:
      fail(LG_ERR_INVALID, "batch width");
  }
#undef LG_MS_CASE
  k_rm_to_cm<<<bblocks(n * k), kBT, 0, s>>>(n, k, kp, ws.io.get(), X);
  LG_LAUNCH_CHECK();
  LG_CUDA(cudaStreamSynchronize(s));
  if (infos)
    for (int c = 0; c < k; ++c) infos[c] = all[c];
  return st;
}

void prepare_columns(Hier& h, int kp, int precision) { hier_plans(h, kp, precision == LG_FP32_HIER); }

void prepare_column_graphs(Hier& h, Workspace& ws, int precision, cudaStream_t s) {
  if (!h.opts.use_graphs || debug_sync() || h.opts.kcycle) return;
  const bool f32 = precision == LG_FP32_HIER;
  for (int kp = 1; kp <= ws.k && kp <= kMaxCols; kp <<= 1) {
    BatchState& bs = batch_state(h, ws, kp, s);
#define LG_PG_CASE(KK)                                                        \
  case KK:                                                                    \
    if (f32) mgraph<float, KK>(h, ws, bs, KK, s); else mgraph<double, KK>(h, ws, bs, KK, s); \
    break;
    switch (kp) {
      LG_PG_CASE(1)
      LG_PG_CASE(2)
      LG_PG_CASE(4)
      LG_PG_CASE(8)
      LG_PG_CASE(16)
      LG_PG_CASE(32)
      default: break;
    }
#undef LG_PG_CASE
  }
}

int pcg_solve_batch(Hier& h, Workspace& ws, int k, const double* B, double* X, double tol, int precision,
                    cudaStream_t s, lg_info* infos) {
  if (k == 1) return pcg_solve(h, ws, B, X, tol, precision, s, infos);
  return pcg_solve_columns(h, ws, k, B, X, tol, precision, s, infos);
}

namespace {

// x = M f for k columns (F, X device, column-major, leading dimension n, in
// the caller's numbering), starting from x = 0: the multi-column cycle alone.
__global__ void k_m_gather_perm(int64_t n, int kp, const int32_t* __restrict__ perm, const double* __restrict__ src,
                                double* __restrict__ dst) {
  LG_GRID_STRIDE(e, n * kp) {
    const int64_t i = e / kp;
    dst[e] = src[(int64_t)perm[i] * kp + (e - i * kp)];
  }
}

template <typename T>
__global__ void k_m_scatter_out(int64_t n, int kp, const int32_t* __restrict__ perm, const T* __restrict__ src,
                                double* __restrict__ dst) {
  LG_GRID_STRIDE(e, n * kp) {
    const int64_t i = e / kp;
    dst[(int64_t)perm[i] * kp + (e - i * kp)] = (double)src[e];
  }
}

template <typename T>
static void mcycle_apply(Hier& h, Workspace& ws, int k, const double* F, double* X, cudaStream_t s) {
  const Level& L0 = *h.levels[0];
  const int64_t n = L0.n;
  const int kp = pow2_at_least(k);
  BatchState& bs = batch_state(h, ws, kp, s);
  k_cm_to_rm<<<bblocks(n * kp), kBT, 0, s>>>(n, k, kp, F, ws.z.get());
  LG_LAUNCH_CHECK();
  k_m_gather_perm<<<bblocks(n * kp), kBT, 0, s>>>(n, kp, h.perm.get(), ws.z.get(), ws.r.get());
  LG_LAUNCH_CHECK();
  LevelVecs<T>& V = mvecs<T>(ws)[0];
  T* d0 = nullptr;
  const T* dinv = nullptr;
  T it = T(0);
  if (L0.kind == LG_LEVEL_AGG) {
    d0 = V.dA.get();
    dinv = L0.op<T>().dinv;
    it = (T)h.cheb[0].inv_theta;
  }
  k_m_cycle_in<T><<<bblocks(n * kp), kBT, 0, s>>>(n, kp, ws.r.get(), V.f.get(), d0, dinv, it);
  LG_LAUNCH_CHECK();
  mcycle<T>(h, ws, bs, 0, kp, s);
  k_m_scatter_out<T><<<bblocks(n * kp), kBT, 0, s>>>(n, kp, h.perm.get(), V.x.get(), ws.io.get());
  LG_LAUNCH_CHECK();
  k_rm_to_cm<<<bblocks(n * k), kBT, 0, s>>>(n, k, kp, ws.io.get(), X);
  LG_LAUNCH_CHECK();
}

}  // namespace

void vcycle_apply_batch(Hier& h, Workspace& ws, int k, const double* F, double* X, int precision, cudaStream_t s) {
  if (ws.k < pow2_at_least(k)) fail(LG_ERR_INVALID, "workspace narrower than the batch");
  if (h.opts.kcycle) {  // the SpMM cycle is the V-cycle: K-cycle columns one at a time
    const int64_t n = h.levels[0]->n;
    for (int c = 0; c < k; ++c) vcycle_apply(h, ws, F + (size_t)c * n, X + (size_t)c * n, precision, s);
    return;
  }
  if (precision == LG_FP32_HIER) mcycle_apply<float>(h, ws, k, F, X, s);
  else mcycle_apply<double>(h, ws, k, F, X, s);
}

// The multi-column schedule of level l, once built: the stretch length and
// the virtual rows of its operator plan and of its W plan (0 where none).
bool batch_plan_info(const Hier& h, int level, int64_t out[4]) {
  std::lock_guard<std::mutex> lk(g_plans_mu);
  const auto* hp = static_cast<const HierPlans*>(h.mplans.get());
  if (!hp || level < 0 || level >= (int)hp->op.size()) return false;
  const MPlanStore* op = hp->op[level].get();
  const MPlanStore* lp = hp->lp[level].get();
  out[0] = op && op->plan.nv ? op->plan.ch : 0;
  out[1] = op ? op->plan.nv : 0;
  out[2] = lp && lp->plan.nv ? lp->plan.ch : 0;
  out[3] = lp ? lp->plan.nv : 0;
  return true;
}

}  // namespace lg
