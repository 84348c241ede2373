// Multi-right-hand-side solve: the V-cycle and the FP64 outer CG on k
// columns at once (k <= 32), vectors stored row-major [n][k] so that the k
// values of one vertex are contiguous.
//
// Every SpMV of the cycle becomes an SpMM pass over the lanes of a warp split
// into S = 32 / KP entry slices of KP column lanes (KP = k rounded up to a
// power of two); each lane of a slice accumulates one column, so the k values
// gathered for an entry are one coalesced access and every matrix entry is
// read once for all columns. Rows of at most kShortM entries take one slice
// each (S rows per warp); longer rows take a warp, its slices walking every
// S-th entry; rows longer than kChunkM entries are cut into chunks, one block
// each, combined by the last block of the row in chunk order. The CG scalars
// are per column; a column that has converged keeps its iterate (alpha = 0)
// while the others go on.
#include <algorithm>
#include <cmath>
#include <map>

#include "lg_hier.h"
#include "lg_rows.cuh"

namespace lg {

constexpr int kBT = 256;
constexpr int kChunkM = 256;

#define LG_GRID_STRIDE(i, n) \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

static inline int bblocks(int64_t n) { return grid_for(n, kBT, kSMs * 8); }

static int pow2_at_least(int k) {
  int p = 1;
  while (p < k) p <<= 1;
  return p;
}

// ---------------------------------------------------------------------------
// Plans of the SpMM passes: rows longer than kChunkM entries in chunks.
// ---------------------------------------------------------------------------
constexpr int kShortM = 16;  // rows of at most this many entries take one entry slice each

struct MPlan {
  int64_t nshort = 0, nmed = 0;
  const int32_t* short_rows = nullptr;  // rows of <= kShortM entries, ascending
  const int32_t* med_rows = nullptr;    // rows of kShortM+1 .. kChunkM entries, ascending
  int64_t nchunks = 0;
  const int32_t* chunk_row = nullptr;
  const int64_t* chunk_beg = nullptr;
  const int32_t* chunk_lrow = nullptr;
  const int32_t* lrow_first = nullptr;
  const int32_t* lrow_count = nullptr;
  double* partial = nullptr;  // nchunks * kMaxCols
  unsigned* ticket = nullptr;
};

__global__ void k_mplan_count(int64_t n, const int64_t* __restrict__ rowptr, int64_t* __restrict__ nch,
                              uint8_t* __restrict__ islong, uint8_t* __restrict__ isshort,
                              uint8_t* __restrict__ ismed) {
  LG_GRID_STRIDE(i, n) {
    const int64_t deg = rowptr[i + 1] - rowptr[i];
    islong[i] = deg > kChunkM;
    isshort[i] = deg <= kShortM;
    ismed[i] = deg > kShortM && deg <= kChunkM;
    nch[i] = deg > kChunkM ? (deg + kChunkM - 1) / kChunkM : 0;
  }
}

__global__ void k_mplan_list(int64_t n, const uint8_t* __restrict__ flag, const int64_t* __restrict__ pos,
                             int32_t* __restrict__ list) {
  LG_GRID_STRIDE(i, n) if (flag[i]) list[pos[i]] = (int32_t)i;
}

__global__ void k_mplan_fill(int64_t n, const int64_t* __restrict__ rowptr, const uint8_t* __restrict__ islong,
                             const int64_t* __restrict__ cstart, const int64_t* __restrict__ lidx, int32_t* chunk_row,
                             int64_t* chunk_beg, int32_t* chunk_lrow, int32_t* lrow_first, int32_t* lrow_count) {
  LG_GRID_STRIDE(i, n) {
    if (!islong[i]) continue;
    const int64_t lr = lidx[i], c0 = cstart[i], cnt = cstart[i + 1] - cstart[i];
    lrow_first[lr] = (int32_t)c0;
    lrow_count[lr] = (int32_t)cnt;
    for (int64_t q = 0; q < cnt; ++q) {
      chunk_row[c0 + q] = (int32_t)i;
      chunk_beg[c0 + q] = rowptr[i] + q * kChunkM;
      chunk_lrow[c0 + q] = (int32_t)lr;
    }
  }
}

struct MPlanStore {
  MPlan plan;
  DBuf<int32_t> short_rows, med_rows;
  DBuf<int32_t> chunk_row, chunk_lrow, lrow_first, lrow_count;
  DBuf<int64_t> chunk_beg;
  DBuf<double> partial;
  DBuf<unsigned> ticket;
  void build(int64_t n, const int64_t* rowptr, cudaStream_t s, int64_t* counter) {
    DBuf<int64_t> nch(n + 1, s), lidx(n + 1, s), sidx(n + 1, s), midx(n + 1, s);
    DBuf<uint8_t> islong(n, s), isshort(n, s), ismed(n, s);
    const int g = grid_for(n, 256, kSMs * 16);
    if (n > 0) {
      k_mplan_count<<<g, 256, 0, s>>>(n, rowptr, nch.get(), islong.get(), isshort.get(), ismed.get());
      LG_LAUNCH_CHECK();
    }
    exclusive_scan(nch.get(), nch.get(), n, s);
    exclusive_scan_flags(islong.get(), lidx.get(), n, s);
    exclusive_scan_flags(isshort.get(), sidx.get(), n, s);
    exclusive_scan_flags(ismed.get(), midx.get(), n, s);
    int64_t tot[4];
    LG_CUDA(cudaMemcpyAsync(&tot[0], nch.get() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    LG_CUDA(cudaMemcpyAsync(&tot[1], lidx.get() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    LG_CUDA(cudaMemcpyAsync(&tot[2], sidx.get() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    LG_CUDA(cudaMemcpyAsync(&tot[3], midx.get() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    LG_CUDA(cudaStreamSynchronize(s));
    plan.nshort = tot[2];
    plan.nmed = tot[3];
    short_rows.alloc(plan.nshort > 0 ? plan.nshort : 1, s, counter);
    med_rows.alloc(plan.nmed > 0 ? plan.nmed : 1, s, counter);
    if (n > 0) {
      k_mplan_list<<<g, 256, 0, s>>>(n, isshort.get(), sidx.get(), short_rows.get());
      LG_LAUNCH_CHECK();
      k_mplan_list<<<g, 256, 0, s>>>(n, ismed.get(), midx.get(), med_rows.get());
      LG_LAUNCH_CHECK();
    }
    plan.short_rows = short_rows.get();
    plan.med_rows = med_rows.get();
    plan.nchunks = tot[0];
    const int64_t nlong = tot[1];
    chunk_row.alloc(plan.nchunks, s, counter);
    chunk_beg.alloc(plan.nchunks, s, counter);
    chunk_lrow.alloc(plan.nchunks, s, counter);
    lrow_first.alloc(nlong, s, counter);
    lrow_count.alloc(nlong, s, counter);
    partial.alloc((size_t)(plan.nchunks > 0 ? plan.nchunks : 1) * kMaxCols, s, counter);
    ticket.alloc(nlong > 0 ? nlong : 1, s, counter);
    LG_CUDA(cudaMemsetAsync(ticket.get(), 0, sizeof(unsigned) * (nlong > 0 ? nlong : 1), s));
    if (nlong > 0) {
      k_mplan_fill<<<g, 256, 0, s>>>(n, rowptr, islong.get(), nch.get(), lidx.get(), chunk_row.get(),
                                     chunk_beg.get(), chunk_lrow.get(), lrow_first.get(), lrow_count.get());
      LG_LAUNCH_CHECK();
    }
    plan.chunk_row = chunk_row.get();
    plan.chunk_beg = chunk_beg.get();
    plan.chunk_lrow = chunk_lrow.get();
    plan.lrow_first = lrow_first.get();
    plan.lrow_count = lrow_count.get();
    plan.partial = partial.get();
    plan.ticket = ticket.get();
  }
};

// ---------------------------------------------------------------------------
// Terms over one column c of [n][k] vectors.
// ---------------------------------------------------------------------------
template <typename T>
struct MLap;

template <>
struct MLap<float> {  // difference form, as the single-vector FP32 pass
  const float* __restrict__ w;
  const float* __restrict__ x;
  const double* __restrict__ d;
  int k;
  __device__ __forceinline__ float row(int64_t i, int c) const { return x[i * k + c]; }
  __device__ __forceinline__ float acc(float s, int64_t e, int32_t j, int c, float xi) const {
    return fmaf(w[e], xi - __ldg(&x[(int64_t)j * k + c]), s);
  }
  __device__ __forceinline__ float finish(int64_t, int, float, float s) const { return s; }
};

template <>
struct MLap<double> {  // d_i x_i - sum_j w_ij x_j, as the single-vector FP64 pass
  const double* __restrict__ w;
  const double* __restrict__ x;
  const double* __restrict__ d;
  int k;
  __device__ __forceinline__ double row(int64_t, int) const { return 0.0; }
  __device__ __forceinline__ double acc(double s, int64_t e, int32_t j, int c, double) const {
    return fma(w[e], __ldg(&x[(int64_t)j * k + c]), s);
  }
  __device__ __forceinline__ double finish(int64_t i, int c, double, double s) const {
    return fma(d[i], x[i * k + c], -s);
  }
};

template <typename T>
struct MGather {  // restriction by member lists: sum v[j][c]
  const T* __restrict__ v;
  int k;
  __device__ __forceinline__ T row(int64_t, int) const { return T(0); }
  __device__ __forceinline__ T acc(T s, int64_t, int32_t j, int c, T) const { return s + __ldg(&v[(int64_t)j * k + c]); }
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
  int k;
  __device__ __forceinline__ float row(int64_t i, int c) const { return __ldg(&xc[(int64_t)agg[i] * k + c]); }
  __device__ __forceinline__ float acc(float s, int64_t e, int32_t a, int c, float xa) const {
    return fmaf(w[e], xa - __ldg(&xc[(int64_t)a * k + c]), s);
  }
  __device__ __forceinline__ float finish(int64_t, int, float, float s) const { return s; }
};

template <>
struct MLp<double> {
  const double* __restrict__ w;
  const double* __restrict__ xc;
  const int32_t* __restrict__ agg;
  const double* __restrict__ d;
  int k;
  __device__ __forceinline__ double row(int64_t, int) const { return 0.0; }
  __device__ __forceinline__ double acc(double s, int64_t e, int32_t a, int c, double) const {
    return fma(w[e], __ldg(&xc[(int64_t)a * k + c]), s);
  }
  __device__ __forceinline__ double finish(int64_t i, int c, double, double s) const {
    return fma(d[i], __ldg(&xc[(int64_t)agg[i] * k + c]), -s);
  }
};

template <typename T>
struct MWGather {  // elimination restriction: sum coef_e v[j][c]
  const T* __restrict__ coef;
  const T* __restrict__ v;
  int k;
  __device__ __forceinline__ T row(int64_t, int) const { return T(0); }
  __device__ __forceinline__ T acc(T s, int64_t e, int32_t j, int c, T) const {
    return fma(coef[e], __ldg(&v[(int64_t)j * k + c]), s);
  }
  __device__ __forceinline__ T finish(int64_t, int, T, T s) const { return s; }
};

// ---------------------------------------------------------------------------
// The SpMM pass: warp per row (S slices x KP column lanes), chunks for long rows.
// ---------------------------------------------------------------------------
template <typename T, int KP, class Term, class Epi>
__global__ void __launch_bounds__(kBT)
k_mrows(int64_t n, int k, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, Term term, MPlan plan,
        Epi epi, const double* gate) {
  if (gate && *gate == 0.0) return;  // a pass gated off does nothing (every block reads the same flag)
  constexpr int S = 32 / KP;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = lane & (KP - 1), slice = lane / KP;
  const bool active = c < k;
  const int cc = active ? c : 0;
  const int64_t bid = blockIdx.x;
  if (bid < plan.nchunks) {
    __shared__ T sred[kBT / 32][KP];
    const int64_t row = plan.chunk_row[bid];
    const int64_t beg = plan.chunk_beg[bid];
    const int64_t rend = rowptr[row + 1];
    const int64_t end = beg + kChunkM < rend ? beg + kChunkM : rend;
    const T rv = term.row(row, cc);
    T s = T(0);
    const int sl = warp * S + slice;  // slice among the block's 8 S slices
    for (int64_t e = beg + sl; e < end; e += (kBT / 32) * S) s = term.acc(s, e, col[e], cc, rv);
#pragma unroll
    for (int o = KP; o < 32; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (slice == 0) sred[warp][c] = s;
    __syncthreads();
    if (threadIdx.x < KP) {
      T t = T(0);
      for (int w = 0; w < kBT / 32; ++w) t += sred[w][threadIdx.x];
      plan.partial[bid * kMaxCols + threadIdx.x] = (double)t;
      __threadfence();  // each column's partial is visible before the ticket is taken
    }
    __syncthreads();
    __shared__ bool last;
    if (threadIdx.x == 0) {
      const int32_t lr = plan.chunk_lrow[bid];
      __threadfence();
      const unsigned tk = atomicAdd((unsigned*)&plan.ticket[lr], 1u);
      last = tk == (unsigned)plan.lrow_count[lr] - 1u;
      if (last) plan.ticket[lr] = 0u;
    }
    __syncthreads();
    if (last && threadIdx.x < KP && threadIdx.x < k) {
      __threadfence();
      const int32_t lr = plan.chunk_lrow[bid];
      const int32_t f0 = plan.lrow_first[lr], cnt = plan.lrow_count[lr];
      T tot = T(0);
      for (int32_t q = 0; q < cnt; ++q) tot += (T)__ldcg(&plan.partial[(int64_t)(f0 + q) * kMaxCols + threadIdx.x]);
      epi(row, (int)threadIdx.x, term.finish(row, (int)threadIdx.x, term.row(row, (int)threadIdx.x), tot));
    }
    return;
  }
  const int64_t nshort_blk = (plan.nshort + (kBT / 32) * S - 1) / ((kBT / 32) * S);
  if (bid < plan.nchunks + nshort_blk) {
    // short rows: one entry slice (KP column lanes) per row, S rows per warp
    const int64_t idx = ((bid - plan.nchunks) * (kBT / 32) + warp) * S + slice;
    if (idx >= plan.nshort) return;
    const int64_t row = plan.short_rows[idx];
    const int64_t beg = rowptr[row], end = rowptr[row + 1];
    const T rv = term.row(row, cc);
    T s = T(0);
    for (int64_t e = beg; e < end; ++e) s = term.acc(s, e, col[e], cc, rv);
    if (active) epi(row, c, term.finish(row, c, rv, s));
    return;
  }
  // medium rows: one warp per row, the S slices splitting its entries
  const int64_t midx = (bid - plan.nchunks - nshort_blk) * (kBT / 32) + warp;
  if (midx >= plan.nmed) return;
  const int64_t row = plan.med_rows[midx];
  const int64_t beg = rowptr[row], end = rowptr[row + 1];
  const T rv = term.row(row, cc);
  T s0 = T(0), s1 = T(0);
  int64_t e = beg + slice;
  for (; e + S < end; e += 2 * S) {
    const int32_t j0 = col[e], j1 = col[e + S];
    s0 = term.acc(s0, e, j0, cc, rv);
    s1 = term.acc(s1, e + S, j1, cc, rv);
  }
  if (e < end) s0 = term.acc(s0, e, col[e], cc, rv);
  T s = s0 + s1;
#pragma unroll
  for (int o = KP; o < 32; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (slice == 0 && active) epi(row, c, term.finish(row, c, rv, s));
}

template <typename T, class Term, class Epi>
static void launch_mrows(int kp, int64_t n, int k, const int64_t* rowptr, const int32_t* col, const Term& term,
                         const MPlan& plan, const Epi& epi, cudaStream_t s, const double* gate = nullptr) {
  const int64_t S = 32 / kp;
  const int64_t grid = plan.nchunks + (plan.nshort + (kBT / 32) * S - 1) / ((kBT / 32) * S) +
                       (plan.nmed + (kBT / 32) - 1) / (kBT / 32);
  if (grid <= 0) return;
  (void)n;
  switch (kp) {
    case 2: k_mrows<T, 2><<<(unsigned)grid, kBT, 0, s>>>(n, k, rowptr, col, term, plan, epi, gate); break;
    case 4: k_mrows<T, 4><<<(unsigned)grid, kBT, 0, s>>>(n, k, rowptr, col, term, plan, epi, gate); break;
    case 8: k_mrows<T, 8><<<(unsigned)grid, kBT, 0, s>>>(n, k, rowptr, col, term, plan, epi, gate); break;
    case 16: k_mrows<T, 16><<<(unsigned)grid, kBT, 0, s>>>(n, k, rowptr, col, term, plan, epi, gate); break;
    case 32: k_mrows<T, 32><<<(unsigned)grid, kBT, 0, s>>>(n, k, rowptr, col, term, plan, epi, gate); break;
    default: fail(LG_ERR_INVALID, "column block width");
  }
  LG_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// Epilogues over (row i, column c), vectors [n][k].
// ---------------------------------------------------------------------------
template <typename T>
struct MEpiCheb {  // one Chebyshev step (see lg_cycle.cu, EpiCheb)
  const T* g;
  const T* rin;
  T* rout;
  const T* dinv;
  T* dout;
  T* x;
  int x_mode, add_d, k;
  T c1, c2;
  __device__ __forceinline__ void operator()(int64_t i, int c, T s) const {
    const int64_t e = i * k + c;
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
  int k;
  __device__ __forceinline__ void operator()(int64_t I, int c, T s) const {
    fc[I * k + c] = s;
    if (d0) d0[I * k + c] = s * dinvc[I] * inv_theta;
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
  int k;
  __device__ __forceinline__ void operator()(int64_t cr, int c, T s) const {
    const T v = f[(int64_t)cfine[cr] * k + c] + s;
    fc[cr * k + c] = v;
    if (d0) d0[cr * k + c] = v * dinvc[cr] * inv_theta;
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
  int k;
  __device__ __forceinline__ void operator()(int64_t i, int c, T s) const {
    const int64_t e = i * k + c;
    const T r0 = r[e] - s;
    r[e] = r0;
    d0[e] = inv_theta * dinv[i] * r0;
    x[e] = x[e] + xc[(int64_t)agg[i] * k + c];
  }
};

struct MEpiStore {
  double* y;
  int k;
  __device__ __forceinline__ void operator()(int64_t i, int c, double s) const { y[i * k + c] = s; }
};

struct MEpiTrueRes {
  const double* bm;
  double* r;
  int k;
  __device__ __forceinline__ void operator()(int64_t i, int c, double s) const { r[i * k + c] = bm[i * k + c] - s; }
};

// ---------------------------------------------------------------------------
// Element-wise kernels over [n][k].
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_m_elim_prolong(int64_t n, int k, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                 const T* __restrict__ w, const T* __restrict__ dinv, const int32_t* __restrict__ cmap,
                                 const T* __restrict__ f, const T* __restrict__ xc, T* __restrict__ x) {
  LG_GRID_STRIDE(e, n * k) {
    const int64_t i = e / k;
    const int c = (int)(e - i * k);
    const int32_t cm = cmap[i];
    if (cm >= 0) {
      x[e] = xc[(int64_t)cm * k + c];
    } else {
      T s = f[e];
      for (int64_t q = rowptr[i]; q < rowptr[i + 1]; ++q) s += w[q] * xc[(int64_t)cmap[col[q]] * k + c];
      x[e] = s * dinv[i];
    }
  }
}

template <typename T>
__global__ void k_m_agg_prolong(int64_t n, int k, const int32_t* __restrict__ agg, const T* __restrict__ xc,
                                T* __restrict__ x) {
  LG_GRID_STRIDE(e, n * k) {
    const int64_t i = e / k;
    x[e] += xc[(int64_t)agg[i] * k + (e - i * k)];
  }
}

template <typename T>
__global__ void k_m_axpy1(int64_t m, const T* __restrict__ d, T* __restrict__ x) {
  LG_GRID_STRIDE(e, m) x[e] += d[e];
}

// x = L_c^+ f on k columns: one warp per coarse row, lanes over columns.
template <typename T>
__global__ void k_m_coarse_apply(int64_t n, int k, const double* __restrict__ pinv, const T* __restrict__ f,
                                 T* __restrict__ x) {
  const int lane = threadIdx.x & 31;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n;
       i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    for (int c = lane; c < k; c += 32) {
      double s = 0.0;
      for (int64_t j = 0; j < n; ++j) s += pinv[i * n + j] * (double)f[j * k + c];
      x[i * k + c] = (T)s;
    }
  }
}

// Level-0 input: f = (T) r (column block), d_0 = D^-1 f / theta.
template <typename T>
__global__ void k_m_cycle_in(int64_t n, int k, const double* __restrict__ r, T* __restrict__ f, T* __restrict__ d0,
                             const T* __restrict__ dinv, T inv_theta) {
  LG_GRID_STRIDE(e, n * k) {
    const T v = (T)r[e];
    f[e] = v;
    if (d0) d0[e] = v * dinv[e / k] * inv_theta;
  }
}

// ---------------------------------------------------------------------------
// Per-column reductions. Threads are laid out as (row slot, column): thread
// t serves column t % KP of rows t / KP, t / KP + 256 / KP, ...; sums of one
// column combine across the lanes of a warp by xor shuffles, then across the
// warps of a block, then across blocks (last block, block order). NV values
// per column. Returns true in thread 0 of the last block only.
// ---------------------------------------------------------------------------
template <int KP, int NV>
__device__ __forceinline__ bool col_grid_sum(double (&v)[NV], double* partials /* gridDim * NV * KP */,
                                             unsigned* ticket, double* out /* NV * KP */) {
  __shared__ double sm[kBT / 32][NV][KP];
  __shared__ bool am_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, c = threadIdx.x & (KP - 1);
#pragma unroll
  for (int q = 0; q < NV; ++q)
#pragma unroll
    for (int o = KP; o < 32; o <<= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  if (lane < KP)
#pragma unroll
    for (int q = 0; q < NV; ++q) sm[warp][q][c] = v[q];
  __syncthreads();
  if (threadIdx.x < KP) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double t = 0.0;
      for (int w = 0; w < kBT / 32; ++w) t += sm[w][q][threadIdx.x];
      partials[((int64_t)blockIdx.x * NV + q) * KP + threadIdx.x] = t;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    am_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  // the last block adds the blocks' partials: thread t takes column t % KP and
  // blocks t / KP, t / KP + kParts, ... (kParts = kBT / KP), then the kParts
  // sums of each column are added in part order
  {
    constexpr int kParts = kBT / KP;
    __shared__ double fin[kParts][NV][KP];
    const int cc = threadIdx.x % KP, part = threadIdx.x / KP;
    double t[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) t[q] = 0.0;
    for (unsigned b = part; b < gridDim.x; b += kParts)
#pragma unroll
      for (int q = 0; q < NV; ++q) t[q] += __ldcg(&partials[((int64_t)b * NV + q) * KP + cc]);
#pragma unroll
    for (int q = 0; q < NV; ++q) fin[part][q][cc] = t[q];
    __syncthreads();
    if (threadIdx.x < KP) {
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        double u = 0.0;
        for (int pp = 0; pp < kParts; ++pp) u += fin[pp][q][threadIdx.x];
        out[q * KP + threadIdx.x] = u;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x != 0) return false;
  *ticket = 0u;
  return true;  // one thread of the last block, which alone updates the column scalars
}

#define LG_COL_STRIDE(i, n)                                                                    \
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / KP; i < (n);             \
       i += ((int64_t)gridDim.x * blockDim.x) / KP)

// Per-column scalars, column c at scal[c * kMS + field].
enum MScal : int {
  mBB = 0, mRZ, mPQ, mAlpha, mBeta, mMeanZ, mRR, mSumB, mBreak, mDone, mIter, mTol2BB, mNeedTrue, mActive, mConv,
  kMS = 16
};
// Loop scalars after the k column blocks (scal + k kMS).
enum MGlob : int { gIter = 0, gNeed, gMaxit, gEvery, kMG = 4 };

template <int KP>
__global__ void k_m_colsum(int64_t n, int k, const double* __restrict__ v, double* partials, unsigned* ticket,
                           double* out /* KP */) {
  const int c = threadIdx.x & (KP - 1);
  double acc[1] = {0.0};
  if (c < k) LG_COL_STRIDE(i, n) acc[0] += v[i * k + c];
  col_grid_sum<KP, 1>(acc, partials, ticket, out);
}

// b_m = b - mean(b) per column (b in the caller's numbering, gathered);
// x = 0; r = b_m; p = 0 (see k_pcg_init); column scalars initialised.
template <int KP>
__global__ void k_m_init(int64_t n, int k, const double* __restrict__ b, const int32_t* __restrict__ perm,
                         const double* __restrict__ colsum, double* __restrict__ bm, double* __restrict__ x,
                         double* __restrict__ r, double* __restrict__ p, double* scal, double* partials,
                         unsigned* ticket, double* tmp,
                         double tol, int maxit, int every) {
  const int c = threadIdx.x & (KP - 1);
  double acc[1] = {0.0};
  if (c < k) {
    const double mean = colsum[c] / (double)n;
    LG_COL_STRIDE(i, n) {
      const double v = b[(int64_t)perm[i] * k + c] - mean;
      bm[i * k + c] = v;
      r[i * k + c] = v;
      x[i * k + c] = 0.0;
      p[i * k + c] = 0.0;
      acc[0] += v * v;
    }
  }
  if (col_grid_sum<KP, 1>(acc, partials, ticket, tmp)) {
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
__global__ void k_m_z_reduce(int64_t n, int k, const T* __restrict__ z, const double* __restrict__ r,
                             const double* __restrict__ ro, double* scal, double* partials, unsigned* ticket,
                             double* tmp) {
  const int first = scal[k * kMS + gIter] == 0.0;
  const int c = threadIdx.x & (KP - 1);
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (c < k) {
    LG_COL_STRIDE(i, n) {
      const int64_t e = i * k + c;
      const double zi = (double)z[e], ri = r[e], roi = first ? 0.0 : ro[e];
      acc[0] += zi;
      acc[1] += zi * ri;
      acc[2] += zi * roi;
      acc[3] += ri;
      acc[4] += roi;
    }
  }
  if (col_grid_sum<KP, 5>(acc, partials, ticket, tmp)) {
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

template <typename T>
__global__ void k_m_p_update(int64_t n, int k, const T* __restrict__ z, double* __restrict__ p, const double* scal) {
  LG_GRID_STRIDE(e, n * k) {
    const int c = (int)(e % k);
    const double* sc = scal + c * kMS;
    // a frozen column keeps p = 0 (its scalars may be 0/0)
    p[e] = sc[mActive] != 0.0 ? ((double)z[e] - sc[mMeanZ]) + sc[mBeta] * p[e] : 0.0;
  }
}

template <int KP>
__global__ void k_m_pq(int64_t n, int k, const double* __restrict__ p, const double* __restrict__ q, double* scal,
                       double* partials, unsigned* ticket, double* tmp) {
  const int c = threadIdx.x & (KP - 1);
  double acc[1] = {0.0};
  if (c < k) LG_COL_STRIDE(i, n) acc[0] += p[i * k + c] * q[i * k + c];
  if (col_grid_sum<KP, 1>(acc, partials, ticket, tmp)) {
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

// r_old = r; x += alpha p; r -= alpha q (alpha = 0 freezes a finished column); ||r||^2.
template <int KP>
__global__ void k_m_xr(int64_t n, int k, double* __restrict__ x, double* __restrict__ r, double* __restrict__ ro,
                       const double* __restrict__ p, const double* __restrict__ q, double* scal, double* partials,
                       unsigned* ticket, double* tmp, cudaGraphConditionalHandle handle, int in_graph) {
  const int c = threadIdx.x & (KP - 1);
  double acc[1] = {0.0};
  if (c < k) {
    const double a = scal[c * kMS + mAlpha];
    const bool live = scal[c * kMS + mActive] != 0.0;  // frozen columns keep x and r
    LG_COL_STRIDE(i, n) {
      const int64_t e = i * k + c;
      const double ri = r[e];
      ro[e] = ri;
      double rn = ri;
      if (live) {
        x[e] += a * p[e];
        rn = ri - a * q[e];
        r[e] = rn;
      }
      acc[0] += rn * rn;
    }
  }
  if (col_grid_sum<KP, 1>(acc, partials, ticket, tmp)) {
    // count the iteration; ask for the true residuals on replacement
    // iterations or when a live column's recurrence residual meets the
    // tolerance; otherwise set the loop condition here (inside the graph)
    double* gl = scal + k * kMS;
    const double it = gl[gIter] + 1.0;
    gl[gIter] = it;
    bool need = fmod(it, gl[gEvery]) == 0.0, any = false;
    for (int cc = 0; cc < k; ++cc) {
      double* sc = scal + cc * kMS;
      sc[mRR] = tmp[cc];
      if (sc[mActive] != 0.0) {
        sc[mIter] += 1.0;
        any = true;
        if (sc[mRR] <= sc[mTol2BB]) need = true;
      }
    }
    gl[gNeed] = need ? 1.0 : 0.0;
    if (!need && in_graph) cudaGraphSetConditional(handle, any && it < gl[gMaxit] ? 1u : 0u);
  }
}

// ||r||^2 per column. Inside the loop (loop = 1, gated by the true-residual
// request) the last block also freezes every live column whose true residual
// meets the tolerance and sets the loop condition: go on while a column is
// live and the iteration bound allows.
template <int KP>
__global__ void k_m_rr(int64_t n, int k, const double* __restrict__ r, double* scal, double* partials,
                       unsigned* ticket, double* tmp, const double* gate, int loop, cudaGraphConditionalHandle handle,
                       int in_graph) {
  if (gate && *gate == 0.0) return;
  const int c = threadIdx.x & (KP - 1);
  double acc[1] = {0.0};
  if (c < k) LG_COL_STRIDE(i, n) acc[0] += r[i * k + c] * r[i * k + c];
  if (col_grid_sum<KP, 1>(acc, partials, ticket, tmp)) {
    for (int cc = 0; cc < k; ++cc) scal[cc * kMS + mRR] = tmp[cc];
    if (loop) {
      double* gl = scal + k * kMS;
      const double it = gl[gIter];
      bool any = false;
      for (int cc = 0; cc < k; ++cc) {
        double* sc = scal + cc * kMS;
        if (sc[mActive] != 0.0 && sc[mRR] <= sc[mTol2BB]) {
          sc[mActive] = 0.0;
          sc[mDone] = 1.0;
          sc[mConv] = it;
        }
        if (sc[mActive] != 0.0) any = true;
      }
      if (in_graph) cudaGraphSetConditional(handle, any && it < gl[gMaxit] ? 1u : 0u);
    }
  }
}

// x columns back to the caller's numbering, column mean removed.
template <int KP>
__global__ void k_m_out(int64_t n, int k, const double* __restrict__ x, const int32_t* __restrict__ perm,
                        const double* __restrict__ colsum, double* __restrict__ out) {
  LG_GRID_STRIDE(e, n * k) {
    const int64_t i = e / k;
    const int c = (int)(e - i * k);
    out[(int64_t)perm[i] * k + c] = x[e] - colsum[c] / (double)n;
  }
}

// ---------------------------------------------------------------------------
// Host side: plans, the multi-column cycle and PCG loop.
// ---------------------------------------------------------------------------
struct BatchState {
  std::vector<std::unique_ptr<MPlanStore>> op, mem, pt, lp;  // per level
  DBuf<double> tmp, colsum;                              // reduction totals of the column kernels
  std::map<std::pair<int, int>, cudaGraphExec_t> graphs;  // captured loop per (FP32?, k)
  ~BatchState() {
    for (auto& g : graphs)
      if (g.second) cudaGraphExecDestroy(g.second);
  }
};

template <typename T> static std::vector<LevelVecs<T>>& mvecs(Workspace& ws);
template <> std::vector<LevelVecs<double>>& mvecs<double>(Workspace& ws) { return ws.v64; }
template <> std::vector<LevelVecs<float>>& mvecs<float>(Workspace& ws) { return ws.v32; }
template <typename T> static const T* mpt_coef(const Level& L);
template <> const double* mpt_coef<double>(const Level& L) { return L.pt_coef.get(); }
template <> const float* mpt_coef<float>(const Level& L) { return L.pt_coef32.get(); }

template <typename T>
static MLp<T> mlp_term(const OpView<T>& w, const T* xc, const int32_t* agg, int k);
template <>
MLp<float> mlp_term<float>(const OpView<float>& w, const float* xc, const int32_t* agg, int k) {
  return MLp<float>{w.w, xc, agg, k};
}
template <>
MLp<double> mlp_term<double>(const OpView<double>& w, const double* xc, const int32_t* agg, int k) {
  return MLp<double>{w.w, xc, agg, w.d, k};
}

template <typename T>
static void mcycle(Hier& h, Workspace& ws, BatchState& bs, int l, int k, int kp, cudaStream_t s) {
  const Level& L = *h.levels[l];
  LevelVecs<T>& V = mvecs<T>(ws)[l];
  const int64_t n = L.n;
  if (L.kind == LG_LEVEL_COARSEST) {
    k_m_coarse_apply<T><<<grid_for(n * 32, kBT, kSMs * 8), kBT, 0, s>>>(n, k, L.pinv.get(), V.f.get(), V.x.get());
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
    launch_mrows<T>(kp, L.nc, k, L.pt_ptr.get(), L.pt_f.get(), MWGather<T>{mpt_coef<T>(L), V.f.get(), k},
                    bs.pt[l]->plan, MEpiElimRestrict<T>{V.f.get(), L.cfine.get(), C.f.get(), d0n, dinvn, itn, k}, s);
    mcycle<T>(h, ws, bs, l + 1, k, kp, s);
    const OpView<T> op = L.op<T>();
    k_m_elim_prolong<T><<<bblocks(n * k), kBT, 0, s>>>(n, k, op.rowptr, op.col, op.w, op.dinv, L.cmap.get(),
                                                       V.f.get(), C.x.get(), V.x.get());
    LG_LAUNCH_CHECK();
    return;
  }
  const OpView<T> op = L.op<T>();
  const MPlan& P = bs.op[l]->plan;
  const Cheb& ch = h.cheb[l];
  const int deg = h.opts.cheb_degree;
  T* g = V.dA.get();
  T* gn = V.dB.get();
  const T* rin = V.f.get();
  for (int st = 1; st < deg; ++st) {
    launch_mrows<T>(kp, n, k, op.rowptr, op.col, MLap<T>{op.w, g, op.d, k}, P,
                    MEpiCheb<T>{g, rin, V.r.get(), op.dinv, gn, V.x.get(), st == 1 ? 1 : 2, st == deg - 1, k,
                                (T)ch.c1[st], (T)ch.c2[st]},
                    s);
    rin = V.r.get();
    std::swap(g, gn);
  }
  launch_mrows<T>(kp, n, k, op.rowptr, op.col, MLap<T>{op.w, g, op.d, k}, P,
                  MEpiCheb<T>{g, rin, V.r.get(), op.dinv, nullptr, deg == 1 ? V.x.get() : nullptr, 1, 0, k, T(0), T(0)},
                  s);
  launch_mrows<T>(kp, L.nc, k, L.mem_ptr.get(), L.mem.get(), MGather<T>{V.r.get(), k}, bs.mem[l]->plan,
                  MEpiRestrict<T>{C.f.get(), d0n, dinvn, itn, k}, s);
  mcycle<T>(h, ws, bs, l + 1, k, kp, s);
  if (L.lp_nnz > 0) {  // x += P x_c, r_0 = r_pre - L P x_c, d_0: one pass over W
    const OpView<T> lp = L.lp<T>();
    launch_mrows<T>(kp, n, k, lp.rowptr, lp.col, mlp_term<T>(lp, C.x.get(), L.agg.get(), k), bs.lp[l]->plan,
                    MEpiPost<T>{V.r.get(), V.x.get(), C.x.get(), L.agg.get(), op.dinv, V.dA.get(), (T)ch.inv_theta, k},
                    s);
  } else {
    k_m_agg_prolong<T><<<bblocks(n * k), kBT, 0, s>>>(n, k, L.agg.get(), C.x.get(), V.x.get());
    LG_LAUNCH_CHECK();
    launch_mrows<T>(kp, n, k, op.rowptr, op.col, MLap<T>{op.w, V.x.get(), op.d, k}, P,
                    MEpiCheb<T>{V.x.get(), V.f.get(), V.r.get(), op.dinv, V.dA.get(), nullptr, 0, 0, k, T(0),
                                (T)ch.inv_theta},
                    s);
  }
  g = V.dA.get();
  gn = V.dB.get();
  for (int st = 1; st < deg; ++st) {
    launch_mrows<T>(kp, n, k, op.rowptr, op.col, MLap<T>{op.w, g, op.d, k}, P,
                    MEpiCheb<T>{g, V.r.get(), V.r.get(), op.dinv, gn, V.x.get(), 2, st == deg - 1, k, (T)ch.c1[st],
                                (T)ch.c2[st]},
                    s);
    std::swap(g, gn);
  }
  if (deg == 1) {
    k_m_axpy1<T><<<bblocks(n * k), kBT, 0, s>>>(n * k, V.dA.get(), V.x.get());
    LG_LAUNCH_CHECK();
  }
}

// One multi-column PCG iteration (as pcg_body in lg_cycle.cu): z = M r, the
// per-column sums, beta and p; q = L p; alpha; x, r and the true-residual
// request; the requested true residuals, which freeze converged columns.
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
  k_m_cycle_in<T><<<bblocks(n * k), kBT, 0, s>>>(n, k, ws.r.get(), V.f.get(), d0, dinv, it);
  LG_LAUNCH_CHECK();
  mcycle<T>(h, ws, bs, 0, k, KP, s);
  const T* z = V.x.get();
  const int vb = grid_for(n * KP, kBT, kSMs * 8);
  k_m_z_reduce<T, KP><<<vb, kBT, 0, s>>>(n, k, z, ws.r.get(), ws.ro.get(), scal, ws.partials.get(),
                                         ws.tickets.get(), tmp);
  LG_LAUNCH_CHECK();
  k_m_p_update<T><<<bblocks(n * k), kBT, 0, s>>>(n, k, z, ws.p.get(), scal);
  LG_LAUNCH_CHECK();
  const OpView<double> op = L0.op<double>();
  launch_mrows<double>(KP, n, k, op.rowptr, op.col, MLap<double>{op.w, ws.p.get(), op.d, k}, bs.op[0]->plan,
                       MEpiStore{ws.q.get(), k}, s);
  k_m_pq<KP><<<vb, kBT, 0, s>>>(n, k, ws.p.get(), ws.q.get(), scal, ws.partials.get(), ws.tickets.get(), tmp);
  LG_LAUNCH_CHECK();
  k_m_xr<KP><<<vb, kBT, 0, s>>>(n, k, ws.x.get(), ws.r.get(), ws.ro.get(), ws.p.get(), ws.q.get(), scal,
                                ws.partials.get(), ws.tickets.get(), tmp, handle, in_graph);
  LG_LAUNCH_CHECK();
  mtrue_res<KP>(h, ws, bs, k, s, scal + k * kMS + gNeed, 1, handle, in_graph);
}

template <int KP>
static void mtrue_res(Hier& h, Workspace& ws, BatchState& bs, int k, cudaStream_t s, const double* gate, int loop,
                      cudaGraphConditionalHandle handle, int in_graph) {
  const Level& L0 = *h.levels[0];
  const int64_t n = L0.n;
  const OpView<double> op = L0.op<double>();
  launch_mrows<double>(KP, n, k, op.rowptr, op.col, MLap<double>{op.w, ws.x.get(), op.d, k}, bs.op[0]->plan,
                       MEpiTrueRes{ws.bm.get(), ws.r.get(), k}, s, gate);
  k_m_rr<KP><<<grid_for(n * KP, kBT, kSMs * 8), kBT, 0, s>>>(n, k, ws.r.get(), ws.scal.get(), ws.partials.get(),
                                                            ws.tickets.get(), bs.tmp.get(), gate, loop, handle,
                                                            in_graph);
  LG_LAUNCH_CHECK();
}

static BatchState& batch_state(Hier& h, Workspace& ws, cudaStream_t s);

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

template <typename T, int KP>
static int msolve(Hier& h, Workspace& ws, int k, const double* B, double* X, double tol, cudaStream_t s,
                  lg_info* infos) {
  const Level& L0 = *h.levels[0];
  const int64_t n = L0.n;
  BatchState& bs = batch_state(h, ws, s);
  double* scal = ws.scal.get();
  double* tmp = bs.tmp.get();
  double* colsum = bs.colsum.get();
  const int maxit = h.opts.max_iter;
  const int every = h.opts.residual_replace > 0 ? h.opts.residual_replace : 1 << 30;
  cudaEvent_t e0, e1;
  LG_CUDA(cudaEventCreate(&e0));
  LG_CUDA(cudaEventCreate(&e1));
  LG_CUDA(cudaEventRecord(e0, s));
  const int vb = grid_for(n * KP, kBT, kSMs * 8);
  k_m_colsum<KP><<<vb, kBT, 0, s>>>(n, k, B, ws.partials.get(), ws.tickets.get(), colsum);
  LG_LAUNCH_CHECK();
  k_m_init<KP><<<vb, kBT, 0, s>>>(n, k, B, h.perm.get(), colsum, ws.bm.get(), ws.x.get(), ws.r.get(), ws.p.get(),
                                  scal, ws.partials.get(), ws.tickets.get(), tmp, tol, maxit, every);
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
  k_m_colsum<KP><<<vb, kBT, 0, s>>>(n, k, ws.x.get(), ws.partials.get(), ws.tickets.get(), colsum);
  LG_LAUNCH_CHECK();
  bool all_done = true;
  for (int c = 0; c < k; ++c)
    if (hs[c * kMS + mDone] == 0.0 && hs[c * kMS + mBB] != 0.0) all_done = false;
  if (!all_done) {
    mtrue_res<KP>(h, ws, bs, k, s, nullptr, 0, cudaGraphConditionalHandle{}, 0);
    read();
  }
  k_m_out<KP><<<bblocks(n * k), kBT, 0, s>>>(n, k, ws.x.get(), h.perm.get(), colsum, ws.io.get());
  LG_LAUNCH_CHECK();
  (void)X;  // the caller transposes ws.io into X
  LG_CUDA(cudaEventRecord(e1, s));
  LG_CUDA(cudaStreamSynchronize(s));
  float ms = 0.f;
  LG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
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

static BatchState& batch_state(Hier& h, Workspace& ws, cudaStream_t s) {
  if (!ws.batch) {
    auto st = std::make_shared<BatchState>();
    st->op.resize(h.levels.size());
    st->mem.resize(h.levels.size());
    st->pt.resize(h.levels.size());
    st->lp.resize(h.levels.size());
    for (size_t l = 0; l < h.levels.size(); ++l) {
      const Level& L = *h.levels[l];
      st->op[l] = std::make_unique<MPlanStore>();
      st->op[l]->build(L.n, L.rowptr.get(), s, &ws.bytes);
      if (L.kind == LG_LEVEL_AGG) {
        st->mem[l] = std::make_unique<MPlanStore>();
        st->mem[l]->build(L.nc, L.mem_ptr.get(), s, &ws.bytes);
      }
      if (L.kind == LG_LEVEL_ELIM) {
        st->pt[l] = std::make_unique<MPlanStore>();
        st->pt[l]->build(L.nc, L.pt_ptr.get(), s, &ws.bytes);
      }
      if (L.lp_nnz > 0) {
        st->lp[l] = std::make_unique<MPlanStore>();
        st->lp[l]->build(L.n, L.lp_ptr.get(), s, &ws.bytes);
      }
    }
    st->tmp.alloc(5 * kMaxCols, s, &ws.bytes);
    st->colsum.alloc(kMaxCols, s, &ws.bytes);
    ws.batch = st;
  }
  return *static_cast<BatchState*>(ws.batch.get());
}

// Column-major (ld = n) <-> row-major [n][k].
__global__ void k_cm_to_rm(int64_t n, int k, const double* __restrict__ cm, double* __restrict__ rm) {
  LG_GRID_STRIDE(e, n * k) {
    const int64_t i = e / k;
    rm[e] = cm[(e - i * k) * n + i];
  }
}

__global__ void k_rm_to_cm(int64_t n, int k, const double* __restrict__ rm, double* __restrict__ cm) {
  LG_GRID_STRIDE(e, n * k) {
    const int64_t i = e / k;
    cm[(e - i * k) * n + i] = rm[e];
  }
}

// B, X: device, column-major n x k with leading dimension n.
int pcg_solve_batch(Hier& h, Workspace& ws, int k, const double* B, double* X, double tol, int precision,
                    cudaStream_t s, lg_info* infos) {
  if (k == 1) return pcg_solve(h, ws, B, X, tol, precision, s, infos);
  if (ws.k < k) fail(LG_ERR_INVALID, "workspace narrower than the batch");
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
  const int kp = pow2_at_least(k);
  const bool f32 = precision == LG_FP32_HIER;
  k_cm_to_rm<<<bblocks(n * k), kBT, 0, s>>>(n, k, B, ws.z.get());
  LG_LAUNCH_CHECK();
  int st = LG_OK;
#define LG_MS_CASE(KK)                                                                  \
  case KK:                                                                              \
    st = f32 ? msolve<float, KK>(h, ws, k, ws.z.get(), nullptr, tol, s, infos)          \
             : msolve<double, KK>(h, ws, k, ws.z.get(), nullptr, tol, s, infos);        \
    break;
  switch (kp) {
    LG_MS_CASE(2)
    LG_MS_CASE(4)
    LG_MS_CASE(8)
    LG_MS_CASE(16)
    LG_MS_CASE(32)
    default:
      fail(LG_ERR_INVALID, "batch width");
  }
#undef LG_MS_CASE
  k_rm_to_cm<<<bblocks(n * k), kBT, 0, s>>>(n, k, ws.io.get(), X);
  LG_LAUNCH_CHECK();
  LG_CUDA(cudaStreamSynchronize(s));
  return st;
}

// x = M f for k columns (F, X device, column-major, leading dimension n, in
// the caller's numbering), starting from x = 0: the multi-column cycle alone.
__global__ void k_m_gather_perm(int64_t n, int k, const int32_t* __restrict__ perm, const double* __restrict__ src,
                                double* __restrict__ dst) {
  LG_GRID_STRIDE(e, n * k) {
    const int64_t i = e / k;
    dst[e] = src[(int64_t)perm[i] * k + (e - i * k)];
  }
}

template <typename T>
__global__ void k_m_scatter_out(int64_t n, int k, const int32_t* __restrict__ perm, const T* __restrict__ src,
                                double* __restrict__ dst) {
  LG_GRID_STRIDE(e, n * k) {
    const int64_t i = e / k;
    dst[(int64_t)perm[i] * k + (e - i * k)] = (double)src[e];
  }
}

template <typename T>
static void mcycle_apply(Hier& h, Workspace& ws, int k, const double* F, double* X, cudaStream_t s) {
  const Level& L0 = *h.levels[0];
  const int64_t n = L0.n;
  BatchState& bs = batch_state(h, ws, s);
  k_cm_to_rm<<<bblocks(n * k), kBT, 0, s>>>(n, k, F, ws.z.get());
  LG_LAUNCH_CHECK();
  k_m_gather_perm<<<bblocks(n * k), kBT, 0, s>>>(n, k, h.perm.get(), ws.z.get(), ws.r.get());
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
  k_m_cycle_in<T><<<bblocks(n * k), kBT, 0, s>>>(n, k, ws.r.get(), V.f.get(), d0, dinv, it);
  LG_LAUNCH_CHECK();
  mcycle<T>(h, ws, bs, 0, k, pow2_at_least(k), s);
  k_m_scatter_out<T><<<bblocks(n * k), kBT, 0, s>>>(n, k, h.perm.get(), V.x.get(), ws.io.get());
  LG_LAUNCH_CHECK();
  k_rm_to_cm<<<bblocks(n * k), kBT, 0, s>>>(n, k, ws.io.get(), X);
  LG_LAUNCH_CHECK();
}

void vcycle_apply_batch(Hier& h, Workspace& ws, int k, const double* F, double* X, int precision, cudaStream_t s) {
  if (ws.k < k) fail(LG_ERR_INVALID, "workspace narrower than the batch");
  if (h.opts.kcycle) {  // the SpMM cycle is the V-cycle: K-cycle columns one at a time
    const int64_t n = h.levels[0]->n;
    for (int c = 0; c < k; ++c) vcycle_apply(h, ws, F + (size_t)c * n, X + (size_t)c * n, precision, s);
    return;
  }
  if (precision == LG_FP32_HIER) mcycle_apply<float>(h, ws, k, F, X, s);
  else mcycle_apply<double>(h, ws, k, F, X, s);
}

}  // namespace lg
