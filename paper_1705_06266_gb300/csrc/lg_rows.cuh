// Row-parallel CSR pass used by every SpMV-shaped kernel of the library.
//
// A pass computes, for every row i of a CSR structure,
//   s_i = finish_i( sum_k term(i, k) )
// over the row's entries, then calls an epilogue with (i, s_i). Rows are
// split into three tiers when the plan is built:
//  - short rows (at most kShortMax entries): aligned groups of G lanes, G in
//    {1, 2, 4, 8} chosen per precision by the setup's autotuner; the group
//    walks its rows with a stride over the grid and prefetches the next row's
//    extent and the epilogue operands before the entry loop;
//  - medium rows (up to plan.long_thresh entries): one warp per row, from a
//    row list;
//  - long rows: chunks of kChunk entries, one block each; the last block of a
//    row to finish (a per-row ticket) adds the chunk partials in chunk order.
// Every addition happens in an order fixed by the row lengths and the plan,
// never by timing, so each pass is bitwise reproducible.
//
// An epilogue may contribute NRED values to grid-wide sums (dot products of
// the Krylov solver); these are combined with lg::grid_sum at the end of the
// launch (the launch grid of a plan is fixed), and epi.finish(totals) runs
// once, in the last block, to derive scalars from them.
#pragma once

#include "lg_common.cuh"

namespace lg {

// The Laplacian applied to x (Section 2.1: L = D - A, D_ii = sum_j w_ij).
// FP32: difference form, sum_j w_ij (x_i - x_j), so L 1 = 0 holds exactly.
// FP64: d_i x_i - sum_j w_ij x_j, one fused multiply-add per entry (FP64
// arithmetic is the scarce resource of the part), with d the stored row sums.
template <typename T>
struct LapTerm;

template <>
struct LapTerm<float> {
  const float* __restrict__ w;
  const float* __restrict__ x;
  const double* __restrict__ d;  // unused
  __device__ __forceinline__ float row(int64_t i) const { return __ldg(&x[i]); }
  __device__ __forceinline__ float operator()(int64_t k, int32_t j, float xi) const {
    return __ldg(&w[k]) * (xi - __ldg(&x[j]));
  }
  __device__ __forceinline__ float finish(float, float s) const { return s; }
};

template <>
struct LapTerm<double> {
  const double* __restrict__ w;
  const double* __restrict__ x;
  const double* __restrict__ d;
  __device__ __forceinline__ double row(int64_t i) const { return __ldg(&d[i]) * __ldg(&x[i]); }
  __device__ __forceinline__ double operator()(int64_t k, int32_t j, double) const {
    return __ldg(&w[k]) * __ldg(&x[j]);
  }
  __device__ __forceinline__ double finish(double dx, double s) const { return dx - s; }
};

// Plain gather-sum: sum_k v[idx_k] (restriction by aggregate member lists).
template <typename T>
struct GatherTerm {
  const T* __restrict__ v;
  __device__ __forceinline__ T row(int64_t) const { return T(0); }
  __device__ __forceinline__ T operator()(int64_t, int32_t j, T) const { return __ldg(&v[j]); }
  __device__ __forceinline__ T finish(T, T s) const { return s; }
};

// Weighted gather-sum: sum_k c_k v[idx_k] (transpose of the elimination prolongation).
template <typename T>
struct WGatherTerm {
  const T* __restrict__ c;
  const T* __restrict__ v;
  __device__ __forceinline__ T row(int64_t) const { return T(0); }
  __device__ __forceinline__ T operator()(int64_t k, int32_t j, T) const { return __ldg(&c[k]) * __ldg(&v[j]); }
  __device__ __forceinline__ T finish(T, T s) const { return s; }
};

// Sum of a row's entries with G lanes, four loads in flight per lane.
template <typename T, int G, class Term>
__device__ __forceinline__ T row_sum(const Term& term, const int32_t* __restrict__ col, int64_t beg, int64_t end,
                                     int lane, T rv) {
  T s0 = T(0), s1 = T(0);
  int64_t k = beg + lane;
  for (; k + 3 * G < end; k += 4 * G) {
    const int32_t j0 = __ldg(&col[k]), j1 = __ldg(&col[k + G]);
    const int32_t j2 = __ldg(&col[k + 2 * G]), j3 = __ldg(&col[k + 3 * G]);
    const T a0 = term(k, j0, rv), a1 = term(k + G, j1, rv);
    const T a2 = term(k + 2 * G, j2, rv), a3 = term(k + 3 * G, j3, rv);
    s0 += a0 + a2;
    s1 += a1 + a3;
  }
  for (; k < end; k += G) s0 += term(k, __ldg(&col[k]), rv);
  return s0 + s1;
}

template <typename T, int G, int NRED, class Term, class Epi>
__global__ void __launch_bounds__(kRowThreads)
k_rows(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, Term term,
       RowPlan plan, Epi epi, double* __restrict__ red_partials, unsigned* red_ticket,
       double* red_out) {
  double red[NRED > 0 ? NRED : 1];
#pragma unroll
  for (int q = 0; q < (NRED > 0 ? NRED : 1); ++q) red[q] = 0.0;
  const int64_t bid = blockIdx.x;

  if (bid < plan.nchunks) {
    // ---- one chunk of a long row ----
    __shared__ T sred[kRowThreads / 32];
    const int64_t c = bid;
    const int64_t row = plan.chunk_row[c];
    const int64_t beg = plan.chunk_beg[c];
    const int64_t rend = rowptr[row + 1];
    const int64_t end = beg + kChunk < rend ? beg + kChunk : rend;
    const T rv = term.row(row);
    T s = row_sum<T, kRowThreads>(term, col, beg, end, threadIdx.x, rv);
    s = group_sum<32>(s, 0xffffffffu);
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
      T t = threadIdx.x < kRowThreads / 32 ? sred[threadIdx.x] : T(0);
      t = group_sum<32>(t, 0xffffffffu);
      if (threadIdx.x == 0) {
        const int32_t lr = plan.chunk_lrow[c];
        plan.partial[c] = (double)t;
        __threadfence();
        unsigned tk = atomicAdd(&plan.ticket[lr], 1u);
        if (tk == (unsigned)plan.lrow_count[lr] - 1u) {
          __threadfence();
          const int32_t f0 = plan.lrow_first[lr], cnt = plan.lrow_count[lr];
          T tot = T(0);
          for (int32_t q = 0; q < cnt; ++q) tot += (T)__ldcg(&plan.partial[f0 + q]);
          plan.ticket[lr] = 0u;
          epi(row, term.finish(rv, tot), epi.pre(row), red);
        }
      }
    }
  } else if (bid < plan.nchunks + plan.med_blocks) {
    // ---- medium rows: one warp per row ----
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (bid - plan.nchunks) * (kRowThreads / 32) + (threadIdx.x >> 5);
    const int64_t stride = (int64_t)plan.med_blocks * (kRowThreads / 32);
    for (int64_t m = w0; m < plan.nmed; m += stride) {
      const int64_t row = plan.med_rows[m];
      const int64_t beg = rowptr[row], end = rowptr[row + 1];
      const auto pre = epi.pre(row);
      const T rv = term.row(row);
      T s = row_sum<T, 32>(term, col, beg, end, lane, rv);
      s = group_sum<32>(s, 0xffffffffu);
      if (lane == 0) epi(row, term.finish(rv, s), pre, red);
    }
  } else {
    // ---- short rows: one aligned group of G lanes per row ----
    const int64_t sb = bid - plan.nchunks - plan.med_blocks;
    constexpr int64_t kGroups = kRowThreads / G;
    const int lane = threadIdx.x & (G - 1);
    const unsigned mask = group_mask<G>();
    const int64_t stride = (int64_t)(sizeof(T) == 8 ? plan.short_blocks64 : plan.short_blocks32) * kGroups;
    int64_t row = sb * kGroups + threadIdx.x / G;
    int64_t beg = 0, end = 0;
    if (row < n) { beg = rowptr[row]; end = rowptr[row + 1]; }
    while (row < n) {
      const int64_t nrow = row + stride;
      int64_t nbeg = 0, nend = 0;
      if (nrow < n) { nbeg = rowptr[nrow]; nend = rowptr[nrow + 1]; }
      if (end - beg <= kShortMax) {
        const auto pre = epi.pre(row);
        const T rv = term.row(row);
        T s = row_sum<T, G>(term, col, beg, end, lane, rv);
        s = group_sum<G>(s, mask);
        if (lane == 0) epi(row, term.finish(rv, s), pre, red);
      }
      row = nrow;
      beg = nbeg;
      end = nend;
    }
  }
  if constexpr (NRED > 0) {
    if (grid_sum<kRowThreads, NRED>(red, red_partials, red_ticket, red_out)) epi.finish(red_out);
  }
}

template <typename T, int NRED, class Term, class Epi>
inline void launch_rows(int64_t n, const int64_t* rowptr, const int32_t* col, const Term& term,
                        const RowPlan& plan, const Epi& epi, cudaStream_t s,
                        double* red_partials = nullptr, unsigned* red_ticket = nullptr,
                        double* red_out = nullptr) {
  const int grid = plan.grid((int)sizeof(T));
  const int G = sizeof(T) == 8 ? plan.G64 : plan.G32;
#define LG_ROWS_CASE(GG)                                                                         \
  case GG:                                                                                       \
    k_rows<T, GG, NRED, Term, Epi><<<grid, kRowThreads, 0, s>>>(n, rowptr, col, term, plan, epi, \
                                                                 red_partials, red_ticket, red_out); \
    break;
  switch (G) {
    LG_ROWS_CASE(1)
    LG_ROWS_CASE(2)
    LG_ROWS_CASE(4)
    LG_ROWS_CASE(8)
    default:
      fail(LG_ERR_INVALID, "row plan group size");
  }
#undef LG_ROWS_CASE
  LG_LAUNCH_CHECK();
}

// An epilogue with nothing to prefetch and nothing to reduce.
struct NoPre {};

}  // namespace lg
