// Row-parallel CSR pass used by every SpMV-shaped kernel of the library.
//
// A pass computes, for every row i of a CSR structure, s_i = sum_k term(i, k)
// over the row's entries, then calls an epilogue with (i, s_i). Rows of at
// most plan.long_thresh entries are handled by aligned groups of G lanes
// (coalesced loads of G consecutive col / value entries, an xor-butterfly
// reduction); longer rows are cut into chunks of kChunk entries handled by one
// block each, and the last block of a row to finish (a per-row ticket) adds
// the chunk partials in chunk order before the epilogue. The order of every
// addition depends only on the row lengths and G, never on timing, so each
// pass is bitwise reproducible.
//
// An epilogue may contribute NRED values to grid-wide sums (dot products of
// the Krylov solver); these are combined with lg::grid_sum at the end of the
// launch (the launch grid of a plan is fixed), and epi.finish(totals) runs
// once, in the last block, to derive scalars from them.
#pragma once

#include "lg_common.cuh"

namespace lg {

// Term of the Laplacian in difference form: w_ij (x_i - x_j), so L 1 = 0
// exactly in any precision (Section 2.1: L = D - A, D_ii = sum_j w_ij).
template <typename T>
struct LapTerm {
  const T* __restrict__ w;
  const T* __restrict__ x;
  __device__ __forceinline__ T row(int64_t i) const { return x[i]; }
  __device__ __forceinline__ T operator()(int64_t k, int32_t j, T xi) const {
    return w[k] * (xi - __ldg(&x[j]));
  }
};

// Plain gather-sum: sum_k v[idx_k] (restriction by aggregate member lists).
template <typename T>
struct GatherTerm {
  const T* __restrict__ v;
  __device__ __forceinline__ T row(int64_t) const { return T(0); }
  __device__ __forceinline__ T operator()(int64_t, int32_t j, T) const { return __ldg(&v[j]); }
};

// Weighted gather-sum: sum_k c_k v[idx_k] (transpose of the elimination prolongation).
template <typename T>
struct WGatherTerm {
  const T* __restrict__ c;
  const T* __restrict__ v;
  __device__ __forceinline__ T row(int64_t) const { return T(0); }
  __device__ __forceinline__ T operator()(int64_t k, int32_t j, T) const { return c[k] * __ldg(&v[j]); }
};

template <typename T, int G, int NRED, class Term, class Epi>
__global__ void __launch_bounds__(kRowThreads)
k_rows(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, Term term,
       RowPlan plan, Epi epi, double* __restrict__ red_partials, unsigned* red_ticket,
       double* red_out) {
  double red[NRED > 0 ? NRED : 1];
#pragma unroll
  for (int q = 0; q < (NRED > 0 ? NRED : 1); ++q) red[q] = 0.0;

  if ((int64_t)blockIdx.x < plan.nchunks) {
    // ---- one chunk of a long row ----
    __shared__ T sred[kRowThreads / 32];
    const int64_t c = blockIdx.x;
    const int64_t row = plan.chunk_row[c];
    const int64_t beg = plan.chunk_beg[c];
    const int64_t rend = rowptr[row + 1];
    const int64_t end = beg + kChunk < rend ? beg + kChunk : rend;
    const T xi = term.row(row);
    T s = T(0);
    for (int64_t k = beg + threadIdx.x; k < end; k += kRowThreads) s += term(k, col[k], xi);
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
          epi(row, tot, red);
        }
      }
    }
  } else {
    // ---- short rows: one aligned group of G lanes per row ----
    const int64_t sb = (int64_t)blockIdx.x - plan.nchunks;
    constexpr int64_t kGroups = kRowThreads / G;
    const int lane = threadIdx.x & (G - 1);
    const unsigned mask = group_mask<G>();
    const int64_t stride = (int64_t)plan.short_blocks * kGroups;
    for (int64_t row = sb * kGroups + threadIdx.x / G; row < n; row += stride) {
      const int64_t beg = rowptr[row], end = rowptr[row + 1];
      if (end - beg > plan.long_thresh) continue;
      const T xi = term.row(row);
      T s = T(0);
      for (int64_t k = beg + lane; k < end; k += G) s += term(k, __ldg(&col[k]), xi);
      s = group_sum<G>(s, mask);
      if (lane == 0) epi(row, s, red);
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
  const int grid = (int)(plan.nchunks + plan.short_blocks);
#define LG_ROWS_CASE(GG)                                                                         \
  case GG:                                                                                       \
    k_rows<T, GG, NRED, Term, Epi><<<grid, kRowThreads, 0, s>>>(n, rowptr, col, term, plan, epi, \
                                                                 red_partials, red_ticket, red_out); \
    break;
  switch (plan.G) {
    LG_ROWS_CASE(2)
    LG_ROWS_CASE(4)
    LG_ROWS_CASE(8)
    LG_ROWS_CASE(16)
    LG_ROWS_CASE(32)
    default:
      fail(LG_ERR_INVALID, "row plan group size");
  }
#undef LG_ROWS_CASE
  LG_LAUNCH_CHECK();
}

}  // namespace lg
