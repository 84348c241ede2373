// Row-parallel CSR pass used by every SpMV-shaped kernel of the library.
//
// A pass computes, for every row i of a CSR structure,
//   s_i = finish_i( sum_k term(i, k) )
// over the row's entries, then calls an epilogue with (i, s_i). The plan
// (lg_common.cuh) bins the rows by length: a row of class c is handled by one
// aligned group of G = 2^c lanes, every lane taking about E entries, so the
// groups of a warp finish together and each lane has its loads in flight at
// once; the group reduces into its first lane, which applies the epilogue
// with operands prefetched before the entry loop. Rows longer than kChunk
// entries are cut into chunks, one block each; the last block of a row to
// finish (a per-row ticket) adds the chunk partials in chunk order. Every
// addition happens in an order fixed by the row lengths and the plan, never
// by timing, so each pass is bitwise reproducible.
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

// One row of class G: group of G lanes, reduction into the group's lane 0.
template <typename T, int G, class Term, class Epi>
__device__ __forceinline__ void class_row(const RowPlan& plan, int c, int64_t b, const int64_t* __restrict__ rowptr,
                                          const int32_t* __restrict__ col, const Term& term, const Epi& epi,
                                          double* red) {
  const int64_t idx = b * (kRowThreads / G) + threadIdx.x / G;
  const int64_t lo = plan.cls_off[c], hi = plan.cls_off[c + 1];
  const int lane = threadIdx.x & (G - 1);
  if (lo + idx >= hi) return;  // the whole group leaves together
  const int64_t row = plan.rows_by_class[lo + idx];
  const int64_t beg = rowptr[row], end = rowptr[row + 1];
  const auto pre = epi.pre(row);
  const T rv = term.row(row);
  T s = row_sum<T, G>(term, col, beg, end, lane, rv);
  s = group_sum_first<G>(s, group_mask<G>(), lane);
  if (lane == 0) epi(row, term.finish(rv, s), pre, red);
}

template <typename T, int NRED, class Term, class Epi>
__global__ void __launch_bounds__(kRowThreads)
k_rows(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, Term term, RowPlan plan, Epi epi,
       double* __restrict__ red_partials, unsigned* red_ticket, double* red_out, const double* gate) {
  // a pass gated off (gate[0] == 0, read by every block alike) does nothing
  if (gate && *gate == 0.0) return;
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
    s = group_sum_first<32>(s, 0xffffffffu, threadIdx.x & 31);
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
      T t = threadIdx.x < kRowThreads / 32 ? sred[threadIdx.x] : T(0);
      t = group_sum_first<kRowThreads / 32>(t, 0xffffffffu, threadIdx.x);
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
  } else {
    // ---- binned rows: find the class of this block ----
    const int b = (int)(bid - plan.nchunks);
    int c = 0;
#pragma unroll
    for (int q = 1; q < kClasses; ++q) c += b >= plan.blk_off[q];
    const int64_t bb = b - plan.blk_off[c];
    switch (c) {
      case 0: class_row<T, 1>(plan, 0, bb, rowptr, col, term, epi, red); break;
      case 1: class_row<T, 2>(plan, 1, bb, rowptr, col, term, epi, red); break;
      case 2: class_row<T, 4>(plan, 2, bb, rowptr, col, term, epi, red); break;
      case 3: class_row<T, 8>(plan, 3, bb, rowptr, col, term, epi, red); break;
      case 4: class_row<T, 16>(plan, 4, bb, rowptr, col, term, epi, red); break;
      default: class_row<T, 32>(plan, 5, bb, rowptr, col, term, epi, red); break;
    }
  }
  if constexpr (NRED > 0) {
    if (grid_sum<kRowThreads, NRED>(red, red_partials, red_ticket, red_out)) epi.finish(red_out);
  }
}

template <typename T, int NRED, class Term, class Epi>
inline void launch_rows(int64_t /*n*/, const int64_t* rowptr, const int32_t* col, const Term& term,
                        const RowPlan& plan, const Epi& epi, cudaStream_t s,
                        double* red_partials = nullptr, unsigned* red_ticket = nullptr,
                        double* red_out = nullptr, const double* gate = nullptr) {
  const int grid = plan.grid();
  if (grid <= 0) return;
  k_rows<T, NRED, Term, Epi><<<grid, kRowThreads, 0, s>>>(rowptr, col, term, plan, epi, red_partials, red_ticket,
                                                          red_out, gate);
  LG_LAUNCH_CHECK();
}

// An epilogue with nothing to prefetch and nothing to reduce.
struct NoPre {};

}  // namespace lg
