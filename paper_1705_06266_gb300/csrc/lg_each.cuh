// A visitor over the rows of a CSR structure, for the setup passes
// (validation, connectivity, strength of connection, aggregation voting,
// entry counting and emission).
//
// Rows are taken from length bins (RowBins, lg_prims.h): a row of class c is
// visited by an aligned group of 2^c lanes, each lane taking every 2^c-th
// entry, so short rows (the bulk of a power-law graph) do not leave most of a
// warp idle; a row longer than kChunk entries is visited by a whole block.
// The per-row partial states of the lanes are combined by an xor tree over
// the group (then over the warps of the block, in warp order), so every
// combination happens in an order fixed by the row length, and the row is
// finished by one lane.
//
// A functor F gives
//   using Acc = ...;                                   per-lane row state (trivially copyable)
//   Acc  init(int64_t row, int64_t beg, int64_t end)   identity of merge plus per-row constants
//   void add(Acc&, int64_t row, int64_t k)             entry k of the row
//   void merge(Acc&, const Acc&)                       combine partial states
//   Acc  shfl(const Acc&, int o)                       __shfl_xor_sync over the full warp by o
//   long long finish(int64_t row, const Acc&, int64_t beg, int64_t end)
// finish runs once per row; its return values are summed over all rows into
// *total (when given) with one atomic add per block.
#pragma once

#include "lg_prims.h"

namespace lg {

template <int G, class F>
__device__ __forceinline__ long long each_group(const F& f, const int64_t* __restrict__ rowptr, const RowBins& b,
                                                int c, int64_t bb) {
  constexpr int kPer = kEachThreads / G;
  const int64_t idx = b.off[c] + bb * kPer + threadIdx.x / G;
  const bool valid = idx < b.off[c + 1];
  const int gl = threadIdx.x & (G - 1);
  int64_t row = 0, beg = 0, end = 0;
  if (valid) {
    row = b.rows[idx];
    beg = rowptr[row];
    end = rowptr[row + 1];
  }
  typename F::Acc a = f.init(row, beg, end);
  for (int64_t k = beg + gl; k < end; k += G) f.add(a, row, k);
  if constexpr (G > 1) {
#pragma unroll
    for (int o = G / 2; o >= 1; o >>= 1) f.merge(a, f.shfl(a, o));
  }
  return (valid && gl == 0) ? f.finish(row, a, beg, end) : 0ll;
}

template <class F>
__device__ __forceinline__ long long each_long(const F& f, const int64_t* __restrict__ rowptr, int64_t row) {
  using Acc = typename F::Acc;
  __shared__ __align__(16) unsigned char raw[(kEachThreads / 32) * sizeof(Acc)];
  Acc* sm = reinterpret_cast<Acc*>(raw);
  const int64_t beg = rowptr[row], end = rowptr[row + 1];
  Acc a = f.init(row, beg, end);
  for (int64_t k = beg + threadIdx.x; k < end; k += kEachThreads) f.add(a, row, k);
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) f.merge(a, f.shfl(a, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = a;
  __syncthreads();
  long long t = 0;
  if (threadIdx.x == 0) {
    for (int w = 1; w < kEachThreads / 32; ++w) f.merge(a, sm[w]);
    t = f.finish(row, a, beg, end);
  }
  return t;
}

template <class F>
__global__ void __launch_bounds__(kEachThreads)
k_each(F f, const int64_t* __restrict__ rowptr, RowBins b, unsigned long long* total) {
  const int bid = blockIdx.x;
  const int64_t nlong = b.off[kClasses + 1] - b.off[kClasses];
  long long t = 0;
  if (bid < nlong) {
    t = each_long(f, rowptr, b.rows[b.off[kClasses] + bid]);
  } else {
    // class blocks run from the longest class down: class c owns [blk[c], blk[c-1])
    int c = 0;
#pragma unroll
    for (int q = 0; q < kClasses - 1; ++q) c += bid < b.blk[q];
    const int64_t bb = bid - b.blk[c];
    switch (c) {
      case 0: t = each_group<1>(f, rowptr, b, 0, bb); break;
      case 1: t = each_group<2>(f, rowptr, b, 1, bb); break;
      case 2: t = each_group<4>(f, rowptr, b, 2, bb); break;
      case 3: t = each_group<8>(f, rowptr, b, 3, bb); break;
      case 4: t = each_group<16>(f, rowptr, b, 4, bb); break;
      default: t = each_group<32>(f, rowptr, b, 5, bb); break;
    }
  }
  if (total) {
    __shared__ long long wsum[kEachThreads / 32];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      long long s = 0;
      for (int w = 0; w < kEachThreads / 32; ++w) s += wsum[w];
      if (s) atomicAdd(total, (unsigned long long)s);
    }
  }
}

template <class F>
inline void each_row(const F& f, const int64_t* rowptr, const RowBins& b, cudaStream_t s,
                     unsigned long long* total = nullptr) {
  if (b.grid <= 0) return;
  k_each<F><<<b.grid, kEachThreads, 0, s>>>(f, rowptr, b, total);
  LG_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// Emission: each row writes its kept entries contiguously, in entry order,
// from position off[row] (an exclusive scan of the kept counts). A group
// walks its row G entries at a time, every lane of the group taking the same
// number of steps, and ranks the kept entries of a step by a ballot over the
// group's lanes. A functor E gives
//   using Row = ...;                                   per-row constants
//   Row  row(int64_t i)
//   bool special(const Row&)                           row emitted by emit_special instead
//   void emit_special(const Row&, int64_t i, int64_t beg, int64_t end, int64_t pos)   (one lane)
//   bool take(const Row&, int64_t i, int64_t k)        keep entry k?
//   void put(const Row&, int64_t i, int64_t k, int64_t pos)
// ---------------------------------------------------------------------------
template <int G, class E>
__device__ __forceinline__ void emit_group(const E& e, const int64_t* __restrict__ rowptr,
                                           const int64_t* __restrict__ off, const RowBins& b, int c, int64_t bb) {
  constexpr int kPer = kEachThreads / G;
  const int64_t idx = b.off[c] + bb * kPer + threadIdx.x / G;
  if (idx >= b.off[c + 1]) return;  // whole groups leave together
  const int gl = threadIdx.x & (G - 1);
  const int64_t i = b.rows[idx];
  const int64_t beg = rowptr[i], end = rowptr[i + 1];
  const typename E::Row r = e.row(i);
  int64_t pos = off[i];
  if (e.special(r)) {
    if (gl == 0) e.emit_special(r, i, beg, end, pos);
    return;
  }
  const unsigned gmask = group_mask<G>();
  const unsigned below = (1u << (threadIdx.x & 31)) - 1u;
  for (int64_t k0 = beg; k0 < end; k0 += G) {
    const int64_t k = k0 + gl;
    const bool t = k < end && e.take(r, i, k);
    const unsigned m = __ballot_sync(gmask, t) & gmask;
    if (t) e.put(r, i, k, pos + __popc(m & below));
    pos += __popc(m);
  }
}

template <class E>
__device__ __forceinline__ void emit_long(const E& e, const int64_t* __restrict__ rowptr,
                                          const int64_t* __restrict__ off, int64_t i) {
  __shared__ int wcount[kEachThreads / 32];
  const int64_t beg = rowptr[i], end = rowptr[i + 1];
  const typename E::Row r = e.row(i);
  int64_t pos = off[i];
  if (e.special(r)) {  // uniform over the block
    if (threadIdx.x == 0) e.emit_special(r, i, beg, end, pos);
    return;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned below = (1u << lane) - 1u;
  for (int64_t k0 = beg; k0 < end; k0 += kEachThreads) {
    const int64_t k = k0 + threadIdx.x;
    const bool t = k < end && e.take(r, i, k);
    const unsigned m = __ballot_sync(0xffffffffu, t);
    if (lane == 0) wcount[warp] = __popc(m);
    __syncthreads();
    int64_t before = 0, all = 0;
    for (int q = 0; q < kEachThreads / 32; ++q) {
      before += q < warp ? wcount[q] : 0;
      all += wcount[q];
    }
    if (t) e.put(r, i, k, pos + before + __popc(m & below));
    pos += all;
    __syncthreads();
  }
}

template <class E>
__global__ void __launch_bounds__(kEachThreads)
k_emit(E e, const int64_t* __restrict__ rowptr, const int64_t* __restrict__ off, RowBins b) {
  const int bid = blockIdx.x;
  const int64_t nlong = b.off[kClasses + 1] - b.off[kClasses];
  if (bid < nlong) {
    emit_long(e, rowptr, off, b.rows[b.off[kClasses] + bid]);
    return;
  }
  int c = 0;
#pragma unroll
  for (int q = 0; q < kClasses - 1; ++q) c += bid < b.blk[q];
  const int64_t bb = bid - b.blk[c];
  switch (c) {
    case 0: emit_group<1>(e, rowptr, off, b, 0, bb); break;
    case 1: emit_group<2>(e, rowptr, off, b, 1, bb); break;
    case 2: emit_group<4>(e, rowptr, off, b, 2, bb); break;
    case 3: emit_group<8>(e, rowptr, off, b, 3, bb); break;
    case 4: emit_group<16>(e, rowptr, off, b, 4, bb); break;
    default: emit_group<32>(e, rowptr, off, b, 5, bb); break;
  }
}

template <class E>
inline void emit_rows(const E& e, const int64_t* rowptr, const int64_t* off, const RowBins& b, cudaStream_t s) {
  if (b.grid <= 0) return;
  k_emit<E><<<b.grid, kEachThreads, 0, s>>>(e, rowptr, off, b);
  LG_LAUNCH_CHECK();
}

// xor shuffles of the common field types, for the functors' shfl.
__device__ __forceinline__ double each_shfl(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ long long each_shfl(long long v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ int each_shfl(int v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ unsigned long long each_shfl(unsigned long long v, int o) {
  return __shfl_xor_sync(0xffffffffu, v, o);
}

}  // namespace lg
