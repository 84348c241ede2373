// Row-parallel CSR pass used by every SpMV-shaped kernel of the library.
//
// A pass computes, for every row i of a CSR structure,
//   s_i = finish_i( sum_k term(i, k) )
// over the row's entries, then calls an epilogue with (i, s_i). The plan
// (lg_common.cuh) bins the rows by length: a row of class c is handled by one
// aligned group of G = 2^c lanes, every lane taking about E entries, so the
// groups of a warp finish together. For G <= 8 a warp takes 32 rows, a group
// working through G of them and a reduce-scatter handing each lane one
// finished row, so the per-row work (finish, epilogue) runs on all lanes at
// once (this matters for FP64, whose narrow pipe charges an instruction its
// full warp time however few lanes are active); for G = 16, 32 the group
// reduces into its first lane. Rows longer than kChunk
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

// Loads with L1 eviction hints: the CSR arrays are read once per pass and
// should not take L1 lines from the gathered vector, whose entries (the
// high-degree vertices especially) are re-read by many rows.
__device__ __forceinline__ int32_t ld_stream(const int32_t* p) {
  int32_t v;
  asm("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ float ld_stream(const float* p) {
  float v;
  asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ double ld_stream(const double* p) {
  double v;
  asm("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ float ld_keep(const float* p) {
  float v;
  asm("ld.global.nc.L1::evict_last.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ double ld_keep(const double* p) {
  double v;
  asm("ld.global.nc.L1::evict_last.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}

// The Laplacian applied to x (Section 2.1: L = D - A, D_ii = sum_j w_ij).
// FP32: difference form, sum_j w_ij (x_i - x_j), so L 1 = 0 holds exactly.
// FP64: d_i x_i - sum_j w_ij x_j, one fused multiply-add per entry (FP64
// arithmetic is the scarce resource of the part), with d the stored row sums.
template <typename T>
struct LapTerm;

// Each term type gives row(i) (a per-row value the entry loop needs),
// acc(s, k, j, rv) (s plus the contribution of entry k with column j, as one
// fused multiply-add where there is a product) and finish(i, rv, s) (the
// row's result from its entry sum, evaluated once per row).
// Terms that gather from one vector also give src() (that vector), wload(k)
// (entry k's weight) and accw(s, wk, xj, rv) (acc from the loaded weight and
// gathered value), so the column-segmented long-row pass can issue the weight
// loads early and read xj from a staged copy.
// A null w means every weight is wc (a constant-weight operator): the pass
// then streams the column indices alone.
template <>
struct LapTerm<float> {
  const float* __restrict__ w;
  const float* __restrict__ x;
  const double* __restrict__ d;  // unused
  float wc;
  __device__ __forceinline__ float row(int64_t i) const { return __ldg(&x[i]); }
  __device__ __forceinline__ float acc(float s, int64_t k, int32_t j, float xi) const {
    return fmaf(w ? ld_stream(&w[k]) : wc, xi - ld_keep(&x[j]), s);
  }
  __device__ __forceinline__ const float* src() const { return x; }
  __device__ __forceinline__ float wload(int64_t k) const { return w ? ld_stream(&w[k]) : wc; }
  __device__ __forceinline__ float accw(float s, float wk, float xj, float xi) const { return fmaf(wk, xi - xj, s); }
  __device__ __forceinline__ float finish(int64_t, float, float s) const { return s; }
};

template <>
struct LapTerm<double> {
  const double* __restrict__ w;
  const double* __restrict__ x;
  const double* __restrict__ d;
  double wc;
  __device__ __forceinline__ double row(int64_t) const { return 0.0; }
  __device__ __forceinline__ double acc(double s, int64_t k, int32_t j, double) const {
    return fma(w ? ld_stream(&w[k]) : wc, ld_keep(&x[j]), s);
  }
  __device__ __forceinline__ const double* src() const { return x; }
  __device__ __forceinline__ double wload(int64_t k) const { return w ? ld_stream(&w[k]) : wc; }
  __device__ __forceinline__ double accw(double s, double wk, double xj, double) const { return fma(wk, xj, s); }
  __device__ __forceinline__ double finish(int64_t i, double, double s) const {
    return fma(__ldg(&d[i]), __ldg(&x[i]), -s);
  }
};

// The Laplacian term of an operator view (its weights, or its constant weight).
template <typename T, class View>
__device__ __host__ inline LapTerm<T> lap_term(const View& op, const T* x) {
  return LapTerm<T>{op.w, x, op.d, op.wc};
}

// Whether a term can be served column-segmented (it has src(), wload(), accw()).
template <class Term, class = void>
struct SegTerm {
  static constexpr bool value = false;
};
template <class Term>
struct SegTerm<Term, decltype((void)&Term::src)> {
  static constexpr bool value = true;
};

// Plain gather-sum: sum_k v[idx_k] (restriction by aggregate member lists).
template <typename T>
struct GatherTerm {
  const T* __restrict__ v;
  __device__ __forceinline__ T row(int64_t) const { return T(0); }
  __device__ __forceinline__ T acc(T s, int64_t, int32_t j, T) const { return s + __ldg(&v[j]); }
  __device__ __forceinline__ T finish(int64_t, T, T s) const { return s; }
};

// Weighted gather-sum: sum_k c_k v[idx_k] (transpose of the elimination prolongation).
template <typename T>
struct WGatherTerm {
  const T* __restrict__ c;
  const T* __restrict__ v;
  __device__ __forceinline__ T row(int64_t) const { return T(0); }
  __device__ __forceinline__ T acc(T s, int64_t k, int32_t j, T) const { return fma(__ldg(&c[k]), __ldg(&v[j]), s); }
  __device__ __forceinline__ T finish(int64_t, T, T s) const { return s; }
};

// Sum of a row's entries with G lanes, lane l taking entries l, l + G, ...
// FP64 (bound by the narrow FP64 pipe, where an instruction costs its full
// warp slot however few lanes are active): every lane of the warp runs the
// same number of steps (the warp's largest per-lane count), the steps past a
// lane's own count predicated off, so rows of different lengths in one warp
// cost the longest row's steps once, instead of an unrolled loop and a
// remainder loop that diverge; and one accumulation chain, since a second
// would cost an extra add per row. FP32 (bound by the latency of the
// gathers): four entries' loads issued together per step, two chains.
template <typename T, int G, class Term>
__device__ __forceinline__ T row_sum(const Term& term, const int32_t* __restrict__ col, int64_t beg, int64_t end,
                                     int lane, T rv) {
  if constexpr (sizeof(T) == 8) {
    const int64_t k0 = beg + lane;
    const int cnt = k0 < end ? (int)((end - k0 + G - 1) / G) : 0;
    const int steps = __reduce_max_sync(0xffffffffu, cnt);
    T s = T(0);
#pragma unroll 4
    for (int t = 0; t < steps; ++t) {
      if (t < cnt) {
        const int64_t k = k0 + (int64_t)t * G;
        s = term.acc(s, k, ld_stream(&col[k]), rv);
      }
    }
    return s;
  } else {
    T s0 = T(0), s1 = T(0);
    int64_t k = beg + lane;
    for (; k + 3 * G < end; k += 4 * G) {
      const int32_t j0 = ld_stream(&col[k]), j1 = ld_stream(&col[k + G]);
      const int32_t j2 = ld_stream(&col[k + 2 * G]), j3 = ld_stream(&col[k + 3 * G]);
      s0 = term.acc(s0, k, j0, rv);
      s1 = term.acc(s1, k + G, j1, rv);
      s0 = term.acc(s0, k + 2 * G, j2, rv);
      s1 = term.acc(s1, k + 3 * G, j3, rv);
    }
    for (; k < end; k += G) s0 = term.acc(s0, k, ld_stream(&col[k]), rv);
    return s0 + s1;
  }
}

// Rows of class G, R per group of G lanes (R divides G): the group works
// through its R rows one per round, keeping one partial sum per round. A
// recursive-halving exchange over the top log2(R) lane bits then leaves every
// lane with a partial of one row (the round given by those bits), and a tree
// over the remaining bits completes it in each of the G/R lanes of that
// subgroup; the first of them finishes the row and applies the epilogue.
// With R = G every lane finishes one row, so the per-row work (finish,
// epilogue) runs on all lanes at once, which matters for FP64, whose narrow
// pipe charges an instruction its full warp time however few lanes are
// active. Rows of round j: list entries base + j (32/G) + group.
template <typename T, int G, int R, class Term, class Epi>
__device__ __forceinline__ void class_rows_batched(const RowPlan& plan, int c, int64_t b,
                                                   const int64_t* __restrict__ rowptr,
                                                   const int32_t* __restrict__ col, const Term& term,
                                                   const Epi& epi, double* red) {
  constexpr int kGroups = 32 / G;
  constexpr int kSub = G / R;  // lanes that end up sharing one row
  const int lane = threadIdx.x & 31;
  const int grp = lane / G, gl = lane & (G - 1);
  const int64_t base = (b * (kRowThreads / 32) + (threadIdx.x >> 5)) * (kGroups * R);
  const int64_t lo = plan.cls_off[c], cnt = plan.cls_off[c + 1] - lo;
  if (base >= cnt) return;  // the whole warp leaves together
  T part[R];
#pragma unroll
  for (int j = 0; j < R; ++j) {
    // every lane takes part (row_sum steps the whole warp together); a group
    // past the end of the class sums an empty row
    const int64_t idx = base + j * kGroups + grp;
    int64_t row = 0, rb = 0, re = 0;
    if (idx < cnt) {
      row = plan.rows_by_class[lo + idx];
      rb = rowptr[row];
      re = rowptr[row + 1];
    }
    part[j] = row_sum<T, G>(term, col, rb, re, gl, term.row(row));
  }
  if constexpr (G > 1) {
    const unsigned mask = group_mask<G>();
#pragma unroll
    for (int h = G / 2, m = R; h >= kSub; h >>= 1, m >>= 1) {
      const bool upper = (gl & h) != 0;
#pragma unroll
      for (int q = 0; q < m / 2; ++q) {
        const T send = upper ? part[q] : part[q + m / 2];
        const T keep = upper ? part[q + m / 2] : part[q];
        part[q] = keep + __shfl_xor_sync(mask, send, h, G);
      }
    }
#pragma unroll
    for (int h = kSub / 2; h >= 1; h >>= 1) part[0] += __shfl_xor_sync(mask, part[0], h, G);
  }
  if (gl % kSub != 0) return;
  const int64_t idx = base + (gl / kSub) * kGroups + grp;  // the row this subgroup owns
  if (idx < cnt) {
    const int64_t row = plan.rows_by_class[lo + idx];
    const T rv = term.row(row);
    epi(row, term.finish(row, rv, part[0]), epi.pre(row), red);
  }
}

// FP64 rows of the two widest classes (one row per group of G = 16 or 32
// lanes, kRowThreads / G rows per block). Completing each row by an xor tree
// in its group and finishing it on one lane would cost about a dozen FP64
// warp instructions per row, nearly all lanes idle. Instead the groups'
// partial sums go to shared memory and one warp completes every row of the
// block: kLanes = 32 / rows lanes per row each add 8 partials (full-width
// adds), an xor tree over those kLanes lanes finishes the sum, and the
// epilogues of the block's rows run side by side.
template <typename T, int G, class Term, class Epi>
__device__ __forceinline__ void class_rows_block(const RowPlan& plan, int c, int64_t b,
                                                 const int64_t* __restrict__ rowptr,
                                                 const int32_t* __restrict__ col, const Term& term,
                                                 const Epi& epi, double* red) {
  constexpr int kRows = kRowThreads / G;  // 8 or 16
  constexpr int kLanes = 32 / kRows;      // 4 or 2 lanes complete one row
  constexpr int kPer = G / kLanes;        // 8 partials per lane
  __shared__ T sp[kRowThreads];
  const int64_t lo = plan.cls_off[c], cnt = plan.cls_off[c + 1] - lo;
  const int64_t base = b * kRows;
  if (base >= cnt) return;  // uniform over the block
  const int grp = threadIdx.x / G, gl = threadIdx.x & (G - 1);
  int64_t row = 0, rb = 0, re = 0;
  if (base + grp < cnt) {
    row = plan.rows_by_class[lo + base + grp];
    rb = rowptr[row];
    re = rowptr[row + 1];
  }
  sp[threadIdx.x] = row_sum<T, G>(term, col, rb, re, gl, term.row(row));
  __syncthreads();
  if (threadIdx.x < 32) {
    const int r = threadIdx.x / kLanes, q0 = (threadIdx.x % kLanes) * kPer;
    T s = sp[r * G + q0];
#pragma unroll
    for (int q = 1; q < kPer; ++q) s += sp[r * G + q0 + q];
#pragma unroll
    for (int o = kLanes / 2; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (q0 == 0 && base + r < cnt) {
      const int64_t rr = plan.rows_by_class[lo + base + r];
      const T rv = term.row(rr);
      epi(rr, term.finish(rr, rv, s), epi.pre(rr), red);
    }
  }
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
    T t = T(0);
    if constexpr (sizeof(T) == 8) {
      // FP64: the 256 partials through shared memory, each lane of one warp
      // adding 8 of them, then an xor tree (full-width adds throughout)
      __shared__ T sp[kRowThreads];
      sp[threadIdx.x] = s;
      __syncthreads();
      if (threadIdx.x < 32) {
        constexpr int kPer = kRowThreads / 32;
        t = sp[threadIdx.x * kPer];
#pragma unroll
        for (int q = 1; q < kPer; ++q) t += sp[threadIdx.x * kPer + q];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      }
    } else {
      s = group_sum_first<32>(s, 0xffffffffu, threadIdx.x & 31);
      if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = s;
      __syncthreads();
      if (threadIdx.x < 32) {
        t = threadIdx.x < kRowThreads / 32 ? sred[threadIdx.x] : T(0);
        t = group_sum_first<kRowThreads / 32>(t, 0xffffffffu, threadIdx.x);
      }
    }
    if (threadIdx.x < 32) {
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
          epi(row, term.finish(row, rv, tot), epi.pre(row), red);
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
      case 0: class_rows_batched<T, 1, 1>(plan, 0, bb, rowptr, col, term, epi, red); break;
      case 1: class_rows_batched<T, 2, 2>(plan, 1, bb, rowptr, col, term, epi, red); break;
      case 2: class_rows_batched<T, 4, 4>(plan, 2, bb, rowptr, col, term, epi, red); break;
      case 3: class_rows_batched<T, 8, 8>(plan, 3, bb, rowptr, col, term, epi, red); break;
      case 4:
        if constexpr (sizeof(T) == 8) class_rows_block<T, 16>(plan, 4, bb, rowptr, col, term, epi, red);
        else class_rows_batched<T, 16, 1>(plan, 4, bb, rowptr, col, term, epi, red);
        break;
      default:
        if constexpr (sizeof(T) == 8) class_rows_block<T, 32>(plan, 5, bb, rowptr, col, term, epi, red);
        else class_rows_batched<T, 32, 1>(plan, 5, bb, rowptr, col, term, epi, red);
        break;
    }
  }
  if constexpr (NRED > 0) {
    if (grid_sum<kRowThreads, NRED>(red, red_partials, red_ticket, red_out)) epi.finish(red_out);
  }
}

// Long rows, column-segmented (RowPlan::nseg_tiles > 0). Block t takes tile
// t's virtual rows, warp w the ones at w, w + 32, ... (at most 8, their
// partial sums in registers). For each segment of kSegBytes / sizeof(T)
// columns the block stages that stretch of the gathered vector in shared
// memory, then every warp advances each of its virtual rows through the
// entries whose columns fall in the segment (columns ascend within a row, so
// a per-row cursor marks where the next segment starts), lanes taking 32
// consecutive entries at a time, four such groups (columns and weights)
// loaded together; the entries of the last group past the segment's end are
// loaded again in the next segment. At the
// end each virtual row's lane partials are added by a fixed xor tree, a
// row's virtual rows in order, and the epilogue runs once per row. The order
// of every addition follows from the plan alone, so results are bitwise
// reproducible.
template <typename T, class Term, class Epi>
__global__ void __launch_bounds__(kSegThreads, 1)
k_rows_seg(const int32_t* __restrict__ col, Term term, RowPlan plan, Epi epi, const double* gate) {
  if (gate && *gate == 0.0) return;
  constexpr int kCols = kSegBytes / (int)sizeof(T);
  constexpr int kWarps = kSegThreads / 32;
  extern __shared__ __align__(16) unsigned char seg_smem[];
  T* xs = reinterpret_cast<T*>(seg_smem);
  int64_t* cur = reinterpret_cast<int64_t*>(seg_smem + kSegBytes);  // per virtual row: next entry
  T* vsum = reinterpret_cast<T*>(cur + kSegMaxVrows);               // per virtual row: its sum
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int v0 = plan.seg_tile_off[blockIdx.x], nv = plan.seg_tile_off[blockIdx.x + 1] - v0;
  for (int q = threadIdx.x; q < nv; q += kSegThreads) cur[q] = plan.vrow_beg[v0 + q];
  T part[kSegRowsPerWarp];
  T rv[kSegRowsPerWarp];
#pragma unroll
  for (int r = 0; r < kSegRowsPerWarp; ++r) {
    part[r] = T(0);
    const int q = warp + r * kWarps;
    rv[r] = q < nv ? term.row(plan.vrow_row[v0 + q]) : T(0);
  }
  const T* src = term.src();
  const int64_t ncols = plan.ncols;
  for (int64_t c0 = 0; c0 < ncols; c0 += kCols) {
    const int cn = (int)(ncols - c0 < kCols ? ncols - c0 : kCols);
    __syncthreads();  // the previous segment's reads of xs and cur are done
    for (int q = threadIdx.x; q < cn; q += kSegThreads) xs[q] = __ldg(&src[c0 + q]);
    __syncthreads();
    const int64_t bound = c0 + cn;
#pragma unroll
    for (int r = 0; r < kSegRowsPerWarp; ++r) {
      const int q = warp + r * kWarps;
      if (q >= nv) break;  // warp-uniform
      const int64_t end = plan.vrow_end[v0 + q];
      int64_t k = cur[q];
      while (k < end) {
        int32_t j[4];
        T wk[4];
        bool ok[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t e = k + u * 32 + lane;
          const bool in = e < end;
          j[u] = in ? ld_stream(&col[e]) : -1;
          wk[u] = in ? term.wload(e) : T(0);
        }
        int taken = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          // columns ascend from the cursor, so the entries in this segment are
          // a prefix of the 128; the range test also keeps every shared-memory
          // index inside the staged segment
          ok[u] = j[u] >= c0 && (int64_t)j[u] < bound;
          taken += __popc(__ballot_sync(0xffffffffu, ok[u]));
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (ok[u]) part[r] = term.accw(part[r], wk[u], xs[j[u] - c0], rv[r]);
        k += taken;
        if (taken < 128) break;  // the rest of the row lies in later segments
      }
      if (lane == 0) cur[q] = k;
    }
  }
  // each virtual row's sum: a fixed xor tree over the lanes
#pragma unroll
  for (int r = 0; r < kSegRowsPerWarp; ++r) {
    T v = part[r];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int q = warp + r * kWarps;
    if (lane == 0 && q < nv) vsum[q] = v;
  }
  __syncthreads();
  // a row's virtual rows are consecutive within the tile: the first of them adds them in order
  double red[1] = {0.0};
  for (int q = threadIdx.x; q < nv; q += kSegThreads) {
    const int32_t row = plan.vrow_row[v0 + q];
    if (q > 0 && plan.vrow_row[v0 + q - 1] == row) continue;
    T tot = vsum[q];
    for (int u = q + 1; u < nv && plan.vrow_row[v0 + u] == row; ++u) tot += vsum[u];
    const T rvr = term.row(row);
    epi(row, term.finish(row, rvr, tot), epi.pre(row), red);
  }
}

template <typename T, class Term, class Epi>
inline void launch_seg(const int32_t* col, const Term& term, const RowPlan& plan, const Epi& epi, cudaStream_t s,
                       const double* gate) {
  constexpr size_t smem = kSegBytes + kSegMaxVrows * (sizeof(int64_t) + sizeof(T));
  static const cudaError_t attr = cudaFuncSetAttribute(k_rows_seg<T, Term, Epi>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  check_cuda(attr, "cudaFuncSetAttribute(k_rows_seg)");
  k_rows_seg<T, Term, Epi><<<plan.nseg_tiles, kSegThreads, smem, s>>>(col, term, plan, epi, gate);
  LG_LAUNCH_CHECK();
}

template <typename T, int NRED, class Term, class Epi>
inline void launch_rows(int64_t /*n*/, const int64_t* rowptr, const int32_t* col, const Term& term,
                        const RowPlan& plan, const Epi& epi, cudaStream_t s,
                        double* red_partials = nullptr, unsigned* red_ticket = nullptr,
                        double* red_out = nullptr, const double* gate = nullptr) {
  if constexpr (NRED == 0 && SegTerm<Term>::value) {
    if (plan.nseg_tiles > 0) {
      // the long rows column-segmented, then the binned rows (no chunks)
      launch_seg<T>(col, term, plan, epi, s, gate);
      RowPlan rest = plan;
      rest.nchunks = 0;
      const int grid = rest.grid();
      if (grid > 0) {
        k_rows<T, NRED, Term, Epi><<<grid, kRowThreads, 0, s>>>(rowptr, col, term, rest, epi, red_partials,
                                                                red_ticket, red_out, gate);
        LG_LAUNCH_CHECK();
      }
      return;
    }
  }
  const int grid = plan.grid();
  if (grid <= 0) return;
  k_rows<T, NRED, Term, Epi><<<grid, kRowThreads, 0, s>>>(rowptr, col, term, plan, epi, red_partials, red_ticket,
                                                          red_out, gate);
  LG_LAUNCH_CHECK();
}

// An epilogue with nothing to prefetch and nothing to reduce.
struct NoPre {};

}  // namespace lg
