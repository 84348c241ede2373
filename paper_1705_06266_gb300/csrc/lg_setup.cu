// Setup of the multigrid hierarchy on the device (Sections 3.4-3.6, 4).
//
// Every stage is a set of kernels over the current level's CSR; the host only
// reads back counts (|F|, number of aggregates, entries of the next level) to
// size the next allocations, and at the end the per-level eigenvalue
// estimates for the Chebyshev constants.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "lg_hier.h"
#include "lg_each.cuh"
#include "lg_rows.cuh"

namespace lg {

constexpr int kNT = 256;

static inline int blocks_for(int64_t n, int per_block = kNT) { return grid_for(n, per_block, kSMs * 16); }

#define LG_GRID_STRIDE(i, n) \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// Device error word bits.
enum : int {
  kErrRowptr = 1, kErrCol = 2, kErrSelf = 4, kErrOrder = 8, kErrWeight = 16, kErrAsym = 32, kErrLoop = 64
};

// ---------------------------------------------------------------------------
// Input contract (Section 2.1): positive weights, undirected, connected.
// ---------------------------------------------------------------------------
__global__ void k_check_rowptr(int64_t n, int64_t nnz, const int64_t* __restrict__ rowptr, int* err) {
  LG_GRID_STRIDE(i, n + 1) {
    const int64_t v = rowptr[i];
    bool bad = (v < 0 || v > nnz) || (i == 0 && v != 0) || (i == n && v != nnz) || (i < n && rowptr[i + 1] < v);
    if (bad) atomicOr(err, kErrRowptr);
  }
}

__device__ __forceinline__ bool find_col(const int64_t* rowptr, const int32_t* col, int64_t row, int32_t key,
                                         int64_t* pos) {
  int64_t lo = rowptr[row], hi = rowptr[row + 1] - 1;
  while (lo <= hi) {
    int64_t mid = lo + ((hi - lo) >> 1);
    int32_t c = col[mid];
    if (c == key) { *pos = mid; return true; }
    if (c < key) lo = mid + 1; else hi = mid - 1;
  }
  return false;
}

// Per-entry checks of one row: column range, no self-loop, strictly
// increasing columns (so no duplicates), positive finite weight, and the
// mirror entry. The mirror of (i, j) is looked up only from the end with more
// entries (ties: larger id), by binary search in the row of the other end,
// which keeps the searches short on power-law graphs; the looked-up entries
// count +1 and the others -1, and a zero total (every entry either looked up
// or the mirror of one) completes the symmetry check: the looked-up entries
// map one-to-one onto the others, so equal counts leave no entry unmatched.
struct FCheck {
  int64_t n;
  const int64_t* __restrict__ rowptr;
  const int32_t* __restrict__ col;
  const double* __restrict__ w;
  int* err;
  struct Acc {
    long long sign;
    int bits;
  };
  __device__ Acc init(int64_t, int64_t, int64_t) const { return Acc{0, 0}; }
  __device__ void add(Acc& a, int64_t i, int64_t k) const {
    const int32_t j = col[k];
    if (j < 0 || j >= n) { a.bits |= kErrCol; return; }
    if (j == i) { a.bits |= kErrSelf; return; }
    const int64_t b = rowptr[i], di = rowptr[i + 1] - b;
    if (k > b && col[k - 1] >= j) a.bits |= kErrOrder;
    const double wk = w[k];
    if (!(wk > 0.0) || !isfinite(wk)) a.bits |= kErrWeight;
    const int64_t dj = rowptr[j + 1] - rowptr[j];
    if (dj < di || (dj == di && j < i)) {
      int64_t pos;
      if (!find_col(rowptr, col, j, (int32_t)i, &pos) || w[pos] != wk) a.bits |= kErrAsym;
      a.sign += 1;
    } else {
      a.sign -= 1;
    }
  }
  __device__ void merge(Acc& a, const Acc& o) const {
    a.sign += o.sign;
    a.bits |= o.bits;
  }
  __device__ Acc shfl(const Acc& a, int o) const { return Acc{each_shfl(a.sign, o), each_shfl(a.bits, o)}; }
  __device__ long long finish(int64_t, const Acc& a, int64_t, int64_t) const {
    if (a.bits) atomicOr(err, a.bits);
    return a.sign;
  }
};

// Connected components by union-find with lock-free hooking (the larger root
// is hooked under the smaller one by compare-and-swap) and path halving.
// Every loop is bounded; a loop that runs out sets kErrLoop.
__device__ __forceinline__ int32_t cc_find(int32_t* parent, int32_t x, int64_t n, int* err) {
  for (int64_t guard = 0; guard <= n; ++guard) {
    int32_t p = parent[x];
    if (p == x) return x;
    int32_t gp = parent[p];
    if (gp != p) parent[x] = gp;
    x = gp;
  }
  atomicOr(err, kErrLoop);
  return x;
}

__global__ void k_cc_init(int64_t n, int32_t* parent) {
  LG_GRID_STRIDE(i, n) parent[i] = (int32_t)i;
}

// Union of the two ends of every entry (i, j), j > i.
struct FHook {
  int64_t n;
  const int32_t* __restrict__ col;
  int32_t* parent;
  int* err;
  struct Acc {
    int z;
  };
  __device__ Acc init(int64_t, int64_t, int64_t) const { return Acc{0}; }
  __device__ void add(Acc&, int64_t i, int64_t k) const {
    const int32_t j = col[k];
    if (j <= i) return;
    int32_t a = cc_find(parent, (int32_t)i, n, err), b = cc_find(parent, j, n, err);
    int tries = 0;
    while (a != b) {
      const int32_t hi = a > b ? a : b, lo = a > b ? b : a;
      const int32_t old = atomicCAS(&parent[hi], hi, lo);
      if (old == hi) break;
      a = cc_find(parent, old, n, err);
      b = cc_find(parent, lo, n, err);
      if (++tries > (1 << 20)) {
        atomicOr(err, kErrLoop);
        break;
      }
    }
  }
  __device__ void merge(Acc&, const Acc&) const {}
  __device__ Acc shfl(const Acc& a, int) const { return a; }
  __device__ long long finish(int64_t, const Acc&, int64_t, int64_t) const { return 0; }
};

__global__ void k_cc_roots(int64_t n, int32_t* parent, uint8_t* is_root, int* err) {
  LG_GRID_STRIDE(i, n) {
    const int32_t r = cc_find(parent, (int32_t)i, n, err);
    is_root[i] = (r == i);
  }
}

// ---------------------------------------------------------------------------
// Diagonal: d_i = sum_j w_ij, stored as 1/d_i (0 for an isolated vertex).
// ---------------------------------------------------------------------------
struct WeightTerm {
  const double* __restrict__ w;
  __device__ __forceinline__ double row(int64_t) const { return 0.0; }
  __device__ __forceinline__ double acc(double s, int64_t k, int32_t, double) const { return s + w[k]; }
  __device__ __forceinline__ double finish(int64_t, double, double s) const { return s; }
};
struct EpiDinv {
  double* d;
  double* dinv;
  __device__ __forceinline__ NoPre pre(int64_t) const { return NoPre{}; }
  __device__ __forceinline__ void operator()(int64_t i, double s, NoPre, double*) const {
    d[i] = s;
    dinv[i] = s > 0.0 ? 1.0 / s : 0.0;
  }
  __device__ void finish(const double*) const {}
};

// y = L x.
template <typename T>
struct EpiStore {
  T* y;
  __device__ __forceinline__ NoPre pre(int64_t) const { return NoPre{}; }
  __device__ __forceinline__ void operator()(int64_t i, T s, NoPre, double*) const { y[i] = s; }
  __device__ void finish(const double*) const {}
};

// ---------------------------------------------------------------------------
// Low-degree elimination (Section 3.4, Algorithm 2): candidates are vertices
// of degree <= max_degree; each candidate's value is hash(i) (SplitMix64 output i), others +infinity
// (UINT64_MAX); z_i = min over the closed neighbourhood; i goes iff it is a
// candidate and z_i = hash(i).
// ---------------------------------------------------------------------------
__global__ void k_elim_hash(int64_t n, const int64_t* __restrict__ rowptr, int max_degree, uint64_t seed,
                            uint64_t* __restrict__ hc) {
  LG_GRID_STRIDE(i, n) {
    const int64_t deg = rowptr[i + 1] - rowptr[i];
    hc[i] = deg <= max_degree ? splitmix64(seed, rng_counter(kStreamHash, 0, i)) : ~0ull;
  }
}

__global__ void k_elim_select(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                              int max_degree, const uint64_t* __restrict__ hc, uint8_t* __restrict__ is_f) {
  LG_GRID_STRIDE(i, n) {
    const int64_t b = rowptr[i], e = rowptr[i + 1];
    uint8_t f = 0;
    if (e - b <= max_degree) {
      const uint64_t hi = hc[i];
      uint64_t z = hi;
      for (int64_t k = b; k < e; ++k) {
        const uint64_t hj = hc[col[k]];
        z = hj < z ? hj : z;
      }
      f = (z == hi);
    }
    is_f[i] = f;
  }
}

__global__ void k_not(int64_t n, const uint8_t* __restrict__ a, uint8_t* __restrict__ b) {
  LG_GRID_STRIDE(i, n) b[i] = a[i] ? 0 : 1;
}

// cmap: kept vertex -> coarse id (ascending), eliminated -> -1; cfine inverse.
__global__ void k_elim_maps(int64_t n, const uint8_t* __restrict__ is_f, const int64_t* __restrict__ cid,
                            int32_t* __restrict__ cmap, int32_t* __restrict__ cfine) {
  LG_GRID_STRIDE(i, n) {
    if (is_f[i]) {
      cmap[i] = -1;
    } else {
      cmap[i] = (int32_t)cid[i];
      cfine[cid[i]] = (int32_t)i;
    }
  }
}

// Entries of the Schur complement generated by each fine row: a kept row
// gives its kept neighbours (L_CC); an eliminated row f of degree d gives
// the d(d-1) ordered pairs of its neighbours (the fill of
// -L_FC^T L_FF^-1 L_FC; F is independent, so all neighbours are kept).
struct FSchurCount {
  const int32_t* __restrict__ col;
  const uint8_t* __restrict__ is_f;
  int64_t* __restrict__ cnt;
  struct Acc {
    long long c;
  };
  __device__ Acc init(int64_t, int64_t, int64_t) const { return Acc{0}; }
  __device__ void add(Acc& a, int64_t, int64_t k) const { a.c += is_f[col[k]] ? 0 : 1; }
  __device__ void merge(Acc& a, const Acc& o) const { a.c += o.c; }
  __device__ Acc shfl(const Acc& a, int o) const { return Acc{each_shfl(a.c, o)}; }
  __device__ long long finish(int64_t i, const Acc& a, int64_t b, int64_t e) const {
    cnt[i] = is_f[i] ? (e - b) * (e - b - 1) : a.c;
    return 0;
  }
};

// Entries of the Schur complement per kept row a, for the emission grouped by
// row (k_schur_emit_rows): a's kept neighbours, plus deg(f) - 1 fill entries
// for each eliminated neighbour f (F is independent, so f's other neighbours
// are kept). Eliminated rows emit nothing.
struct FSchurCountRows {
  const int64_t* __restrict__ rowptr;
  const int32_t* __restrict__ col;
  const uint8_t* __restrict__ is_f;
  int64_t* __restrict__ cnt;
  struct Acc {
    long long c;
  };
  __device__ Acc init(int64_t, int64_t, int64_t) const { return Acc{0}; }
  __device__ void add(Acc& a, int64_t, int64_t k) const {
    const int32_t j = col[k];
    a.c += is_f[j] ? rowptr[j + 1] - rowptr[j] - 1 : 1;
  }
  __device__ void merge(Acc& a, const Acc& o) const { a.c += o.c; }
  __device__ Acc shfl(const Acc& a, int o) const { return Acc{each_shfl(a.c, o)}; }
  __device__ long long finish(int64_t i, const Acc& a, int64_t, int64_t) const {
    cnt[i] = is_f[i] ? 0 : a.c;
    return 0;
  }
};

// The same entries as ESchur, emitted by kept row a into a's own range, so
// that they come grouped by coarse row. Within the row, the order reproduces
// the global stable sort's ties: contributions to one key come in the order
// of the fine row that ESchur emits them from, i.e. the fill of each
// eliminated neighbour f < a (in a's row order), then a's own entries, then
// the fill of each f > a. Fill values are computed from f's row exactly as
// ESchur does (d_f summed in f's row order, w_fa w_fy / d_f). Rows are taken
// from the length bins: a group of 2^c lanes per row, a whole block for rows
// above kChunk entries (a hub's row must not serialise on one warp).
struct SchurRows {
  const int64_t* __restrict__ rowptr;
  const int32_t* __restrict__ col;
  const double* __restrict__ w;
  const uint8_t* __restrict__ is_f;
  const int32_t* __restrict__ cmap;
  const int64_t* __restrict__ off;
  int cbits;
  uint64_t* __restrict__ keys;
  uint64_t* __restrict__ vals;

  // entry k of kept row a: its counts in the three parts (fill before a, own, fill after a)
  __device__ __forceinline__ void counts(int64_t a, int64_t k, int64_t e, long long& clt, long long& cown,
                                         long long& cgt) const {
    clt = cown = cgt = 0;
    if (k >= e) return;
    const int32_t j = col[k];
    if (is_f[j]) {
      const long long c = rowptr[j + 1] - rowptr[j] - 1;
      (j < a ? clt : cgt) = c;
    } else {
      cown = 1;
    }
  }
  // writes entry k's contribution at p (own) or from p on (fill)
  __device__ __forceinline__ void emit(int64_t a, int64_t k, int64_t p) const {
    const int32_t j = col[k];
    const uint64_t rowkey = (uint64_t)cmap[a] << cbits;
    if (!is_f[j]) {
      keys[p] = rowkey | (uint64_t)cmap[j];
      vals[p] = (uint64_t)__double_as_longlong(w[k]);
      return;
    }
    const int64_t fb = rowptr[j], fe = rowptr[j + 1];
    double df = 0.0, wfa = 0.0;
    for (int64_t q = fb; q < fe; ++q) {
      df += w[q];
      if (col[q] == (int32_t)a) wfa = w[q];
    }
    for (int64_t q = fb; q < fe; ++q) {
      if (col[q] == (int32_t)a) continue;
      keys[p] = rowkey | (uint64_t)cmap[col[q]];
      vals[p] = (uint64_t)__double_as_longlong(wfa * w[q] / df);
      ++p;
    }
  }
};

// inclusive scan of three counts over the G lanes of a group (lane order)
template <int G>
__device__ __forceinline__ void scan3(long long& x, long long& y, long long& z, int gl, unsigned mask) {
#pragma unroll
  for (int o = 1; o < G; o <<= 1) {
    const long long px = __shfl_up_sync(mask, x, o, G), py = __shfl_up_sync(mask, y, o, G),
                    pz = __shfl_up_sync(mask, z, o, G);
    if (gl >= o) {
      x += px;
      y += py;
      z += pz;
    }
  }
}

template <int G>
__device__ __forceinline__ void schur_group(const SchurRows& S, const RowBins& b, int c, int64_t bb) {
  constexpr int kPer = kEachThreads / G;
  const int64_t idx = b.off[c] + bb * kPer + threadIdx.x / G;
  if (idx >= b.off[c + 1]) return;  // whole groups leave together
  const int64_t a = b.rows[idx];
  if (S.is_f[a]) return;
  const int gl = threadIdx.x & (G - 1);
  const unsigned mask = group_mask<G>();
  const int64_t beg = S.rowptr[a], end = S.rowptr[a + 1];
  long long nlt = 0, nown = 0;
  for (int64_t k0 = beg; k0 < end; k0 += G) {
    long long x, y, z;
    S.counts(a, k0 + gl, end, x, y, z);
    scan3<G>(x, y, z, gl, mask);
    nlt += __shfl_sync(mask, x, G - 1, G);
    nown += __shfl_sync(mask, y, G - 1, G);
  }
  int64_t plt = S.off[a], pown = plt + nlt, pgt = pown + nown;
  for (int64_t k0 = beg; k0 < end; k0 += G) {
    const int64_t k = k0 + gl;
    long long cx, cy, cz;
    S.counts(a, k, end, cx, cy, cz);
    long long x = cx, y = cy, z = cz;
    scan3<G>(x, y, z, gl, mask);
    if (k < end) {
      if (cy) S.emit(a, k, pown + y - 1);
      else if (cx) S.emit(a, k, plt + x - cx);
      else if (cz) S.emit(a, k, pgt + z - cz);
    }
    plt += __shfl_sync(mask, x, G - 1, G);
    pown += __shfl_sync(mask, y, G - 1, G);
    pgt += __shfl_sync(mask, z, G - 1, G);
  }
}

// A long row with the whole block: warp scans, then the warps' totals in order.
__device__ __forceinline__ void schur_long(const SchurRows& S, int64_t a) {
  __shared__ long long wt[3][kEachThreads / 32];
  if (S.is_f[a]) return;  // uniform over the block
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t beg = S.rowptr[a], end = S.rowptr[a + 1];
  const auto block_scan = [&](long long& x, long long& y, long long& z, long long& tx, long long& ty,
                              long long& tz) {
    scan3<32>(x, y, z, lane, 0xffffffffu);
    if (lane == 31) {
      wt[0][warp] = x;
      wt[1][warp] = y;
      wt[2][warp] = z;
    }
    __syncthreads();
    long long bx = 0, by = 0, bz = 0;
    tx = ty = tz = 0;
    for (int q = 0; q < kEachThreads / 32; ++q) {
      if (q < warp) {
        bx += wt[0][q];
        by += wt[1][q];
        bz += wt[2][q];
      }
      tx += wt[0][q];
      ty += wt[1][q];
      tz += wt[2][q];
    }
    x += bx;
    y += by;
    z += bz;
    __syncthreads();  // wt is reused by the next step
  };
  long long nlt = 0, nown = 0;
  for (int64_t k0 = beg; k0 < end; k0 += kEachThreads) {
    long long x, y, z, tx, ty, tz;
    S.counts(a, k0 + threadIdx.x, end, x, y, z);
    block_scan(x, y, z, tx, ty, tz);
    nlt += tx;
    nown += ty;
  }
  int64_t plt = S.off[a], pown = plt + nlt, pgt = pown + nown;
  for (int64_t k0 = beg; k0 < end; k0 += kEachThreads) {
    const int64_t k = k0 + threadIdx.x;
    long long cx, cy, cz, tx, ty, tz;
    S.counts(a, k, end, cx, cy, cz);
    long long x = cx, y = cy, z = cz;
    block_scan(x, y, z, tx, ty, tz);
    if (k < end) {
      if (cy) S.emit(a, k, pown + y - 1);
      else if (cx) S.emit(a, k, plt + x - cx);
      else if (cz) S.emit(a, k, pgt + z - cz);
    }
    plt += tx;
    pown += ty;
    pgt += tz;
  }
}

__global__ void __launch_bounds__(kEachThreads) k_schur_emit_rows(SchurRows S, RowBins b) {
  const int bid = blockIdx.x;
  const int64_t nlong = b.off[kClasses + 1] - b.off[kClasses];
  if (bid < nlong) {
    schur_long(S, b.rows[b.off[kClasses] + bid]);
    return;
  }
  int c = 0;
#pragma unroll
  for (int q = 0; q < kClasses - 1; ++q) c += bid < b.blk[q];
  const int64_t bb = bid - b.blk[c];
  switch (c) {
    case 0: schur_group<1>(S, b, 0, bb); break;
    case 1: schur_group<2>(S, b, 1, bb); break;
    case 2: schur_group<4>(S, b, 2, bb); break;
    case 3: schur_group<8>(S, b, 3, bb); break;
    case 4: schur_group<16>(S, b, 4, bb); break;
    default: schur_group<32>(S, b, 5, bb); break;
  }
}

// Keys are (coarse row << cbits) | coarse col; values are FP64 bit patterns.
// Entries are written in fine-row order, kept rows in column order, fill in
// (first neighbour, second neighbour) order, so the sort-and-sum that follows
// adds equal keys in a fixed order. The fill weight is w_fa w_fb / d_f with
// d_f = sum_j w_fj summed sequentially.
struct ESchur {
  const int32_t* __restrict__ col;
  const double* __restrict__ w;
  const uint8_t* __restrict__ is_f;
  const int32_t* __restrict__ cmap;
  int cbits;
  uint64_t* __restrict__ keys;
  uint64_t* __restrict__ vals;
  struct Row {
    unsigned long long key;
    bool f;
  };
  __device__ Row row(int64_t i) const {
    const bool f = is_f[i];
    return Row{f ? 0ull : (unsigned long long)cmap[i] << cbits, f};
  }
  __device__ bool special(const Row& r) const { return r.f; }
  __device__ void emit_special(const Row&, int64_t, int64_t b, int64_t e, int64_t o) const {
    const int64_t d = e - b;
    double df = 0.0;
    for (int64_t k = b; k < e; ++k) df += w[k];
    int64_t t = 0;
    for (int64_t ka = b; ka < e; ++ka)
      for (int64_t kb = b; kb < e; ++kb) {
        if (kb == ka) continue;
        keys[o + t] = ((uint64_t)cmap[col[ka]] << cbits) | (uint64_t)cmap[col[kb]];
        vals[o + t] = (uint64_t)__double_as_longlong(w[ka] * w[kb] / df);
        ++t;
      }
    (void)d;
  }
  __device__ bool take(const Row&, int64_t, int64_t k) const { return !is_f[col[k]]; }
  __device__ void put(const Row& r, int64_t, int64_t k, int64_t p) const {
    keys[p] = r.key | (uint64_t)cmap[col[k]];
    vals[p] = (uint64_t)__double_as_longlong(w[k]);
  }
};

__global__ void k_pt_emit(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                          const uint8_t* __restrict__ is_f, const int32_t* __restrict__ cmap,
                          const int64_t* __restrict__ off, uint64_t* __restrict__ keys, uint64_t* __restrict__ vals) {
  LG_GRID_STRIDE(i, n) {
    if (!is_f[i]) continue;
    const int64_t b = rowptr[i], e = rowptr[i + 1];
    const int64_t o = off[i];
    for (int64_t k = b; k < e; ++k) {
      keys[o + (k - b)] = (uint64_t)cmap[col[k]];
      vals[o + (k - b)] = ((uint64_t)i << 32) | (uint64_t)(k - b);
    }
  }
}

__global__ void k_f_degree(int64_t n, const int64_t* __restrict__ rowptr, const uint8_t* __restrict__ is_f,
                           int64_t* __restrict__ cnt) {
  LG_GRID_STRIDE(i, n) cnt[i] = is_f[i] ? rowptr[i + 1] - rowptr[i] : 0;
}

__global__ void k_pt_fill(int64_t m, const uint64_t* __restrict__ vals, const int64_t* __restrict__ rowptr,
                          const double* __restrict__ w, int32_t* __restrict__ pt_f, double* __restrict__ pt_coef) {
  LG_GRID_STRIDE(q, m) {
    const int64_t f = (int64_t)(vals[q] >> 32), slot = (int64_t)(vals[q] & 0xffffffffu);
    const int64_t b = rowptr[f], e = rowptr[f + 1];
    double df = 0.0;
    for (int64_t k = b; k < e; ++k) df += w[k];
    pt_f[q] = (int32_t)f;
    pt_coef[q] = w[b + slot] / df;
  }
}

// rowptr of a CSR whose entries are sorted by row (row = key >> shift).
__global__ void k_rowptr_sorted(const uint64_t* __restrict__ keys, int64_t m, int shift, int64_t nrows,
                                int64_t* __restrict__ rowptr) {
  LG_GRID_STRIDE(r, nrows + 1) {
    int64_t lo = 0, hi = m;
    while (lo < hi) {
      int64_t mid = (lo + hi) >> 1;
      if ((int64_t)(keys[mid] >> shift) < r) lo = mid + 1; else hi = mid;
    }
    rowptr[r] = lo;
  }
}

// ---------------------------------------------------------------------------
// Strength of connection (Section 3.5).
// ---------------------------------------------------------------------------
constexpr int kMaxVecs = 8;

__global__ void k_strength_init(int64_t n, int m, uint64_t seed, int level, double* __restrict__ y) {
  LG_GRID_STRIDE(i, n) {
    for (int k = 0; k < m; ++k) y[i * m + k] = uniform_pm1(seed, 1 + k, level, i);
  }
}

// One damped Jacobi sweep on L y = 0 for M columns ([n][M] layout):
// x_out = x - omega D^-1 L x, L x in difference form.
template <int M>
struct FJacobi {
  const int32_t* __restrict__ col;
  const double* __restrict__ w;
  const double* __restrict__ dinv;
  double omega;
  const double* __restrict__ x;
  double* __restrict__ xo;
  struct Acc {
    double s[M], xi[M];
  };
  __device__ Acc init(int64_t i, int64_t, int64_t) const {
    Acc a;
#pragma unroll
    for (int q = 0; q < M; ++q) {
      a.s[q] = 0.0;
      a.xi[q] = x[i * M + q];
    }
    return a;
  }
  __device__ void add(Acc& a, int64_t, int64_t k) const {
    const int64_t j = col[k];
    const double wk = w[k];
#pragma unroll
    for (int q = 0; q < M; ++q) a.s[q] += wk * (a.xi[q] - x[j * M + q]);
  }
  __device__ void merge(Acc& a, const Acc& o) const {
#pragma unroll
    for (int q = 0; q < M; ++q) a.s[q] += o.s[q];
  }
  __device__ Acc shfl(const Acc& a, int o) const {
    Acc r = a;
#pragma unroll
    for (int q = 0; q < M; ++q) r.s[q] = each_shfl(a.s[q], o);
    return r;
  }
  __device__ long long finish(int64_t i, const Acc& a, int64_t, int64_t) const {
    const double di = dinv[i];
#pragma unroll
    for (int q = 0; q < M; ++q) xo[i * M + q] = a.xi[q] - omega * di * a.s[q];
    return 0;
  }
};

// C_ij = (x_i . x_j)^2 / (|x_i|^2 |x_j|^2), 0 when the denominator is 0; the
// products and sums are formed the same way for (i, j) and (j, i), so C is
// bitwise symmetric. rowmax_i = max_j C_ij.
template <int M>
struct FAffinity {
  const int32_t* __restrict__ col;
  const double* __restrict__ x;
  double* __restrict__ C;
  double* __restrict__ rowmax;
  struct Acc {
    double mx, xi2, xi[M];
  };
  __device__ Acc init(int64_t i, int64_t, int64_t) const {
    Acc a;
    a.mx = 0.0;
    a.xi2 = 0.0;
#pragma unroll
    for (int q = 0; q < M; ++q) {
      a.xi[q] = x[i * M + q];
      a.xi2 += a.xi[q] * a.xi[q];
    }
    return a;
  }
  __device__ void add(Acc& a, int64_t, int64_t k) const {
    const int64_t j = col[k];
    double xj2 = 0.0, xij = 0.0;
#pragma unroll
    for (int q = 0; q < M; ++q) {
      const double v = x[j * M + q];
      xj2 += v * v;
      xij += a.xi[q] * v;
    }
    const double den = a.xi2 * xj2;
    const double c = den > 0.0 ? (xij * xij) / den : 0.0;
    C[k] = c;
    a.mx = c > a.mx ? c : a.mx;
  }
  __device__ void merge(Acc& a, const Acc& o) const { a.mx = o.mx > a.mx ? o.mx : a.mx; }
  __device__ Acc shfl(const Acc& a, int o) const {
    Acc r = a;
    r.mx = each_shfl(a.mx, o);
    return r;
  }
  __device__ long long finish(int64_t i, const Acc& a, int64_t, int64_t) const {
    rowmax[i] = a.mx;
    return 0;
  }
};

// S_ij = C_ij / max(rowmax_i, rowmax_j) (C symmetric: column max = row max).
struct FNormalize {
  const int32_t* __restrict__ col;
  const double* __restrict__ rowmax;
  double* __restrict__ S;
  struct Acc {
    double ri;
  };
  __device__ Acc init(int64_t i, int64_t, int64_t) const { return Acc{rowmax[i]}; }
  __device__ void add(Acc& a, int64_t, int64_t k) const {
    const double rj = rowmax[col[k]];
    const double mx = a.ri > rj ? a.ri : rj;
    S[k] = mx > 0.0 ? S[k] / mx : 0.0;
  }
  __device__ void merge(Acc&, const Acc&) const {}
  __device__ Acc shfl(const Acc& a, int) const { return a; }
  __device__ long long finish(int64_t, const Acc&, int64_t, int64_t) const { return 0; }
};

// d_i = sum_j w_ij and 1/d_i (0 for an isolated vertex).
struct FRowSum {
  const double* __restrict__ w;
  double* __restrict__ d;
  double* __restrict__ dinv;
  struct Acc {
    double s;
  };
  __device__ Acc init(int64_t, int64_t, int64_t) const { return Acc{0.0}; }
  __device__ void add(Acc& a, int64_t, int64_t k) const { a.s += w[k]; }
  __device__ void merge(Acc& a, const Acc& o) const { a.s += o.s; }
  __device__ Acc shfl(const Acc& a, int o) const { return Acc{each_shfl(a.s, o)}; }
  __device__ long long finish(int64_t i, const Acc& a, int64_t, int64_t) const {
    if (d) d[i] = a.s;
    dinv[i] = a.s > 0.0 ? 1.0 / a.s : 0.0;
    return 0;
  }
};

// ---------------------------------------------------------------------------
// Aggregation (Section 3.5, Algorithm 3).
// status = (state, idx) with Seed > Undecided > Decided. The (+)agg maximum
// over filtered neighbours is taken on a 128-bit key: high word
// state << 62 | FP64 bits of S_ij (S in [0, 1], so its bits fit in 62),
// low word ~idx_j, i.e. larger state, then larger weight, then smaller index.
// ---------------------------------------------------------------------------
__global__ void k_agg_init(int64_t n, int8_t* state, int32_t* idx, int32_t* votes) {
  LG_GRID_STRIDE(i, n) {
    state[i] = LG_UNDECIDED;
    idx[i] = (int32_t)i;
    votes[i] = 0;
  }
}

// Decisions of one step, all reading the status from the start of the step:
// an Undecided vertex whose best neighbour is a Seed joins it (Decided); if
// the best is Undecided it votes for it. Seeds and Decided vertices keep
// their status.
struct FAggDecide {
  const int32_t* __restrict__ col;
  const double* __restrict__ S;
  double filter;
  const int8_t* __restrict__ state;
  const int32_t* __restrict__ idx;
  int8_t* __restrict__ nstate;
  int32_t* __restrict__ nidx;
  int32_t* __restrict__ votes;
  struct Acc {
    unsigned long long hi, lo;  // the (Decided, -1, 0) identity sorts below every real entry
    int und;
  };
  __device__ Acc init(int64_t i, int64_t, int64_t) const { return Acc{0ull, 0ull, state[i] == LG_UNDECIDED}; }
  __device__ void add(Acc& a, int64_t, int64_t p) const {
    if (!a.und) return;
    const double sp = S[p];
    if (!(sp >= filter)) return;
    const int32_t j = col[p];
    const unsigned long long h = ((unsigned long long)state[j] << 62) | (unsigned long long)__double_as_longlong(sp);
    const unsigned long long l = (unsigned long long)(~(uint32_t)idx[j]);
    if (h > a.hi || (h == a.hi && l > a.lo)) {
      a.hi = h;
      a.lo = l;
    }
  }
  __device__ void merge(Acc& a, const Acc& o) const {
    if (o.hi > a.hi || (o.hi == a.hi && o.lo > a.lo)) {
      a.hi = o.hi;
      a.lo = o.lo;
    }
  }
  __device__ Acc shfl(const Acc& a, int o) const { return Acc{each_shfl(a.hi, o), each_shfl(a.lo, o), a.und}; }
  __device__ long long finish(int64_t i, const Acc& a, int64_t, int64_t) const {
    if (!a.und) {
      nstate[i] = state[i];
      nidx[i] = idx[i];
      return 0;
    }
    const int s = (int)(a.hi >> 62);
    const int32_t j = (int32_t)(~(uint32_t)a.lo);
    int8_t ns = LG_UNDECIDED;
    int32_t ni = (int32_t)i;
    if (a.hi != 0) {
      if (s == LG_SEED) {
        ns = LG_DECIDED;
        ni = j;
      } else if (s == LG_UNDECIDED) {
        atomicAdd(&votes[j], 1);
      }
    }
    nstate[i] = ns;
    nidx[i] = ni;
    return 0;
  }
};

__global__ void k_agg_promote(int64_t n, int threshold, const int32_t* __restrict__ votes, int8_t* __restrict__ state,
                              const int32_t* __restrict__ idx) {
  LG_GRID_STRIDE(i, n) {
    if (state[i] == LG_UNDECIDED && idx[i] == i && votes[i] >= threshold) state[i] = LG_SEED;
  }
}

__global__ void k_agg_roots(int64_t n, const int32_t* __restrict__ idx, uint8_t* __restrict__ root) {
  LG_GRID_STRIDE(i, n) root[i] = idx[i] == i;
}

__global__ void k_agg_number(int64_t n, const int32_t* __restrict__ idx, const int64_t* __restrict__ cid,
                             int32_t* __restrict__ agg) {
  LG_GRID_STRIDE(i, n) agg[i] = (int32_t)cid[idx[i]];
}

// ---------------------------------------------------------------------------
// Galerkin product L_c = R L P, P = R^T (Section 3.5): the coarse weight
// between aggregates I != J sums the weights of the edges joining them.
// ---------------------------------------------------------------------------
struct FGalCount {
  const int32_t* __restrict__ col;
  const int32_t* __restrict__ agg;
  int64_t* __restrict__ cnt;
  struct Acc {
    long long c;
    int32_t ai;
  };
  __device__ Acc init(int64_t i, int64_t, int64_t) const { return Acc{0, agg[i]}; }
  __device__ void add(Acc& a, int64_t, int64_t p) const { a.c += agg[col[p]] != a.ai; }
  __device__ void merge(Acc& a, const Acc& o) const { a.c += o.c; }
  __device__ Acc shfl(const Acc& a, int o) const { return Acc{each_shfl(a.c, o), a.ai}; }
  __device__ long long finish(int64_t i, const Acc& a, int64_t, int64_t) const {
    cnt[i] = a.c;
    return 0;
  }
};

// Galerkin entries: (agg_i << cbits | agg_j, w_ij) for every stored (i, j)
// joining two different aggregates, in row order.
struct EGal {
  const int32_t* __restrict__ col;
  const double* __restrict__ w;
  const int32_t* __restrict__ agg;
  int cbits;
  uint64_t* __restrict__ keys;
  uint64_t* __restrict__ vals;
  struct Row {
    int32_t ai;
  };
  __device__ Row row(int64_t i) const { return Row{agg[i]}; }
  __device__ bool special(const Row&) const { return false; }
  __device__ void emit_special(const Row&, int64_t, int64_t, int64_t, int64_t) const {}
  __device__ bool take(const Row& r, int64_t, int64_t k) const { return agg[col[k]] != r.ai; }
  __device__ void put(const Row& r, int64_t, int64_t k, int64_t p) const {
    keys[p] = ((uint64_t)r.ai << cbits) | (uint64_t)agg[col[k]];
    vals[p] = (uint64_t)__double_as_longlong(w[k]);
  }
};

// Offsets of the Galerkin entries grouped by aggregate: the members of each
// aggregate in ascending order (the member lists), each member's entries in
// its row order, which is the order the fine-row emission gives every key,
// so a sort within aggregates sums as the global sort does.
__global__ void k_member_counts(int64_t n, const int32_t* __restrict__ mem, const int64_t* __restrict__ off,
                                int64_t* __restrict__ mc) {
  LG_GRID_STRIDE(m, n) mc[m] = off[mem[m] + 1] - off[mem[m]];
}
__global__ void k_member_offsets(int64_t n, const int32_t* __restrict__ mem, const int64_t* __restrict__ pos,
                                 int64_t* __restrict__ offg) {
  LG_GRID_STRIDE(m, n) offg[mem[m]] = pos[m];
}
__global__ void k_group_offsets(int64_t nc, const int64_t* __restrict__ mem_ptr, const int64_t* __restrict__ pos,
                                int64_t* __restrict__ gp) {
  LG_GRID_STRIDE(a, nc + 1) gp[a] = pos[mem_ptr[a]];
}

// Entries of W = L P off the own aggregate: (i << cbits | agg_j, w_ij) for
// every stored (i, j) with agg_j != agg_i, in row order. Summed over equal
// keys they give W_ia = sum of w_ij over i's neighbours j in aggregate a, so
// that (L P x_c)_i = sum_a W_ia (x_c[agg_i] - x_c[a]): P's columns are the
// aggregates' indicator vectors and L's rows sum to zero.
struct ELp {
  const int32_t* __restrict__ col;
  const double* __restrict__ w;
  const int32_t* __restrict__ agg;
  int cbits;
  uint64_t* __restrict__ keys;
  uint64_t* __restrict__ vals;
  struct Row {
    int32_t ai;
  };
  __device__ Row row(int64_t i) const { return Row{agg[i]}; }
  __device__ bool special(const Row&) const { return false; }
  __device__ void emit_special(const Row&, int64_t, int64_t, int64_t, int64_t) const {}
  __device__ bool take(const Row& r, int64_t, int64_t k) const { return agg[col[k]] != r.ai; }
  __device__ void put(const Row&, int64_t i, int64_t k, int64_t p) const {
    keys[p] = ((uint64_t)i << cbits) | (uint64_t)agg[col[k]];
    vals[p] = (uint64_t)__double_as_longlong(w[k]);
  }
};

__global__ void k_iota_u64(int64_t n, const int32_t* __restrict__ agg, uint64_t* __restrict__ keys,
                           uint64_t* __restrict__ vals) {
  LG_GRID_STRIDE(i, n) {
    keys[i] = (uint64_t)agg[i];
    vals[i] = (uint64_t)i;
  }
}

__global__ void k_u64_to_i32(int64_t n, const uint64_t* __restrict__ a, int32_t* __restrict__ b) {
  LG_GRID_STRIDE(i, n) b[i] = (int32_t)a[i];
}

// ---------------------------------------------------------------------------
// Largest eigenvalue of D^-1 L (Section 3.6): eig_iters Lanczos steps on
// D^-1/2 L D^-1/2 (the Jacobi-preconditioned operator, symmetric in the D
// inner product), start vector from SplitMix64 stream 8, early stop once
// beta_k <= 1e-12 |alpha_k|; the estimate is the largest eigenvalue of the
// tridiagonal, by Sturm-count bisection.
// ---------------------------------------------------------------------------
struct Lanczos {
  double alpha[64], beta[64];
  double nrm2, b2;
  int m, stopped;
};

__global__ void k_lz_start(int64_t n, uint64_t seed, int level, const double* __restrict__ dinv,
                           double* __restrict__ v, double* __restrict__ sdinv, double* partials, unsigned* ticket,
                           Lanczos* lz) {
  double acc[1] = {0.0};
  LG_GRID_STRIDE(i, n) {
    const double u = uniform_pm1(seed, kStreamLanczos, level, i);
    v[i] = u;
    sdinv[i] = sqrt(dinv[i]);
    acc[0] += u * u;
  }
  if (grid_sum<kNT, 1>(acc, partials, ticket, &lz->nrm2)) {
    lz->m = 0;
    lz->stopped = 0;
  }
}

__global__ void k_lz_scale(int64_t n, const Lanczos* lz, double* __restrict__ v, const double* __restrict__ sdinv,
                           double* __restrict__ t, double* __restrict__ vp) {
  const double inv = 1.0 / sqrt(lz->nrm2);
  LG_GRID_STRIDE(i, n) {
    v[i] *= inv;
    t[i] = v[i] * sdinv[i];
    vp[i] = 0.0;
  }
}

// u = D^-1/2 L D^-1/2 v, from s = (L t)_i with t = D^-1/2 v.
struct EpiLanczos {
  const double* sdinv;
  double* u;
  __device__ __forceinline__ double pre(int64_t i) const { return sdinv[i]; }
  __device__ __forceinline__ void operator()(int64_t i, double s, double sd, double*) const { u[i] = sd * s; }
  __device__ void finish(const double*) const {}
};

// alpha_k = v . u
__global__ void k_lz_alpha(int64_t n, int k, Lanczos* lz, const double* __restrict__ v, const double* __restrict__ u,
                           double* partials, unsigned* ticket) {
  if (lz->stopped) return;
  double acc[1] = {0.0};
  LG_GRID_STRIDE(i, n) acc[0] += v[i] * u[i];
  grid_sum<kNT, 1>(acc, partials, ticket, &lz->alpha[k]);
}

__global__ void k_lz_orth(int64_t n, int k, Lanczos* lz, double* __restrict__ u, const double* __restrict__ v,
                          const double* __restrict__ vp, double* partials, unsigned* ticket) {
  if (lz->stopped) return;
  const double a = lz->alpha[k], b = k > 0 ? lz->beta[k - 1] : 0.0;
  double acc[1] = {0.0};
  LG_GRID_STRIDE(i, n) {
    const double ui = u[i] - a * v[i] - b * vp[i];
    u[i] = ui;
    acc[0] += ui * ui;
  }
  if (grid_sum<kNT, 1>(acc, partials, ticket, &lz->b2)) {
    const double bk = sqrt(lz->b2);
    lz->beta[k] = bk;
    lz->m = k + 1;
    if (bk <= 1e-12 * fabs(a)) lz->stopped = 1;
  }
}

__global__ void k_lz_next(int64_t n, int k, const Lanczos* lz, const double* __restrict__ u, double* __restrict__ v,
                          double* __restrict__ vp, const double* __restrict__ sdinv, double* __restrict__ t) {
  if (lz->stopped) return;
  const double inv = 1.0 / lz->beta[k];
  LG_GRID_STRIDE(i, n) {
    vp[i] = v[i];
    const double vi = u[i] * inv;
    v[i] = vi;
    t[i] = vi * sdinv[i];
  }
}

// Number of eigenvalues of the symmetric tridiagonal matrix (diagonal a[0..m),
// off-diagonal b[0..m-1)) below x, by the signs of the LDL^T pivots (Sturm).
static int sturm_count(int m, const double* a, const double* b, double x) {
  int count = 0;
  double q = 1.0;
  for (int i = 0; i < m; ++i) {
    const double off = i > 0 ? b[i - 1] * b[i - 1] / q : 0.0;
    q = (a[i] - x) - off;
    if (q == 0.0) q = -1e-300;
    if (q < 0.0) ++count;
  }
  return count;
}

// Largest eigenvalue of the Lanczos tridiagonal (the Ritz value), by
// bisection between Gershgorin bounds until the interval stops shrinking.
// It runs on the host once per level at the end of the setup, on the alpha
// and beta the device recursion left: a dozen scalars, a few microseconds,
// where a one-thread kernel spent a quarter of a millisecond.
static double ritz_max(const Lanczos& lz) {
  const int m = lz.m;
  const double* a = lz.alpha;
  const double* b = lz.beta;
  if (m < 1) return 0.0;
  double lo = a[0], hi = a[0];
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i < m - 1 ? std::fabs(b[i]) : 0.0);
    lo = std::fmin(lo, a[i] - r);
    hi = std::fmax(hi, a[i] + r);
  }
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_count(m, a, b, mid) == m) hi = mid; else lo = mid;
  }
  return hi;
}

// ---------------------------------------------------------------------------
// Coarsest level: L^+ = (L + 11^T/n)^-1 - 11^T/n (null space span(1),
// Section 2.1), the inverse by in-place Gauss-Jordan (SPD: no pivoting).
// ---------------------------------------------------------------------------
__global__ void k_dense_shifted(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                const double* __restrict__ w, double* __restrict__ M) {
  const double c = 1.0 / (double)n;
  LG_GRID_STRIDE(i, n) {
    double d = 0.0;
    for (int64_t j = 0; j < n; ++j) M[i * n + j] = c;
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      M[i * n + col[p]] = c - w[p];
      d += w[p];
    }
    M[i * n + i] = c + d;
  }
}

__global__ void k_gj_copy(int64_t n, int64_t k, const double* __restrict__ M, double* __restrict__ prow,
                          double* __restrict__ pcol) {
  LG_GRID_STRIDE(i, n) {
    prow[i] = M[k * n + i];
    pcol[i] = M[i * n + k];
  }
}

__global__ void k_gj_update(int64_t n, int64_t k, double* __restrict__ M, const double* __restrict__ prow,
                            const double* __restrict__ pcol, int* err) {
  const double p = prow[k];
  if (!(p > 0.0)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(err, kErrLoop);
    return;
  }
  const double ip = 1.0 / p;
  LG_GRID_STRIDE(e, n * n) {
    const int64_t i = e / n, j = e % n;
    double v;
    if (i == k && j == k) v = ip;
    else if (i == k) v = prow[j] * ip;
    else if (j == k) v = -pcol[i] * ip;
    else v = M[e] - pcol[i] * prow[j] * ip;
    M[e] = v;
  }
}

__global__ void k_unshift(int64_t n, double* __restrict__ M) {
  const double c = 1.0 / (double)n;
  LG_GRID_STRIDE(e, n * n) M[e] -= c;
}

// ---------------------------------------------------------------------------
// FP32 copies of the hierarchy.
// ---------------------------------------------------------------------------
__global__ void k_to_f32(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  LG_GRID_STRIDE(i, n) b[i] = (float)a[i];
}

// ---------------------------------------------------------------------------
// Vertex renumbering by descending degree (stable: ties keep their order).
// ---------------------------------------------------------------------------
__global__ void k_degree_keys(int64_t n, const int64_t* __restrict__ rowptr, uint64_t* __restrict__ key,
                              uint64_t* __restrict__ val) {
  LG_GRID_STRIDE(i, n) {
    const int64_t deg = rowptr[i + 1] - rowptr[i];
    key[i] = 0xffffffffull - (uint64_t)deg;
    val[i] = (uint64_t)i;
  }
}

// Keys of the random ordering (Section 3.3): a SplitMix64 value per vertex
// (stream kStreamOrder), the vertex id breaking the (unlikely) ties.
__global__ void k_random_keys(int64_t n, uint64_t seed, uint64_t* __restrict__ key, uint64_t* __restrict__ val) {
  LG_GRID_STRIDE(i, n) {
    key[i] = splitmix64(seed, rng_counter(kStreamOrder, 0, i)) >> 32;
    val[i] = (uint64_t)i;
  }
}

// Columns and weights of sorted (row << cbits | column, weight bits) entries.
__global__ void k_unpack_entries(int64_t nent, const uint64_t* __restrict__ keys, const uint64_t* __restrict__ vals,
                                 uint64_t cmask, int32_t* __restrict__ col, double* __restrict__ w) {
  LG_GRID_STRIDE(k, nent) {
    col[k] = (int32_t)(keys[k] & cmask);
    w[k] = __longlong_as_double((long long)vals[k]);
  }
}

// Degrees in the new numbering.
__global__ void k_perm_degrees(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ inv,
                               int64_t* __restrict__ deg_new) {
  LG_GRID_STRIDE(i, n) deg_new[inv[i]] = rowptr[i + 1] - rowptr[i];
}

__global__ void k_perm_from_sorted(int64_t n, const uint64_t* __restrict__ val, int32_t* __restrict__ perm,
                                   int32_t* __restrict__ inv) {
  LG_GRID_STRIDE(i, n) {
    const int32_t old = (int32_t)val[i];
    perm[i] = old;
    inv[old] = (int32_t)i;
  }
}

__global__ void k_iota_i32(int64_t n, int32_t* __restrict__ a) {
  LG_GRID_STRIDE(i, n) a[i] = (int32_t)i;
}

// Entries of the renumbered graph: (inv[i], inv[j]) for every stored (i, j).
// Entries of the renumbered operator, keyed (new row, new column). With
// rp_new (the new rows' offsets) each row's entries go where the new row
// starts, so they come grouped by new row for a sort within rows; without,
// they stay at their old positions for a global sort.
struct FPermEmit {
  const int32_t* __restrict__ col;
  const double* __restrict__ w;
  const int32_t* __restrict__ inv;
  const int64_t* __restrict__ rp_new;
  int cbits;
  uint64_t* __restrict__ keys;
  uint64_t* __restrict__ vals;
  struct Acc {
    unsigned long long row;
    int64_t shift;
  };
  __device__ Acc init(int64_t i, int64_t beg, int64_t) const {
    return Acc{(unsigned long long)inv[i] << cbits, rp_new ? rp_new[inv[i]] - beg : 0};
  }
  __device__ void add(Acc& a, int64_t, int64_t k) const {
    keys[a.shift + k] = a.row | (uint64_t)inv[col[k]];
    vals[a.shift + k] = (uint64_t)__double_as_longlong(w[k]);
  }
  __device__ void merge(Acc&, const Acc&) const {}
  __device__ Acc shfl(const Acc& a, int) const { return a; }
  __device__ long long finish(int64_t, const Acc&, int64_t, int64_t) const { return 0; }
};

// ---------------------------------------------------------------------------
// FP32-only hierarchies: an elimination level below the finest keeps only its
// eliminated rows (the cycle reads nothing else of its operator: the kept
// vertices take their coarse value, Section 3.4).
// ---------------------------------------------------------------------------
__global__ void k_frow_count(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ cmap,
                             int64_t* __restrict__ cnt) {
  LG_GRID_STRIDE(i, n) cnt[i] = cmap[i] < 0 ? rowptr[i + 1] - rowptr[i] : 0;
}

__global__ void k_frow_copy(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            const float* __restrict__ w32, const int32_t* __restrict__ cmap,
                            const int64_t* __restrict__ nptr, int32_t* __restrict__ ncol, float* __restrict__ nw32) {
  LG_GRID_STRIDE(i, n) {
    if (cmap[i] >= 0) continue;
    const int64_t b = rowptr[i], e = rowptr[i + 1], o = nptr[i];
    for (int64_t k = b; k < e; ++k) {
      ncol[o + (k - b)] = col[k];
      nw32[o + (k - b)] = w32[k];
    }
  }
}

// ===========================================================================
// Host side.
// ===========================================================================
static int read_err(const DBuf<int>& e, cudaStream_t s) {
  int v = 0;
  LG_CUDA(cudaMemcpyAsync(&v, e.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
  LG_CUDA(cudaStreamSynchronize(s));
  return v;
}

static int64_t read_i64(const int64_t* p, cudaStream_t s) {
  int64_t v = 0;
  LG_CUDA(cudaMemcpyAsync(&v, p, sizeof(int64_t), cudaMemcpyDefault, s));
  LG_CUDA(cudaStreamSynchronize(s));
  return v;
}

// Row plan and 1/diag of a level's operator.
static void prepare_operator(Level& L, cudaStream_t s, int64_t* counter) {
  build_row_plan(L.plan, L.n, L.nnz, L.rowptr.get(), s, counter, L.n);
  L.d.alloc(L.n, s, counter);
  L.dinv.alloc(L.n, s, counter);
  launch_rows<double, 0>(L.n, L.rowptr.get(), L.col.get(), WeightTerm{L.w.get()}, L.plan.plan,
                         EpiDinv{L.d.get(), L.dinv.get()}, s);
}

void run_laplacian_apply(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w, const double* x,
                         double* y, cudaStream_t s) {
  RowPlanStore ps;
  const int64_t nnz = read_i64(rowptr + n, s);
  build_row_plan(ps, n, nnz, rowptr, s, nullptr);
  DBuf<double> d(n, s), dinv(n, s);
  launch_rows<double, 0>(n, rowptr, col, WeightTerm{w}, ps.plan, EpiDinv{d.get(), dinv.get()}, s);
  launch_rows<double, 0>(n, rowptr, col, LapTerm<double>{w, x, d.get()}, ps.plan, EpiStore<double>{y}, s);
  LG_CUDA(cudaStreamSynchronize(s));
}

int64_t run_elim_select(int64_t n, const int64_t* rowptr, const int32_t* col, int max_degree, uint64_t seed,
                        uint8_t* is_f, cudaStream_t s) {
  DBuf<uint64_t> hc(n, s);
  DBuf<int64_t> cnt(n + 1, s);
  k_elim_hash<<<blocks_for(n), kNT, 0, s>>>(n, rowptr, max_degree, seed, hc.get());
  LG_LAUNCH_CHECK();
  k_elim_select<<<blocks_for(n), kNT, 0, s>>>(n, rowptr, col, max_degree, hc.get(), is_f);
  LG_LAUNCH_CHECK();
  exclusive_scan_flags(is_f, cnt.get(), n, s);
  return read_i64(cnt.get() + n, s);
}

void run_strength(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w, uint64_t seed, int level,
                  int m, int sweeps, double omega, double* S, cudaStream_t s, const RowBins* bins_in,
                  const double* dinv_in) {
  if (m < 1 || m > kMaxVecs) fail(LG_ERR_INVALID, "strength_vecs must be 1..8");
  RowBinsStore own;
  if (!bins_in) make_bins(own, n, rowptr, s);
  const RowBins& bins = bins_in ? *bins_in : own.bins;
  DBuf<double> dv, xa((size_t)n * m, s), xb((size_t)n * m, s), rowmax(n, s);
  const double* dinv = dinv_in;
  if (!dinv) {
    dv.alloc(n, s);
    each_row(FRowSum{w, nullptr, dv.get()}, rowptr, bins, s);
    dinv = dv.get();
  }
  k_strength_init<<<blocks_for(n), kNT, 0, s>>>(n, m, seed, level, xa.get());
  LG_LAUNCH_CHECK();
  double* x = xa.get();
  double* xo = xb.get();
  auto sweep = [&](auto mtag) {
    constexpr int M = decltype(mtag)::value;
    for (int sw = 0; sw < sweeps; ++sw) {
      each_row(FJacobi<M>{col, w, dinv, omega, x, xo}, rowptr, bins, s);
      std::swap(x, xo);
    }
    each_row(FAffinity<M>{col, x, S, rowmax.get()}, rowptr, bins, s);
  };
  switch (m) {
    case 1: sweep(std::integral_constant<int, 1>{}); break;
    case 2: sweep(std::integral_constant<int, 2>{}); break;
    case 3: sweep(std::integral_constant<int, 3>{}); break;
    case 4: sweep(std::integral_constant<int, 4>{}); break;
    case 5: sweep(std::integral_constant<int, 5>{}); break;
    case 6: sweep(std::integral_constant<int, 6>{}); break;
    case 7: sweep(std::integral_constant<int, 7>{}); break;
    default: sweep(std::integral_constant<int, 8>{}); break;
  }
  each_row(FNormalize{col, rowmax.get(), S}, rowptr, bins, s);
  if (!bins_in) LG_CUDA(cudaStreamSynchronize(s));
}

int64_t run_aggregate(int64_t n, const int64_t* rowptr, const int32_t* col, const double* S, int iters, int threshold,
                      int32_t* agg, int8_t* state_out, int32_t* votes_out, cudaStream_t s, const RowBins* bins_in) {
  RowBinsStore own;
  if (!bins_in) make_bins(own, n, rowptr, s);
  const RowBins& bins = bins_in ? *bins_in : own.bins;
  DBuf<int8_t> st(n, s), nst(n, s);
  DBuf<int32_t> idx(n, s), nidx(n, s), votes(n, s);
  DBuf<uint8_t> root(n, s);
  DBuf<int64_t> cid(n + 1, s);
  k_agg_init<<<blocks_for(n), kNT, 0, s>>>(n, st.get(), idx.get(), votes.get());
  LG_LAUNCH_CHECK();
  int8_t *a = st.get(), *b = nst.get();
  int32_t *ia = idx.get(), *ib = nidx.get();
  for (int it = 1; it <= iters; ++it) {
    const double filter = std::ldexp(1.0, -it);  // 0.5^iter
    each_row(FAggDecide{col, S, filter, a, ia, b, ib, votes.get()}, rowptr, bins, s);
    k_agg_promote<<<blocks_for(n), kNT, 0, s>>>(n, threshold, votes.get(), b, ib);
    LG_LAUNCH_CHECK();
    std::swap(a, b);
    std::swap(ia, ib);
  }
  k_agg_roots<<<blocks_for(n), kNT, 0, s>>>(n, ia, root.get());
  LG_LAUNCH_CHECK();
  exclusive_scan_flags(root.get(), cid.get(), n, s);
  k_agg_number<<<blocks_for(n), kNT, 0, s>>>(n, ia, cid.get(), agg);
  LG_LAUNCH_CHECK();
  if (state_out) LG_CUDA(cudaMemcpyAsync(state_out, a, n, cudaMemcpyDeviceToDevice, s));
  if (votes_out) LG_CUDA(cudaMemcpyAsync(votes_out, votes.get(), 4 * n, cudaMemcpyDeviceToDevice, s));
  return read_i64(cid.get() + n, s);
}

// Elimination stage: fills L's ELIM fields and returns the Schur complement level.
static std::unique_ptr<Level> eliminate(Level& L, const uint8_t* is_f, int64_t nf, bool grouped, cudaStream_t s,
                                        int64_t* counter) {
  const int64_t n = L.n;
  DBuf<uint8_t> keep(n, s);
  DBuf<int64_t> cid(n + 1, s), cnt(n + 1, s);
  k_not<<<blocks_for(n), kNT, 0, s>>>(n, is_f, keep.get());
  LG_LAUNCH_CHECK();
  exclusive_scan_flags(keep.get(), cid.get(), n, s);
  const int64_t nc = n - nf;
  L.kind = LG_LEVEL_ELIM;
  L.nf = nf;
  L.nc = nc;
  L.cmap.alloc(n, s, counter);
  L.cfine.alloc(nc, s, counter);
  k_elim_maps<<<blocks_for(n), kNT, 0, s>>>(n, is_f, cid.get(), L.cmap.get(), L.cfine.get());
  LG_LAUNCH_CHECK();

  // Schur complement entries, sorted and summed into the coarse CSR: emitted
  // by kept row and sorted within rows, or emitted by fine row and sorted
  // globally; both give the same order and sums.
  if (grouped)
    each_row(FSchurCountRows{L.rowptr.get(), L.col.get(), is_f, cnt.get()}, L.rowptr.get(), bins_of(L.plan.plan, n),
             s);
  else
    each_row(FSchurCount{L.col.get(), is_f, cnt.get()}, L.rowptr.get(), bins_of(L.plan.plan, n), s);
  exclusive_scan(cnt.get(), cnt.get(), n, s);
  const int64_t nent = read_i64(cnt.get() + n, s);
  const int cbits = bits_for(nc);
  auto C = std::make_unique<Level>();
  {
    DBuf<uint64_t> keys(nent, s), vals(nent, s);
    if (grouped) {
      const RowBins bins = bins_of(L.plan.plan, n);
      if (bins.grid > 0) {
        k_schur_emit_rows<<<bins.grid, kEachThreads, 0, s>>>(
            SchurRows{L.rowptr.get(), L.col.get(), L.w.get(), is_f, L.cmap.get(), cnt.get(), cbits, keys.get(),
                      vals.get()},
            bins);
        LG_LAUNCH_CHECK();
      }
    } else {
      emit_rows(ESchur{L.col.get(), L.w.get(), is_f, L.cmap.get(), cbits, keys.get(), vals.get()}, L.rowptr.get(),
                cnt.get(), bins_of(L.plan.plan, n), s);
    }
    CsrOut out;
    accumulate_csr(keys, vals, nent, nc, cbits, out, s, counter, grouped ? cnt.get() : nullptr, n);
    C->n = nc;
    C->nnz = out.nnz;
    C->rowptr = std::move(out.rowptr);
    C->col = std::move(out.col);
    C->w = std::move(out.w);
  }
  // Transpose of P's F rows, per kept vertex.
  k_f_degree<<<blocks_for(n), kNT, 0, s>>>(n, L.rowptr.get(), is_f, cnt.get());
  LG_LAUNCH_CHECK();
  exclusive_scan(cnt.get(), cnt.get(), n, s);
  const int64_t npt = read_i64(cnt.get() + n, s);
  {
    DBuf<uint64_t> keys(npt, s), vals(npt, s);
    k_pt_emit<<<blocks_for(n), kNT, 0, s>>>(n, L.rowptr.get(), L.col.get(), is_f, L.cmap.get(), cnt.get(),
                                           keys.get(), vals.get());
    LG_LAUNCH_CHECK();
    radix_sort_pairs(keys.get(), vals.get(), npt, bits_for(nc), s);
    L.pt_ptr.alloc(nc + 1, s, counter);
    L.pt_f.alloc(npt, s, counter);
    L.pt_coef.alloc(npt, s, counter);
    k_rowptr_sorted<<<blocks_for(nc + 1), kNT, 0, s>>>(keys.get(), npt, 0, nc, L.pt_ptr.get());
    LG_LAUNCH_CHECK();
    k_pt_fill<<<blocks_for(npt), kNT, 0, s>>>(npt, vals.get(), L.rowptr.get(), L.w.get(), L.pt_f.get(),
                                             L.pt_coef.get());
    LG_LAUNCH_CHECK();
    build_row_plan(L.pt_plan, nc, npt, L.pt_ptr.get(), s, counter);
  }
  return C;
}

// Smallest aggregation level that gets W = L P (see galerkin).
constexpr int64_t kLpMinRows = 4096;

// Aggregation stage products: member CSR of R, the Galerkin level, and
// W = L P when `lp` (levels of at least kLpMinRows vertices).
static std::unique_ptr<Level> galerkin(Level& L, bool lp, bool grouped, cudaStream_t s, int64_t* counter,
                                       StageClock& clk) {
  const int64_t n = L.n, nc = L.nc;
  // member lists, ascending vertex order inside each aggregate (stable sort by aggregate)
  {
    DBuf<uint64_t> keys(n, s), vals(n, s);
    k_iota_u64<<<blocks_for(n), kNT, 0, s>>>(n, L.agg.get(), keys.get(), vals.get());
    LG_LAUNCH_CHECK();
    radix_sort_pairs(keys.get(), vals.get(), n, bits_for(nc), s);
    L.mem.alloc(n, s, counter);
    L.mem_ptr.alloc(nc + 1, s, counter);
    k_u64_to_i32<<<blocks_for(n), kNT, 0, s>>>(n, vals.get(), L.mem.get());
    LG_LAUNCH_CHECK();
    k_rowptr_sorted<<<blocks_for(nc + 1), kNT, 0, s>>>(keys.get(), n, 0, nc, L.mem_ptr.get());
    LG_LAUNCH_CHECK();
    build_row_plan(L.mem_plan, nc, n, L.mem_ptr.get(), s, counter);
  }
  clk.mark("member_lists");
  DBuf<int64_t> cnt(n + 1, s);
  each_row(FGalCount{L.col.get(), L.agg.get(), cnt.get()}, L.rowptr.get(), bins_of(L.plan.plan, n), s);
  exclusive_scan(cnt.get(), cnt.get(), n, s);
  const int64_t nent = read_i64(cnt.get() + n, s);
  const int cbits = bits_for(nc);
  auto C = std::make_unique<Level>();
  {
    DBuf<uint64_t> keys(nent, s), vals(nent, s);
    DBuf<int64_t> offg, gp;
    if (grouped) {  // each fine row's entries where its aggregate's group places them
      DBuf<int64_t> pos(n + 1, s);
      offg.alloc(n, s);
      gp.alloc(nc + 1, s);
      k_member_counts<<<blocks_for(n), kNT, 0, s>>>(n, L.mem.get(), cnt.get(), pos.get());
      LG_LAUNCH_CHECK();
      exclusive_scan(pos.get(), pos.get(), n, s);
      k_member_offsets<<<blocks_for(n), kNT, 0, s>>>(n, L.mem.get(), pos.get(), offg.get());
      LG_LAUNCH_CHECK();
      k_group_offsets<<<blocks_for(nc + 1), kNT, 0, s>>>(nc, L.mem_ptr.get(), pos.get(), gp.get());
      LG_LAUNCH_CHECK();
    }
    emit_rows(EGal{L.col.get(), L.w.get(), L.agg.get(), cbits, keys.get(), vals.get()}, L.rowptr.get(),
              grouped ? offg.get() : cnt.get(), bins_of(L.plan.plan, n), s);
    offg.release();
    CsrOut out;
    accumulate_csr(keys, vals, nent, nc, cbits, out, s, counter, grouped ? gp.get() : nullptr, nc);
    C->n = nc;
    C->nnz = out.nnz;
    C->rowptr = std::move(out.rowptr);
    C->col = std::move(out.col);
    C->w = std::move(out.w);
  }
  clk.mark("galerkin");
  // W = L P: the same entries keyed by fine row (accumulate_csr sorts them),
  // once the Galerkin product's scratch is back. Not for levels of a few
  // thousand vertices, whose passes are launch-bound: W saves nothing there.
  if (lp && n >= kLpMinRows) {
    DBuf<uint64_t> lkeys(nent, s), lvals(nent, s);
    emit_rows(ELp{L.col.get(), L.w.get(), L.agg.get(), cbits, lkeys.get(), lvals.get()}, L.rowptr.get(), cnt.get(),
              bins_of(L.plan.plan, n), s);
    CsrOut lo;
    accumulate_csr(lkeys, lvals, nent, n, cbits, lo, s, counter, grouped ? cnt.get() : nullptr, n);
    L.lp_nnz = lo.nnz;
    L.lp_ptr = std::move(lo.rowptr);
    L.lp_col = std::move(lo.col);
    L.lp_w = std::move(lo.w);
    build_row_plan(L.lp_plan, n, L.lp_nnz, L.lp_ptr.get(), s, counter, nc);
    L.lp_d.alloc(n, s, counter);
    DBuf<double> unused(n, s);
    launch_rows<double, 0>(n, L.lp_ptr.get(), L.lp_col.get(), WeightTerm{L.lp_w.get()}, L.lp_plan.plan,
                           EpiDinv{L.lp_d.get(), unused.get()}, s);
    if (L.lp_nnz > 0) {
      L.lp_w32.alloc(L.lp_nnz, s, counter);
      k_to_f32<<<blocks_for(L.lp_nnz), kNT, 0, s>>>(L.lp_nnz, L.lp_w.get(), L.lp_w32.get());
      LG_LAUNCH_CHECK();
    }
    clk.mark("w_lp");
  }
  return C;
}

static void lanczos(Level& L, const lg_options& o, int level, Lanczos* lz_level, cudaStream_t s) {
  const int64_t n = L.n;
  const int iters = std::min(o.eig_iters, 64);
  DBuf<double> v(n, s), vp(n, s), u(n, s), t(n, s), sdinv(n, s);
  const int nb = blocks_for(n);
  DBuf<double> partials((size_t)nb, s);
  DBuf<unsigned> ticket(1, s);
  Lanczos* lz = lz_level;
  LG_CUDA(cudaMemsetAsync(ticket.get(), 0, sizeof(unsigned), s));
  k_lz_start<<<nb, kNT, 0, s>>>(n, o.seed, level, L.dinv.get(), v.get(), sdinv.get(), partials.get(), ticket.get(),
                                lz);
  LG_LAUNCH_CHECK();
  k_lz_scale<<<nb, kNT, 0, s>>>(n, lz, v.get(), sdinv.get(), t.get(), vp.get());
  LG_LAUNCH_CHECK();
  for (int k = 0; k < iters; ++k) {
    // stopped iterations leave alpha[k] untouched; only the first m entries are used
    launch_rows<double, 0>(n, L.rowptr.get(), L.col.get(), LapTerm<double>{L.w.get(), t.get(), L.d.get()}, L.plan.plan,
                           EpiLanczos{sdinv.get(), u.get()}, s);
    k_lz_alpha<<<nb, kNT, 0, s>>>(n, k, lz, v.get(), u.get(), partials.get(), ticket.get());
    LG_LAUNCH_CHECK();
    k_lz_orth<<<nb, kNT, 0, s>>>(n, k, lz, u.get(), v.get(), vp.get(), partials.get(), ticket.get());
    LG_LAUNCH_CHECK();
    k_lz_next<<<nb, kNT, 0, s>>>(n, k, lz, u.get(), v.get(), vp.get(), sdinv.get(), t.get());
    LG_LAUNCH_CHECK();
  }
}

static void coarsest_pinv(Level& L, int* err, cudaStream_t s, int64_t* counter) {
  const int64_t n = L.n;
  L.kind = LG_LEVEL_COARSEST;
  L.pinv.alloc((size_t)n * n, s, counter);
  DBuf<double> prow(n, s), pcol(n, s);
  k_dense_shifted<<<blocks_for(n), kNT, 0, s>>>(n, L.rowptr.get(), L.col.get(), L.w.get(), L.pinv.get());
  LG_LAUNCH_CHECK();
  const int gb = blocks_for(n * n);
  for (int64_t k = 0; k < n; ++k) {
    k_gj_copy<<<blocks_for(n), kNT, 0, s>>>(n, k, L.pinv.get(), prow.get(), pcol.get());
    LG_LAUNCH_CHECK();
    k_gj_update<<<gb, kNT, 0, s>>>(n, k, L.pinv.get(), prow.get(), pcol.get(), err);
    LG_LAUNCH_CHECK();
  }
  k_unshift<<<gb, kNT, 0, s>>>(n, L.pinv.get());
  LG_LAUNCH_CHECK();
}

// Smallest and largest weight of an operator as IEEE bit patterns: the
// weights are validated positive, where the bit order is the value order.
__global__ void k_wrange(int64_t nnz, const double* __restrict__ w, unsigned long long* mm) {
  unsigned long long lo = ~0ull, hi = 0ull;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(w[k]);
    lo = b < lo ? b : lo;
    hi = b > hi ? b : hi;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long a = __shfl_xor_sync(0xffffffffu, lo, o), c = __shfl_xor_sync(0xffffffffu, hi, o);
    lo = a < lo ? a : lo;
    hi = c > hi ? c : hi;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&mm[0], lo);
    atomicMax(&mm[1], hi);
  }
}

// A finest operator whose weights are all one value (an unweighted graph,
// or one scaled uniformly) keeps only its pattern: the passes take the
// value as a constant and stream 4 bytes per entry instead of 8 + 4 (FP64)
// or 4 + 4 (FP32). The products are bitwise those of the stored weights.
// Runs once the coarser levels, which read the finest weights, are built.
static void detect_constant_weights(Level& L, cudaStream_t s) {
  if (L.nnz == 0 || !L.w.get()) return;
  DBuf<unsigned long long> mm(2, s);
  const unsigned long long init[2] = {~0ull, 0ull};
  LG_CUDA(cudaMemcpyAsync(mm.get(), init, sizeof(init), cudaMemcpyHostToDevice, s));
  k_wrange<<<grid_for(L.nnz, kNT, kSMs * 8), kNT, 0, s>>>(L.nnz, L.w.get(), mm.get());
  LG_LAUNCH_CHECK();
  unsigned long long out[2];
  LG_CUDA(cudaMemcpyAsync(out, mm.get(), sizeof(out), cudaMemcpyDeviceToHost, s));
  LG_CUDA(cudaStreamSynchronize(s));
  if (out[0] != out[1]) return;
  double v;
  std::memcpy(&v, &out[0], sizeof(v));
  L.wconst_on = true;
  L.wconst = v;
  L.w.release();
  L.w32.release();
}

static void make_f32(Level& L, cudaStream_t s, int64_t* counter) {
  if (L.nnz > 0 && L.w.get()) {
    L.w32.alloc(L.nnz, s, counter);
    k_to_f32<<<blocks_for(L.nnz), kNT, 0, s>>>(L.nnz, L.w.get(), L.w32.get());
    LG_LAUNCH_CHECK();
  }
  if (L.dinv.get()) {
    L.dinv32.alloc(L.n, s, counter);
    k_to_f32<<<blocks_for(L.n), kNT, 0, s>>>(L.n, L.dinv.get(), L.dinv32.get());
    LG_LAUNCH_CHECK();
  }
  if (L.pt_coef.get() && L.pt_coef.size() > 0) {
    L.pt_coef32.alloc(L.pt_coef.size(), s, counter);
    k_to_f32<<<blocks_for((int64_t)L.pt_coef.size()), kNT, 0, s>>>((int64_t)L.pt_coef.size(), L.pt_coef.get(),
                                                                    L.pt_coef32.get());
    LG_LAUNCH_CHECK();
  }
}

// ---------------------------------------------------------------------------
// Autotuner of the row binning: each candidate E (entries per lane) is timed
// on the level's own operator, one FP64 and one FP32 plain y = L x pass
// (1 warm-up + 3 timed launches each), and the fastest kept. Choices are
// cached per (n, nnz) for the life of the process, so rebuilding a hierarchy
// of the same graph gives the same launch plans and bitwise the same results.
// ---------------------------------------------------------------------------
static std::mutex g_tune_mu;
static std::map<std::pair<int64_t, int64_t>, int> g_tune_cache;

template <typename T>
static float time_apply(const Level& L, const T* x, T* y, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
  OpView<T> op = L.op<T>();
  const LapTerm<T> term = lap_term(op, x);
  launch_rows<T, 0>(op.n, op.rowptr, op.col, term, op.plan, EpiStore<T>{y}, s);
  LG_CUDA(cudaEventRecord(e0, s));
  for (int r = 0; r < 3; ++r) launch_rows<T, 0>(op.n, op.rowptr, op.col, term, op.plan, EpiStore<T>{y}, s);
  LG_CUDA(cudaEventRecord(e1, s));
  LG_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  LG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  return ms;
}

static void tune_level(Level& L, cudaStream_t s) {
  const auto key = std::make_pair(L.n, L.nnz);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      if (it->second != L.plan.plan.E) bin_rows(L.plan, L.n, L.rowptr.get(), it->second, s);
      return;
    }
  }
  DBuf<double> x(L.n, s), y(L.n, s);
  DBuf<float> x32(L.n, s), y32(L.n, s);
  LG_CUDA(cudaMemsetAsync(x.get(), 0, sizeof(double) * L.n, s));
  LG_CUDA(cudaMemsetAsync(x32.get(), 0, sizeof(float) * L.n, s));
  cudaEvent_t e0, e1;
  LG_CUDA(cudaEventCreate(&e0));
  LG_CUDA(cudaEventCreate(&e1));
  int best = 0;
  float best_ms = 0.f;
  for (int E : {2, 4, 8}) {
    bin_rows(L.plan, L.n, L.rowptr.get(), E, s);
    const float ms = time_apply<double>(L, x.get(), y.get(), s, e0, e1) +
                     time_apply<float>(L, x32.get(), y32.get(), s, e0, e1);
    if (best == 0 || ms < best_ms) {
      best = E;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best != L.plan.plan.E) bin_rows(L.plan, L.n, L.rowptr.get(), best, s);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache.emplace(key, best);
}

// Release what an FP32-hierarchy solve never reads (option fp32_only): the
// FP64 copies of every operator but the finest (whose FP64 weights and row
// sums the outer PCG applies), the FP64 W = L P weights and elimination
// coefficients, and the kept vertices' rows of every elimination level
// below the finest. The level sizes (n, nnz) keep their logical values.
static void release_fp64_copies(Hier& h, cudaStream_t s, int64_t* counter) {
  for (size_t l = 0; l < h.levels.size(); ++l) {
    Level& L = *h.levels[l];
    if (L.kind == LG_LEVEL_COARSEST) continue;  // its FP64 pseudo-inverse is the coarsest solve
    L.lp_w.release();
    L.lp_d.release();
    L.pt_coef.release();
    L.dinv.release();
    if (l == 0) continue;
    L.w.release();
    L.d.release();
    if (L.kind != LG_LEVEL_ELIM || L.nnz == 0) continue;
    const int64_t n = L.n;
    DBuf<int64_t> nptr(n + 1, s, counter);
    k_frow_count<<<blocks_for(n), kNT, 0, s>>>(n, L.rowptr.get(), L.cmap.get(), nptr.get());
    LG_LAUNCH_CHECK();
    exclusive_scan(nptr.get(), nptr.get(), n, s);
    const int64_t kept = read_i64(nptr.get() + n, s);
    DBuf<int32_t> ncol(kept, s, counter);
    DBuf<float> nw32(kept, s, counter);
    k_frow_copy<<<blocks_for(n), kNT, 0, s>>>(n, L.rowptr.get(), L.col.get(), L.w32.get(), L.cmap.get(), nptr.get(),
                                              ncol.get(), nw32.get());
    LG_LAUNCH_CHECK();
    L.rowptr = std::move(nptr);
    L.col = std::move(ncol);
    L.w32 = std::move(nw32);
    L.plan = RowPlanStore();
    build_row_plan(L.plan, n, kept, L.rowptr.get(), s, counter);
  }
  h.fp32_only = true;
}

// While any setup runs, device memory its stages free stays in the device's
// stream-ordered pool instead of going back to the driver at each
// synchronisation, so that the next stage's allocation (tens of GB at scale
// 26) is not mapped again. The pool's threshold is put back when the last
// running setup ends; the memory held above it is released at the next
// synchronisation.
class PoolHold {
 public:
  explicit PoolHold(int device) {
    std::lock_guard<std::mutex> lk(mu());
    if (users()++ > 0) return;
    if (cudaDeviceGetDefaultMemPool(&pool(), device) != cudaSuccess) {
      cudaGetLastError();
      pool() = nullptr;
      return;
    }
    uint64_t keep = ~0ull;
    if (cudaMemPoolGetAttribute(pool(), cudaMemPoolAttrReleaseThreshold, &saved()) != cudaSuccess ||
        cudaMemPoolSetAttribute(pool(), cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
      cudaGetLastError();
      pool() = nullptr;
    }
  }
  ~PoolHold() {
    std::lock_guard<std::mutex> lk(mu());
    if (--users() > 0 || !pool()) return;
    if (cudaMemPoolSetAttribute(pool(), cudaMemPoolAttrReleaseThreshold, &saved()) != cudaSuccess) cudaGetLastError();
    pool() = nullptr;
  }
  PoolHold(const PoolHold&) = delete;
  PoolHold& operator=(const PoolHold&) = delete;

 private:
  static std::mutex& mu() {
    static std::mutex m;
    return m;
  }
  static int& users() {
    static int u = 0;
    return u;
  }
  static cudaMemPool_t& pool() {
    static cudaMemPool_t p = nullptr;
    return p;
  }
  static uint64_t& saved() {
    static uint64_t v = 0;
    return v;
  }
};

void setup_hierarchy(Hier& h, int64_t n, const int64_t* rowptr, const int32_t* col, const double* w) {
  PoolHold hold(h.device);
  cudaStream_t s = h.stream;
  const lg_options& o = h.opts;
  int64_t* counter = &h.bytes;
  if (o.elim_max_degree < 0 || o.elim_max_degree > 6) fail(LG_ERR_INVALID, "elim_max_degree must be 0..6");
  if (o.strength_vecs < 1 || o.strength_vecs > 7) fail(LG_ERR_INVALID, "strength_vecs must be 1..7");
  if (o.cheb_degree < 1 || o.cheb_degree > 8) fail(LG_ERR_INVALID, "cheb_degree must be 1..8");
  if (o.max_levels < 1) fail(LG_ERR_INVALID, "max_levels");
  if (o.elim_rounds < 1 || o.elim_rounds > 64) fail(LG_ERR_INVALID, "elim_rounds must be 1..64");
  if (o.reorder < 0 || o.reorder > 2) fail(LG_ERR_INVALID, "reorder must be 0, 1 or 2");
  if (o.fp32_only && o.precision != LG_FP32_HIER) fail(LG_ERR_INVALID, "fp32_only needs precision LG_FP32_HIER");

  h.dev_err.alloc(1, s);
  LG_CUDA(cudaMemsetAsync(h.dev_err.get(), 0, sizeof(int), s));
  cudaEvent_t e0, e1;
  LG_CUDA(cudaEventCreate(&e0));
  LG_CUDA(cudaEventCreate(&e1));
  LG_CUDA(cudaEventRecord(e0, s));
  StageClock clk;
  clk.on = h.time_stages;
  clk.s = s;
  clk.mark("start");

  // ---- level 0: copy the input and check the contract ----
  const int64_t nnz = read_i64(rowptr + n, s);
  auto cur = std::make_unique<Level>();
  cur->n = n;
  cur->nnz = nnz;
  cur->rowptr.alloc(n + 1, s, counter);
  cur->col.alloc(nnz, s, counter);
  cur->w.alloc(nnz, s, counter);
  LG_CUDA(cudaMemcpyAsync(cur->rowptr.get(), rowptr, sizeof(int64_t) * (n + 1), cudaMemcpyDefault, s));
  if (nnz > 0) {
    LG_CUDA(cudaMemcpyAsync(cur->col.get(), col, sizeof(int32_t) * nnz, cudaMemcpyDefault, s));
    LG_CUDA(cudaMemcpyAsync(cur->w.get(), w, sizeof(double) * nnz, cudaMemcpyDefault, s));
  }
  k_check_rowptr<<<blocks_for(n + 1), kNT, 0, s>>>(n, nnz, cur->rowptr.get(), h.dev_err.get());
  LG_LAUNCH_CHECK();
  if (read_err(h.dev_err, s)) fail(LG_ERR_INVALID, "rowptr");
  RowBinsStore in_bins;
  make_bins(in_bins, n, cur->rowptr.get(), s);
  DBuf<unsigned long long> sign(1, s);
  LG_CUDA(cudaMemsetAsync(sign.get(), 0, sizeof(unsigned long long), s));
  each_row(FCheck{n, cur->rowptr.get(), cur->col.get(), cur->w.get(), h.dev_err.get()}, cur->rowptr.get(),
           in_bins.bins, s, sign.get());
  unsigned long long sign_h = 0;
  LG_CUDA(cudaMemcpyAsync(&sign_h, sign.get(), sizeof(sign_h), cudaMemcpyDeviceToHost, s));
  if (read_err(h.dev_err, s) || sign_h != 0) fail(LG_ERR_INVALID, "graph entries");
  {
    DBuf<int32_t> parent(n, s);
    DBuf<uint8_t> is_root(n, s);
    DBuf<int64_t> cnt(n + 1, s);
    k_cc_init<<<blocks_for(n), kNT, 0, s>>>(n, parent.get());
    LG_LAUNCH_CHECK();
    each_row(FHook{n, cur->col.get(), parent.get(), h.dev_err.get()}, cur->rowptr.get(), in_bins.bins, s);
    k_cc_roots<<<blocks_for(n), kNT, 0, s>>>(n, parent.get(), is_root.get(), h.dev_err.get());
    LG_LAUNCH_CHECK();
    exclusive_scan_flags(is_root.get(), cnt.get(), n, s);
    const int64_t ncomp = read_i64(cnt.get() + n, s);
    if (read_err(h.dev_err, s)) fail(LG_ERR_TIMEOUT, "connected components did not settle");
    if (ncomp != 1) fail(LG_ERR_DISCONNECTED, "graph is not connected");
  }
  clk.mark("validate");
  h.nnz0 = nnz + n;
  h.perm.alloc(n, s, counter);
  if (o.reorder && n > 1) {
    DBuf<uint64_t> key(n, s), val(n, s);
    DBuf<int32_t> inv(n, s);
    if (o.reorder == 2)
      k_random_keys<<<blocks_for(n), kNT, 0, s>>>(n, o.seed, key.get(), val.get());
    else
      k_degree_keys<<<blocks_for(n), kNT, 0, s>>>(n, cur->rowptr.get(), key.get(), val.get());
    LG_LAUNCH_CHECK();
    radix_sort_pairs(key.get(), val.get(), n, 32, s);
    k_perm_from_sorted<<<blocks_for(n), kNT, 0, s>>>(n, val.get(), h.perm.get(), inv.get());
    LG_LAUNCH_CHECK();
    const int cbits = bits_for(n);
    DBuf<uint64_t> keys(nnz, s), vals(nnz, s);
    DBuf<int64_t> rp_new;
    if (o.row_sorts) {
      rp_new.alloc(n + 1, s, counter);
      k_perm_degrees<<<blocks_for(n), kNT, 0, s>>>(n, cur->rowptr.get(), inv.get(), rp_new.get());
      LG_LAUNCH_CHECK();
      exclusive_scan(rp_new.get(), rp_new.get(), n, s);
    }
    each_row(FPermEmit{cur->col.get(), cur->w.get(), inv.get(), rp_new.get(), cbits, keys.get(), vals.get()},
             cur->rowptr.get(), in_bins.bins, s);
    if (o.row_sorts) {
      // the validated input repeats no entry, so the rows sorted in place are
      // the renumbered CSR as they stand (no sums: the accumulation would
      // reproduce them value for value)
      sort_within_rows(keys, vals, nnz, rp_new.get(), n, cbits, s);
      DBuf<int32_t> ncol(nnz, s, counter);
      DBuf<double> nw(nnz, s, counter);
      k_unpack_entries<<<blocks_for(nnz), kNT, 0, s>>>(nnz, keys.get(), vals.get(), (1ull << cbits) - 1ull,
                                                      ncol.get(), nw.get());
      LG_LAUNCH_CHECK();
      cur->rowptr = std::move(rp_new);
      cur->col = std::move(ncol);
      cur->w = std::move(nw);
    } else {
      CsrOut out;
      accumulate_csr(keys, vals, nnz, n, cbits, out, s, counter);
      cur->rowptr = std::move(out.rowptr);
      cur->col = std::move(out.col);
      cur->w = std::move(out.w);
    }
  } else {
    k_iota_i32<<<blocks_for(n), kNT, 0, s>>>(n, h.perm.get());
    LG_LAUNCH_CHECK();
  }
  clk.mark("reorder");
  prepare_operator(*cur, s, counter);
  clk.mark("operator_plans");

  // ---- coarsening loop ----
  DBuf<Lanczos> lz_dev(o.max_levels + 1, s);  // each aggregation level's Lanczos recursion
  std::vector<int> lam_level;
  auto stop = [&](const Level& L) {
    return (double)(L.nnz + L.n) <= o.coarse_nnz || (int)h.levels.size() >= o.max_levels - 1;
  };
  for (;;) {
    if (stop(*cur)) break;
    // up to elim_rounds elimination levels in a row, each while the gate passes
    bool done = false;
    for (int round = 0; o.elim_enable && o.elim_max_degree > 0 && round < o.elim_rounds; ++round) {
      NvtxRange range("lg elimination level");
      DBuf<uint8_t> is_f(cur->n, s);
      const int64_t nf = run_elim_select(cur->n, cur->rowptr.get(), cur->col.get(), o.elim_max_degree, o.seed,
                                         is_f.get(), s);
      clk.mark("elim_select");
      if (!((double)nf > o.elim_min_frac * (double)cur->n)) break;
      auto next = eliminate(*cur, is_f.get(), nf, o.row_sorts != 0, s, counter);
      clk.mark("elim_schur");
      h.levels.push_back(std::move(cur));
      cur = std::move(next);
      prepare_operator(*cur, s, counter);
      clk.mark("operator_plans");
      if (stop(*cur)) {
        done = true;
        break;
      }
    }
    if (done) break;
    NvtxRange range("lg aggregation level");
    const int level = (int)h.levels.size();
    DBuf<double> S(cur->nnz, s);
    // the level's bins match those lg_strength / lg_aggregate derive for the same CSR (E = 4,
    // before autotuning), so the strength values here are bitwise those of the single steps
    const RowBins bins = bins_of(cur->plan.plan, cur->n);
    run_strength(cur->n, cur->rowptr.get(), cur->col.get(), cur->w.get(), o.seed, level, o.strength_vecs,
                 o.strength_sweeps, o.jacobi_omega, S.get(), s, &bins);
    clk.mark("strength");
    cur->agg.alloc(cur->n, s, counter);
    const int64_t nc = run_aggregate(cur->n, cur->rowptr.get(), cur->col.get(), S.get(), o.agg_iters,
                                     o.vote_threshold, cur->agg.get(), nullptr, nullptr, s, &bins);
    clk.mark("aggregate");
    if ((double)nc > o.stagnation_frac * (double)cur->n) {
      cur->agg.release();
      break;
    }
    cur->kind = LG_LEVEL_AGG;
    cur->nc = nc;
    lanczos(*cur, o, level, lz_dev.get() + level, s);
    clk.mark("lanczos");
    lam_level.push_back(level);
    auto next = galerkin(*cur, o.lp_residual != 0, o.row_sorts != 0, s, counter, clk);
    h.levels.push_back(std::move(cur));
    cur = std::move(next);
    prepare_operator(*cur, s, counter);
    clk.mark("operator_plans");
  }
  if (cur->n > o.max_coarse_n) fail(LG_ERR_SETUP, "coarsest level too large for the dense solve");
  {
    NvtxRange range("lg coarsest pseudo-inverse");
    coarsest_pinv(*cur, h.dev_err.get(), s, counter);
  }
  clk.mark("coarsest_pinv");
  h.levels.push_back(std::move(cur));
  if (o.const_weights) detect_constant_weights(*h.levels[0], s);
  clk.mark("constant_weights");
  for (auto& L : h.levels) make_f32(*L, s, counter);
  clk.mark("fp32_copies");
  if (read_err(h.dev_err, s)) fail(LG_ERR_SETUP, "coarsest pseudo-inverse failed");
  if (o.autotune) {
    NvtxRange range("lg row-binning tuner");
    for (auto& L : h.levels) {
      if (L->nnz < 20000) continue;
      tune_level(*L, s);
    }
  }
  clk.mark("autotune");
  if (o.fp32_only) {
    release_fp64_copies(h, s, counter);
    clk.mark("fp32_only_release");
  }

  h.first_agg = -1;
  for (size_t l = 0; l < h.levels.size() && h.first_agg < 0; ++l)
    if (h.levels[l]->kind == LG_LEVEL_AGG) h.first_agg = (int)l;

  // ---- Chebyshev constants from the eigenvalue estimates ----
  std::vector<Lanczos> lz(h.levels.size());
  LG_CUDA(cudaMemcpyAsync(lz.data(), lz_dev.get(), sizeof(Lanczos) * h.levels.size(), cudaMemcpyDeviceToHost, s));
  LG_CUDA(cudaEventRecord(e1, s));
  LG_CUDA(cudaStreamSynchronize(s));
  float ms = 0.f;
  LG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  h.setup_ms = ms;
  h.setup_stages = clk.collect();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h.cheb.assign(h.levels.size(), Cheb{});
  for (int l : lam_level) {
    Level& L = *h.levels[l];
    L.lambda = ritz_max(lz[l]);
    const double a = o.cheb_lo * L.lambda, b = o.cheb_hi * L.lambda;
    const double theta = 0.5 * (b + a), delta = 0.5 * (b - a);
    const double sigma = theta / delta;
    Cheb& c = h.cheb[l];
    c.inv_theta = 1.0 / theta;
    double rho = 1.0 / sigma;
    for (int st = 1; st < o.cheb_degree && st < 8; ++st) {
      const double rn = 1.0 / (2.0 * sigma - rho);
      c.c1[st] = rn * rho;
      c.c2[st] = 2.0 * rn / delta;
      rho = rn;
    }
  }
}

}  // namespace lg
