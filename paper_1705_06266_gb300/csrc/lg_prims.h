// Host-callable device primitives: scans, stable radix sort, sort-based
// sparse accumulation, and the SpMV row plan.
#pragma once

#include "lg_common.cuh"

namespace lg {

// out[i] = sum_{j<i} in[i]; out[n] = total. `in` and `out` may alias. Returns
// nothing; read out[n] for the total.
void exclusive_scan(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s);
// Same over int32 inputs (out is int64).
void exclusive_scan32(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s);
// Exclusive scan of the predicate flag[i] != 0 (uint8).
void exclusive_scan_flags(const uint8_t* flag, int64_t* out, int64_t n, cudaStream_t s);

// Stable LSD radix sort of (key, val) pairs on the low `bits` bits of key.
// keys/vals are sorted in place (tmp buffers are allocated internally).
void radix_sort_pairs(uint64_t* keys, uint64_t* vals, int64_t n, int bits, cudaStream_t s);

// Stable sort of the entries of each group [rp[g], rp[g+1]) by key, for
// entries emitted grouped by row (the row bits of the key equal within a
// group and ascending from group to group), which then end up sorted as a
// global stable sort would leave them. keys/vals are sorted in place; the
// scratch is bounded (rows of more than 16384 entries are sorted a batch of
// about 2^28 entries at a time).
void sort_within_rows(DBuf<uint64_t>& keys, DBuf<uint64_t>& vals, int64_t nent, const int64_t* rp, int64_t ngroups,
                      int cbits, cudaStream_t s);

// Sparse accumulation: entries (key = row << cbits | col, value) are sorted
// stably by key and equal keys summed in their input order. Produces a CSR
// with nrows rows: rowptr (nrows+1), col, w. `vals` holds doubles bit-cast to
// uint64. Returns the number of distinct entries. With `grouped` (ngroups + 1
// offsets), the entries come grouped by row as sort_within_rows takes them
// and are sorted within their groups instead of globally.
struct CsrOut {
  DBuf<int64_t> rowptr;
  DBuf<int32_t> col;
  DBuf<double> w;
  int64_t nnz = 0;
};
void accumulate_csr(DBuf<uint64_t>& keys, DBuf<uint64_t>& vals, int64_t nent, int64_t nrows,
                    int cbits, CsrOut& out, cudaStream_t s, int64_t* counter, const int64_t* grouped = nullptr,
                    int64_t ngroups = 0);

// Bits needed to hold values 0..v-1.
inline int bits_for(int64_t v) {
  int b = 1;
  while (b < 62 && (int64_t(1) << b) < v) ++b;
  return b;
}

// Owned storage of a RowPlan.
struct RowPlanStore {
  RowPlan plan;
  DBuf<int32_t> rows_by_class, chunk_row, chunk_lrow, lrow_first, lrow_count;
  DBuf<int64_t> chunk_beg;
  DBuf<double> partial;
  DBuf<unsigned> ticket;
  DBuf<int32_t> seg_tile_off, vrow_row;
  DBuf<int64_t> vrow_beg, vrow_end;
};
// Rows of a CSR structure grouped by length for the setup passes (lg_each.cuh):
// class c < kClasses holds rows of at most E 2^c entries (the last class: at
// most kChunk) and is visited by groups of 2^c lanes, kEachThreads / 2^c rows
// per block; each row longer than kChunk gets a block of its own. Blocks are
// ordered long rows first, then classes from the longest rows down, so the
// heaviest work starts first.
constexpr int kEachThreads = 256;
struct RowBins {
  const int32_t* rows = nullptr;    // row ids class by class, long rows last
  int64_t off[kClasses + 2] = {0};  // class c: rows[off[c], off[c+1]); long rows: [off[kClasses], off[kClasses+1])
  int blk[kClasses] = {0};          // first block of class c
  int grid = 0;
};
// The bins of a built plan (its classes and long rows).
RowBins bins_of(const RowPlan& p, int64_t n);
// Bins of a CSR structure without a plan (E = 4), owning the row list.
struct RowBinsStore {
  DBuf<int32_t> rows;
  RowBins bins;
};
void make_bins(RowBinsStore& b, int64_t n, const int64_t* rowptr, cudaStream_t s);

// Build the plan for a CSR structure with n rows and nnz entries (rows binned
// with E = 4 entries per lane). ncols > 0 (the length of the vector the rows
// gather from) lets the long rows be served column-segmented when that
// vector is short enough next to their entries (see RowPlan).
void build_row_plan(RowPlanStore& ps, int64_t n, int64_t nnz, const int64_t* rowptr, cudaStream_t s,
                    int64_t* counter, int64_t ncols = 0);
// Re-bin the rows of a built plan for E entries per lane.
void bin_rows(RowPlanStore& ps, int64_t n, const int64_t* rowptr, int E, cudaStream_t s);

}  // namespace lg
