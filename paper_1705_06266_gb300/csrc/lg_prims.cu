// Device primitives: scans, stable LSD radix sort, sort-based sparse
// accumulation and the SpMV row plan.
#include <algorithm>
#include <vector>

#include "lg_prims.h"

namespace lg {

// ---------------------------------------------------------------------------
// Exclusive scan (reduce - scan block sums - scan with offsets).
// ---------------------------------------------------------------------------
constexpr int kScanNT = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanNT * kScanItems;

struct LoadI64 { const int64_t* p; __device__ int64_t operator()(int64_t i) const { return p[i]; } };
struct LoadI32 { const int32_t* p; __device__ int64_t operator()(int64_t i) const { return p[i]; } };
struct LoadFlag { const uint8_t* p; __device__ int64_t operator()(int64_t i) const { return p[i] != 0; } };

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t* total) {
  __shared__ int64_t wsum[kScanNT / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int64_t t = lane < kScanNT / 32 ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < kScanNT / 32) wsum[lane] = t;
  }
  __syncthreads();
  int64_t before = (wid > 0 ? wsum[wid - 1] : 0) + x - v;
  if (total) *total = wsum[kScanNT / 32 - 1];
  __syncthreads();
  return before;
}

template <class Load>
__global__ void __launch_bounds__(kScanNT) k_scan_reduce(Load ld, int64_t n, int64_t* bsum) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int64_t acc = 0;
  for (int i = threadIdx.x; i < kScanTile; i += kScanNT) {
    int64_t idx = base + i;
    if (idx < n) acc += ld(idx);
  }
  int64_t tot;
  block_exclusive_scan(acc, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// Exclusive scan of bsum[0..nb) in place by one block; writes the grand total to *total_out.
__global__ void __launch_bounds__(kScanNT) k_scan_blocks(int64_t* bsum, int64_t nb, int64_t* total_out) {
  int64_t carry = 0;
  for (int64_t base = 0; base < nb; base += kScanNT) {
    int64_t i = base + threadIdx.x;
    int64_t v = i < nb ? bsum[i] : 0;
    int64_t tot;
    int64_t ex = block_exclusive_scan(v, &tot);
    if (i < nb) bsum[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) *total_out = carry;
}

template <class Load>
__global__ void __launch_bounds__(kScanNT) k_scan_final(Load ld, int64_t n, const int64_t* bsum, int64_t* out) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t sum = 0;
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    int64_t idx = base + q;
    v[q] = idx < n ? ld(idx) : 0;
    sum += v[q];
  }
  int64_t run = bsum[blockIdx.x] + block_exclusive_scan(sum, nullptr);
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    int64_t idx = base + q;
    if (idx < n) out[idx] = run;
    run += v[q];
  }
}

template <class Load>
static void scan_impl(Load ld, int64_t* out, int64_t n, cudaStream_t s) {
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb == 0) {
    LG_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
    return;
  }
  DBuf<int64_t> bsum(nb, s);
  k_scan_reduce<<<(unsigned)nb, kScanNT, 0, s>>>(ld, n, bsum.get());
  LG_LAUNCH_CHECK();
  k_scan_blocks<<<1, kScanNT, 0, s>>>(bsum.get(), nb, out + n);
  LG_LAUNCH_CHECK();
  k_scan_final<<<(unsigned)nb, kScanNT, 0, s>>>(ld, n, bsum.get(), out);
  LG_LAUNCH_CHECK();
}

void exclusive_scan(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) {
  scan_impl(LoadI64{in}, out, n, s);
}
void exclusive_scan32(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s) {
  scan_impl(LoadI32{in}, out, n, s);
}
void exclusive_scan_flags(const uint8_t* flag, int64_t* out, int64_t n, cudaStream_t s) {
  scan_impl(LoadFlag{flag}, out, n, s);
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort, 8-bit digits. Per pass: a per-tile digit histogram,
// an exclusive scan of the digit-major histogram (digit, tile), and a
// scatter in which each warp ranks its 256 consecutive elements with
// __match_any_sync; element order inside a tile is (warp, round, lane), so
// equal digits keep their input order.
// ---------------------------------------------------------------------------
constexpr int kRsNT = 256;
constexpr int kRsWarps = kRsNT / 32;
constexpr int kRsRounds = 8;
constexpr int kRsTile = kRsNT * kRsRounds;
constexpr int kRadix = 256;

__global__ void __launch_bounds__(kRsNT) k_rs_hist(const uint64_t* __restrict__ keys, int64_t n, int shift,
                                                     int32_t* __restrict__ hist, int64_t ntiles) {
  __shared__ uint32_t h[kRadix];
  for (int d = threadIdx.x; d < kRadix; d += kRsNT) h[d] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRsTile;
  for (int i = threadIdx.x; i < kRsTile; i += kRsNT) {
    int64_t idx = base + i;
    if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 0xff], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += kRsNT) hist[(int64_t)d * ntiles + blockIdx.x] = (int32_t)h[d];
}

__global__ void __launch_bounds__(kRsNT) k_rs_scatter(const uint64_t* __restrict__ kin, const uint64_t* __restrict__ vin,
                                                        uint64_t* __restrict__ kout, uint64_t* __restrict__ vout,
                                                        int64_t n, int shift, const int64_t* __restrict__ off,
                                                        int64_t ntiles) {
  __shared__ int64_t start[kRsWarps][kRadix];
  __shared__ uint32_t cnt[kRsWarps][kRadix];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kRsWarps * kRadix; i += kRsNT) (&cnt[0][0])[i] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRsTile + (int64_t)warp * (kRsRounds * 32);
  uint64_t k[kRsRounds], v[kRsRounds];
  uint32_t dg[kRsRounds];
#pragma unroll
  for (int r = 0; r < kRsRounds; ++r) {
    int64_t e = base + r * 32 + lane;
    if (e < n) {
      k[r] = kin[e];
      v[r] = vin[e];
      dg[r] = (uint32_t)((k[r] >> shift) & 0xff);
    } else {
      dg[r] = 0xffffffffu;
    }
  }
  // count each digit per warp
#pragma unroll
  for (int r = 0; r < kRsRounds; ++r) {
    bool valid = dg[r] != 0xffffffffu;
    unsigned active = __ballot_sync(0xffffffffu, valid);
    if (valid) {
      unsigned peers = __match_any_sync(active, dg[r]);
      if (lane == __ffs(peers) - 1) cnt[warp][dg[r]] += __popc(peers);
    }
    __syncwarp();
  }
  __syncthreads();
  // start of each (warp, digit) run in the output
  for (int d = threadIdx.x; d < kRadix; d += kRsNT) {
    int64_t run = off[(int64_t)d * ntiles + blockIdx.x];
    for (int w = 0; w < kRsWarps; ++w) {
      start[w][d] = run;
      run += cnt[w][d];
    }
  }
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < kRsRounds; ++r) {
    bool valid = dg[r] != 0xffffffffu;
    unsigned active = __ballot_sync(0xffffffffu, valid);
    unsigned peers = 0;
    int64_t pos = 0;
    if (valid) {
      peers = __match_any_sync(active, dg[r]);
      pos = start[warp][dg[r]] + __popc(peers & lt);
      kout[pos] = k[r];
      vout[pos] = v[r];
    }
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) start[warp][dg[r]] += __popc(peers);
    __syncwarp();
  }
}

void radix_sort_pairs(uint64_t* keys, uint64_t* vals, int64_t n, int bits, cudaStream_t s) {
  if (n <= 1) return;
  const int64_t ntiles = (n + kRsTile - 1) / kRsTile;
  DBuf<uint64_t> k2(n, s), v2(n, s);
  DBuf<int32_t> hist((size_t)kRadix * ntiles, s);
  DBuf<int64_t> off((size_t)kRadix * ntiles + 1, s);
  uint64_t *ka = keys, *va = vals, *kb = k2.get(), *vb = v2.get();
  const int passes = (bits + 7) / 8;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    k_rs_hist<<<(unsigned)ntiles, kRsNT, 0, s>>>(ka, n, shift, hist.get(), ntiles);
    LG_LAUNCH_CHECK();
    exclusive_scan32(hist.get(), off.get(), (int64_t)kRadix * ntiles, s);
    k_rs_scatter<<<(unsigned)ntiles, kRsNT, 0, s>>>(ka, va, kb, vb, n, shift, off.get(), ntiles);
    LG_LAUNCH_CHECK();
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (ka != keys) {
    LG_CUDA(cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
    LG_CUDA(cudaMemcpyAsync(vals, va, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
  }
}

// ---------------------------------------------------------------------------
// Sparse accumulation by sorted keys.
// ---------------------------------------------------------------------------
__global__ void k_seg_heads(const uint64_t* __restrict__ keys, int64_t n, uint8_t* __restrict__ head) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    head[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

__global__ void k_seg_starts(const uint8_t* __restrict__ head, const int64_t* __restrict__ segid, int64_t n,
                             int64_t* __restrict__ start) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (head[i]) start[segid[i]] = i;
}

// One thread per distinct key: the sum of its run in input order.
__global__ void k_seg_sum(const uint64_t* __restrict__ keys, const uint64_t* __restrict__ vals,
                          const int64_t* __restrict__ start, int64_t nseg, int64_t n, uint64_t cmask,
                          int32_t* __restrict__ col, double* __restrict__ w, uint64_t* __restrict__ segkey) {
  for (int64_t sgi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; sgi < nseg; sgi += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = start[sgi], e = (sgi + 1 < nseg) ? start[sgi + 1] : n;
    double acc = 0.0;
    for (int64_t q = b; q < e; ++q) acc += __longlong_as_double((long long)vals[q]);
    const uint64_t key = keys[b];
    col[sgi] = (int32_t)(key & cmask);
    w[sgi] = acc;
    segkey[sgi] = key;
  }
}

// rowptr[r] = number of distinct keys whose row is below r.
__global__ void k_rowptr_from_keys(const uint64_t* __restrict__ segkey, int64_t nseg, int cbits, int64_t nrows,
                                   int64_t* __restrict__ rowptr) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r <= nrows; r += (int64_t)gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = nseg;
    while (lo < hi) {
      int64_t mid = (lo + hi) >> 1;
      if ((int64_t)(segkey[mid] >> cbits) < r) lo = mid + 1; else hi = mid;
    }
    rowptr[r] = lo;
  }
}

// ---------------------------------------------------------------------------
// Sort within rows. When the entries come grouped by row (row r's at
// [rp[r], rp[r+1]) in the order they were emitted, the rows' key bits equal
// within a row and ascending from row to row), sorting every row's entries
// stably by key gives the order a global stable sort would, with one read
// and one write of the entries instead of one per 8 key bits. In place, by
// length:
//  - rows of at most 32 entries: a group of 2^c lanes per row, each entry
//    ranked by comparing it with the others (ties by position);
//  - rows of at most 512 entries: one block per row, a bitonic network in
//    shared memory over (column, position) pairs, which are distinct, so the
//    result is the stable order;
//  - rows of at most kWrBlockMax entries: one block per row, a stable LSD
//    radix sort of the row in shared memory (k_wr_radix);
//  - rows of at most kWrOneBlockMax entries: one block per row, the same radix
//    sort with the row's columns and positions in global scratch
//    (k_wr_radix_long), a batch of rows of about kWrBatch entries at a time,
//    which bounds the scratch;
//  - longer rows (the hubs'): one block would take too long over one of
//    them, so they are gathered, a batch at a time, into one array keyed
//    (index in the batch, column), radix sorted together by the whole GPU and
//    written back.
// Rows are independent, so which block takes which row does not matter.
// ---------------------------------------------------------------------------
constexpr int kWrBlockMax = 16384;
constexpr int64_t kWrOneBlockMax = 65536;
constexpr int64_t kWrBatch = int64_t(1) << 28;
constexpr int kWrClasses = 17;  // 0: <= 1 entry; 1..5: lane groups; 6..14: blocks of 2^c; 15: long; 16: hub

__device__ __forceinline__ int wr_class(int64_t len) {
  if (len <= 1) return 0;
  if (len > kWrOneBlockMax) return kWrClasses - 1;
  if (len > kWrBlockMax) return kWrClasses - 2;
  int c = 1;
  while ((int64_t(1) << c) < len) ++c;
  return c;
}

// Pass 0 counts the rows of each class; pass 1 lists them (off: class offsets,
// fill: per-class cursors). One block-level histogram per block.
__global__ void k_wr_bin(int64_t nrows, const int64_t* __restrict__ rp, int pass, int64_t* __restrict__ cnt,
                         const int64_t* __restrict__ off, unsigned long long* __restrict__ fill,
                         int32_t* __restrict__ rows) {
  __shared__ unsigned int h[kWrClasses];
  __shared__ unsigned long long base[kWrClasses];
  const int64_t per = (nrows + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * per, r1 = r0 + per < nrows ? r0 + per : nrows;
  if (threadIdx.x < kWrClasses) h[threadIdx.x] = 0;
  __syncthreads();
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) atomicAdd(&h[wr_class(rp[r + 1] - rp[r])], 1u);
  __syncthreads();
  if (pass == 0) {
    if (threadIdx.x < kWrClasses && h[threadIdx.x]) atomicAdd((unsigned long long*)&cnt[threadIdx.x], h[threadIdx.x]);
    return;
  }
  if (threadIdx.x < kWrClasses) {
    base[threadIdx.x] = h[threadIdx.x] ? (unsigned long long)off[threadIdx.x] + atomicAdd(&fill[threadIdx.x], h[threadIdx.x]) : 0ull;
    h[threadIdx.x] = 0;
  }
  __syncthreads();
  for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    const int c = wr_class(rp[r + 1] - rp[r]);
    rows[base[c] + atomicAdd(&h[c], 1u)] = (int32_t)r;
  }
}

// Rows of at most G entries, one group of G lanes each. Every lane of a group
// reads its entry before the shuffles, so the writes may overwrite the row.
template <int G>
__global__ void k_wr_rank(const int32_t* __restrict__ rows, int64_t nr, const int64_t* __restrict__ rp,
                          uint64_t* keys, uint64_t* vals) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t gi = t / G;
  const int l = (int)(t & (G - 1));
  int64_t b = 0;
  int len = 0;
  if (gi < nr) {
    const int32_t r = rows[gi];
    b = rp[r];
    len = (int)(rp[r + 1] - b);
  }
  uint64_t k = ~0ull, v = 0;
  if (l < len) {
    k = keys[b + l];
    v = vals[b + l];
  }
  int rank = 0;
#pragma unroll
  for (int m = 0; m < G; ++m) {
    const uint64_t km = __shfl_sync(0xffffffffu, k, m, G);
    rank += (m < len) & ((km < k) | ((km == k) & (m < l)));
  }
  if (l < len) {
    keys[b + rank] = k;
    vals[b + rank] = v;
  }
}

// Rows of at most P entries (P a power of two, 64..512), one block each; the
// row's values are held in shared memory beside the pairs.
template <int P>
__global__ void __launch_bounds__(P / 2)
k_wr_block(const int32_t* __restrict__ rows, const int64_t* __restrict__ rp, uint64_t* keys, uint64_t* vals,
           uint64_t cmask) {
  constexpr int T = P / 2;
  constexpr int PB = P <= 64 ? 6 : P <= 128 ? 7 : P <= 256 ? 8 : 9;
  static_assert((1 << PB) == P, "P must be a power of two, 64..512");
  extern __shared__ uint64_t wr_sk[];  // P pairs, then P values
  uint64_t* sv = wr_sk + P;
  const int32_t r = rows[blockIdx.x];
  const int64_t b = rp[r];
  const int len = (int)(rp[r + 1] - b);
  const uint64_t rowbits = keys[b] & ~cmask;
  for (int i = threadIdx.x; i < P; i += T) {
    if (i < len) {
      wr_sk[i] = ((keys[b + i] & cmask) << PB) | (uint64_t)i;
      sv[i] = vals[b + i];
    } else {
      wr_sk[i] = ~0ull;
    }
  }
  __syncthreads();
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < P / 2; t += T) {
        const int lo = 2 * t - (t & (stride - 1)), hi = lo + stride;
        const uint64_t a = wr_sk[lo], c = wr_sk[hi];
        if ((a > c) == ((lo & size) == 0)) {
          wr_sk[lo] = c;
          wr_sk[hi] = a;
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < len; i += T) {
    const uint64_t c = wr_sk[i];
    keys[b + i] = rowbits | (c >> PB);
    vals[b + i] = sv[c & (uint64_t)(P - 1)];
  }
}

// Hub rows of one batch: to one array, keyed (index in the batch, column), and back.
__global__ void k_wr_gather(const int32_t* __restrict__ lrows, const int64_t* __restrict__ rp,
                            const int64_t* __restrict__ loff, int64_t o0, const uint64_t* __restrict__ keys,
                            const uint64_t* __restrict__ vals, uint64_t* __restrict__ tk, uint64_t* __restrict__ tv,
                            int cbits) {
  const int32_t r = lrows[blockIdx.x];
  const int64_t b = rp[r], len = rp[r + 1] - b, o = loff[blockIdx.x] - o0;
  const uint64_t cmask = (1ull << cbits) - 1ull;
  for (int64_t q = threadIdx.x; q < len; q += blockDim.x) {
    tk[o + q] = ((uint64_t)blockIdx.x << cbits) | (keys[b + q] & cmask);
    tv[o + q] = vals[b + q];
  }
}

__global__ void k_wr_scatter(const int32_t* __restrict__ lrows, const int64_t* __restrict__ rp,
                             const int64_t* __restrict__ loff, int64_t o0, const uint64_t* __restrict__ tk,
                             const uint64_t* __restrict__ tv, uint64_t* keys, uint64_t* vals, int cbits) {
  const int32_t r = lrows[blockIdx.x];
  const int64_t b = rp[r], len = rp[r + 1] - b, o = loff[blockIdx.x] - o0;
  const uint64_t cmask = (1ull << cbits) - 1ull;
  const uint64_t rowbits = keys[b] & ~cmask;  // every entry of the row has the same row bits
  __syncthreads();  // the block's reads of keys[b] come before any write to the row
  for (int64_t q = threadIdx.x; q < len; q += blockDim.x) {
    keys[b + q] = rowbits | (tk[o + q] & cmask);
    vals[b + q] = tv[o + q];
  }
}

__global__ void k_wr_long_len(const int32_t* __restrict__ lrows, int64_t nl, const int64_t* __restrict__ rp,
                              int64_t* __restrict__ len) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nl; q += (int64_t)gridDim.x * blockDim.x)
    len[q] = rp[lrows[q] + 1] - rp[lrows[q]];
}

// Rows of at most P entries (P a power of two, 1024..kWrBlockMax), one block
// each: a stable LSD radix sort in shared memory over the column bits, 8 a
// pass. The row's columns stay in place (32-bit); each pass moves 16-bit
// positions. A warp takes a contiguous stretch of the current order, 32
// positions a round, and ranks the entries of a digit by (warp, round, lane),
// so equal digits keep their order and the result is the stable order. The
// values are gathered into registers at the end, every read of the row
// before the first write.
template <int P>
__global__ void __launch_bounds__(P / 4 < 1024 ? P / 4 : 1024)
k_wr_radix(const int32_t* __restrict__ rows, const int64_t* __restrict__ rp, uint64_t* keys, uint64_t* vals,
           int cbits) {
  constexpr int T = P / 4 < 1024 ? P / 4 : 1024;
  constexpr int W = T / 32;       // warps
  constexpr int EPT = P / T;      // positions per lane
  static_assert(P <= 65536, "positions are 16-bit");
  extern __shared__ __align__(16) unsigned char wr_raw[];
  uint32_t* scol = reinterpret_cast<uint32_t*>(wr_raw);            // P columns
  uint16_t* ia = reinterpret_cast<uint16_t*>(scol + P);            // P positions
  uint16_t* ib = ia + P;                                            // P positions
  uint16_t* cnt = ib + P;                                           // W x 256 counts, then starts
  __shared__ uint32_t wsum[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int32_t r = rows[blockIdx.x];
  const int64_t b = rp[r];
  const int len = (int)(rp[r + 1] - b);
  const uint64_t cmask = (1ull << cbits) - 1ull;
  const uint64_t rowbits = keys[b] & ~cmask;
  for (int i = threadIdx.x; i < len; i += T) {
    scol[i] = (uint32_t)(keys[b + i] & cmask);
    ia[i] = (uint16_t)i;
  }
  uint16_t *in = ia, *out = ib;
  for (int shift = 0; shift < cbits; shift += 8) {
    for (int i = threadIdx.x; i < W * 256; i += T) cnt[i] = 0;
    __syncthreads();
    const int base = warp * EPT * 32;
    // counts per (warp, digit)
    for (int q = 0; q < EPT; ++q) {
      const int pos = base + q * 32 + lane;
      const bool valid = pos < len;
      const unsigned act = __ballot_sync(0xffffffffu, valid);
      if (valid) {
        const unsigned d = (scol[in[pos]] >> shift) & 255u;
        const unsigned peers = __match_any_sync(act, d);
        if ((peers & lt) == 0) cnt[warp * 256 + d] += (uint16_t)__popc(peers);
      }
      __syncwarp();
    }
    __syncthreads();
    // starts: digit-major, then warp
    if (threadIdx.x < 256) {
      const int d = threadIdx.x;
      uint32_t tot = 0;
      for (int w = 0; w < W; ++w) tot += cnt[w * 256 + d];
      uint32_t x = tot;  // inclusive scan over the 256 digits
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) wsum[warp] = x;
      __syncwarp();
      asm volatile("bar.sync 1, 256;");
      uint32_t before = x - tot;
      for (int w = 0; w < warp; ++w) before += wsum[w];
      for (int w = 0; w < W; ++w) {
        const uint16_t c = cnt[w * 256 + d];
        cnt[w * 256 + d] = (uint16_t)before;
        before += c;
      }
    }
    __syncthreads();
    // scatter
    for (int q = 0; q < EPT; ++q) {
      const int pos = base + q * 32 + lane;
      const bool valid = pos < len;
      const unsigned act = __ballot_sync(0xffffffffu, valid);
      unsigned d = 0, peers = 0;
      uint16_t e = 0;
      if (valid) {
        e = in[pos];
        d = (scol[e] >> shift) & 255u;
        peers = __match_any_sync(act, d);
        out[cnt[warp * 256 + d] + __popc(peers & lt)] = e;
      }
      __syncwarp();
      if (valid && (peers & lt) == 0) cnt[warp * 256 + d] += (uint16_t)__popc(peers);
      __syncwarp();
    }
    __syncthreads();
    uint16_t* t = in;
    in = out;
    out = t;
  }
  uint64_t v[EPT];
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const int i = threadIdx.x + q * T;
    if (i < len) v[q] = vals[b + in[i]];
  }
  __syncthreads();  // every value of the row is read before the row is overwritten
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const int i = threadIdx.x + q * T;
    if (i < len) {
      keys[b + i] = rowbits | scol[in[i]];
      vals[b + i] = v[q];
    }
  }
}

template <int P>
static void wr_radix_launch(const int32_t* rows, int64_t nr, const int64_t* rp, uint64_t* keys, uint64_t* vals,
                            int cbits, cudaStream_t s) {
  constexpr int T = P / 4 < 1024 ? P / 4 : 1024;
  const size_t smem = (size_t)P * (4 + 2 + 2) + (size_t)(T / 32) * 256 * 2;
  // the kernel's own static shared memory counts against the same 48 KB default
  LG_CUDA(cudaFuncSetAttribute(k_wr_radix<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  for (int64_t q0 = 0; q0 < nr; q0 += 1 << 30) {
    const int64_t m = nr - q0 < (1 << 30) ? nr - q0 : (1 << 30);
    k_wr_radix<P><<<(unsigned)m, T, smem, s>>>(rows + q0, rp, keys, vals, cbits);
    LG_LAUNCH_CHECK();
  }
}

template <int P>
static void wr_block_launch(const int32_t* rows, int64_t nr, const int64_t* rp, uint64_t* keys, uint64_t* vals,
                            uint64_t cmask, cudaStream_t s) {
  constexpr int T = P / 2;
  const size_t smem = 2 * sizeof(uint64_t) * P;
  for (int64_t q0 = 0; q0 < nr; q0 += 1 << 30) {
    const int64_t m = nr - q0 < (1 << 30) ? nr - q0 : (1 << 30);
    k_wr_block<P><<<(unsigned)m, T, smem, s>>>(rows + q0, rp, keys, vals, cmask);
    LG_LAUNCH_CHECK();
  }
}

// A long row, one block: the same stable LSD radix sort as k_wr_radix, with
// the row's columns and positions in global scratch at o (this row's offset
// in the batch) instead of shared memory. Warp w ranks the w-th contiguous
// stretch of the current order, 32 positions a round, so equal digits keep
// their order. At the end the values go through scratch (tv), every read of
// the row before the first write.
constexpr int kWrLongThreads = 1024;
__global__ void __launch_bounds__(kWrLongThreads)
k_wr_radix_long(const int32_t* __restrict__ lrows, const int64_t* __restrict__ rp, const int64_t* __restrict__ loff,
                int64_t o0, uint64_t* keys, uint64_t* vals, uint32_t* __restrict__ scol, uint32_t* __restrict__ pa,
                uint32_t* __restrict__ pb, uint64_t* __restrict__ tv, int cbits) {
  constexpr int W = kWrLongThreads / 32;
  __shared__ uint32_t cnt[W * 256];
  __shared__ uint32_t wsum[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int32_t r = lrows[blockIdx.x];
  const int64_t b = rp[r];
  const int64_t len = rp[r + 1] - b, o = loff[blockIdx.x] - o0;
  const uint64_t cmask = (1ull << cbits) - 1ull;
  const uint64_t rowbits = keys[b] & ~cmask;
  uint32_t* col = scol + o;
  uint32_t *in = pa + o, *out = pb + o;
  for (int64_t i = threadIdx.x; i < len; i += kWrLongThreads) {
    col[i] = (uint32_t)(keys[b + i] & cmask);
    in[i] = (uint32_t)i;
  }
  const int64_t stretch = ((len + W - 1) / W + 31) / 32 * 32;  // positions per warp, whole rounds
  const int64_t p0 = warp * stretch, p1 = p0 + stretch < len ? p0 + stretch : len;
  for (int shift = 0; shift < cbits; shift += 8) {
    for (int i = threadIdx.x; i < W * 256; i += kWrLongThreads) cnt[i] = 0;
    __syncthreads();
    for (int64_t q = p0; q < p0 + stretch; q += 32) {
      const int64_t pos = q + lane;
      const bool valid = pos < p1;
      const unsigned act = __ballot_sync(0xffffffffu, valid);
      if (valid) {
        const unsigned d = (col[in[pos]] >> shift) & 255u;
        const unsigned peers = __match_any_sync(act, d);
        if ((peers & lt) == 0) cnt[warp * 256 + d] += (uint32_t)__popc(peers);
      }
      __syncwarp();
    }
    __syncthreads();
    if (threadIdx.x < 256) {
      const int d = threadIdx.x;
      uint32_t tot = 0;
      for (int w = 0; w < W; ++w) tot += cnt[w * 256 + d];
      uint32_t x = tot;
      for (int k = 1; k < 32; k <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, k);
        if (lane >= k) x += y;
      }
      if (lane == 31) wsum[warp] = x;
      __syncwarp();
      asm volatile("bar.sync 1, 256;");
      uint32_t before = x - tot;
      for (int w = 0; w < warp; ++w) before += wsum[w];
      for (int w = 0; w < W; ++w) {
        const uint32_t c = cnt[w * 256 + d];
        cnt[w * 256 + d] = before;
        before += c;
      }
    }
    __syncthreads();
    for (int64_t q = p0; q < p0 + stretch; q += 32) {
      const int64_t pos = q + lane;
      const bool valid = pos < p1;
      const unsigned act = __ballot_sync(0xffffffffu, valid);
      unsigned d = 0, peers = 0;
      if (valid) {
        const uint32_t e = in[pos];
        d = (col[e] >> shift) & 255u;
        peers = __match_any_sync(act, d);
        out[cnt[warp * 256 + d] + __popc(peers & lt)] = e;
      }
      __syncwarp();
      if (valid && (peers & lt) == 0) cnt[warp * 256 + d] += (uint32_t)__popc(peers);
      __syncwarp();
    }
    // every warp is done with this pass's starts (cnt) and has written all of
    // `out` before the next pass clears cnt and reads `out` as its input
    __syncthreads();
    uint32_t* t = in;
    in = out;
    out = t;
  }
  uint64_t* v = tv + o;
  for (int64_t i = threadIdx.x; i < len; i += kWrLongThreads) v[i] = vals[b + in[i]];
  __syncthreads();  // every value of the row is read before the row is overwritten
  for (int64_t i = threadIdx.x; i < len; i += kWrLongThreads) {
    keys[b + i] = rowbits | col[in[i]];
    vals[b + i] = v[i];
  }
}

static void wr_long(const int32_t* rl, int64_t nr, const int64_t* rp, uint64_t* keys, uint64_t* vals, int cbits,
                    bool hubs, cudaStream_t s) {
  DBuf<int64_t> loff(nr + 1, s);
  k_wr_long_len<<<grid_for(nr, 256, kSMs * 8), 256, 0, s>>>(rl, nr, rp, loff.get());
  LG_LAUNCH_CHECK();
  exclusive_scan(loff.get(), loff.get(), nr, s);
  std::vector<int64_t> ho((size_t)nr + 1);
  LG_CUDA(cudaMemcpyAsync(ho.data(), loff.get(), sizeof(int64_t) * (nr + 1), cudaMemcpyDeviceToHost, s));
  LG_CUDA(cudaStreamSynchronize(s));
  int64_t biggest = 0;
  for (int64_t q0 = 0, q1; q0 < nr; q0 = q1) {  // batches of whole rows, about kWrBatch entries each
    for (q1 = q0 + 1; q1 < nr && ho[q1 + 1] - ho[q0] <= kWrBatch; ++q1) {
    }
    biggest = std::max(biggest, ho[q1] - ho[q0]);
  }
  if (hubs) {  // the whole GPU on each batch: gather, a global radix sort, scatter
    DBuf<uint64_t> tk(biggest, s), tv(biggest, s);
    for (int64_t q0 = 0, q1; q0 < nr; q0 = q1) {
      for (q1 = q0 + 1; q1 < nr && ho[q1 + 1] - ho[q0] <= kWrBatch; ++q1) {
      }
      k_wr_gather<<<(unsigned)(q1 - q0), 256, 0, s>>>(rl + q0, rp, loff.get() + q0, ho[q0], keys, vals, tk.get(),
                                                       tv.get(), cbits);
      LG_LAUNCH_CHECK();
      radix_sort_pairs(tk.get(), tv.get(), ho[q1] - ho[q0], bits_for(q1 - q0) + cbits, s);
      k_wr_scatter<<<(unsigned)(q1 - q0), 256, 0, s>>>(rl + q0, rp, loff.get() + q0, ho[q0], tk.get(), tv.get(),
                                                        keys, vals, cbits);
      LG_LAUNCH_CHECK();
    }
    return;
  }
  DBuf<uint32_t> scol(biggest, s), pa(biggest, s), pb(biggest, s);
  DBuf<uint64_t> tv(biggest, s);
  for (int64_t q0 = 0, q1; q0 < nr; q0 = q1) {
    for (q1 = q0 + 1; q1 < nr && ho[q1 + 1] - ho[q0] <= kWrBatch; ++q1) {
    }
    k_wr_radix_long<<<(unsigned)(q1 - q0), kWrLongThreads, 0, s>>>(rl + q0, rp, loff.get() + q0, ho[q0], keys, vals,
                                                                   scol.get(), pa.get(), pb.get(), tv.get(), cbits);
    LG_LAUNCH_CHECK();
  }
}

void sort_within_rows(DBuf<uint64_t>& keys, DBuf<uint64_t>& vals, int64_t nent, const int64_t* rp, int64_t ngroups,
                      int cbits, cudaStream_t s) {
  if (nent <= 1 || ngroups <= 0) return;
  DBuf<int64_t> cnt(kWrClasses, s);
  DBuf<unsigned long long> fill(kWrClasses, s);
  DBuf<int32_t> rows(ngroups, s);
  LG_CUDA(cudaMemsetAsync(cnt.get(), 0, sizeof(int64_t) * kWrClasses, s));
  LG_CUDA(cudaMemsetAsync(fill.get(), 0, sizeof(unsigned long long) * kWrClasses, s));
  const int gb = grid_for(ngroups, 256, kSMs * 8);
  k_wr_bin<<<gb, 256, 0, s>>>(ngroups, rp, 0, cnt.get(), nullptr, nullptr, nullptr);
  LG_LAUNCH_CHECK();
  int64_t hc[kWrClasses], ho[kWrClasses + 1];
  LG_CUDA(cudaMemcpyAsync(hc, cnt.get(), sizeof(hc), cudaMemcpyDeviceToHost, s));
  LG_CUDA(cudaStreamSynchronize(s));
  ho[0] = 0;
  for (int c = 0; c < kWrClasses; ++c) ho[c + 1] = ho[c] + hc[c];
  LG_CUDA(cudaMemcpyAsync(cnt.get(), ho, sizeof(int64_t) * kWrClasses, cudaMemcpyHostToDevice, s));
  k_wr_bin<<<gb, 256, 0, s>>>(ngroups, rp, 1, nullptr, cnt.get(), fill.get(), rows.get());
  LG_LAUNCH_CHECK();
  uint64_t *k = keys.get(), *v = vals.get();
  const uint64_t cmask = (1ull << cbits) - 1ull;
  for (int c = 1; c < kWrClasses; ++c) {  // class 0 (at most one entry) is sorted already
    const int64_t nr = hc[c];
    if (!nr) continue;
    const int32_t* rl = rows.get() + ho[c];
    const auto lanes = [&](int G) { return grid_for(nr * G, 256, 1 << 30); };
    switch (c) {
      case 1: k_wr_rank<2><<<lanes(2), 256, 0, s>>>(rl, nr, rp, k, v); break;
      case 2: k_wr_rank<4><<<lanes(4), 256, 0, s>>>(rl, nr, rp, k, v); break;
      case 3: k_wr_rank<8><<<lanes(8), 256, 0, s>>>(rl, nr, rp, k, v); break;
      case 4: k_wr_rank<16><<<lanes(16), 256, 0, s>>>(rl, nr, rp, k, v); break;
      case 5: k_wr_rank<32><<<lanes(32), 256, 0, s>>>(rl, nr, rp, k, v); break;
      case 6: wr_block_launch<64>(rl, nr, rp, k, v, cmask, s); break;
      case 7: wr_block_launch<128>(rl, nr, rp, k, v, cmask, s); break;
      case 8: wr_block_launch<256>(rl, nr, rp, k, v, cmask, s); break;
      case 9: wr_block_launch<512>(rl, nr, rp, k, v, cmask, s); break;
      case 10: wr_radix_launch<1024>(rl, nr, rp, k, v, cbits, s); break;
      case 11: wr_radix_launch<2048>(rl, nr, rp, k, v, cbits, s); break;
      case 12: wr_radix_launch<4096>(rl, nr, rp, k, v, cbits, s); break;
      case 13: wr_radix_launch<8192>(rl, nr, rp, k, v, cbits, s); break;
      case 14: wr_radix_launch<16384>(rl, nr, rp, k, v, cbits, s); break;
      case 15: wr_long(rl, nr, rp, k, v, cbits, false, s); break;
      default: wr_long(rl, nr, rp, k, v, cbits, true, s); break;
    }
    LG_LAUNCH_CHECK();
  }
}

void accumulate_csr(DBuf<uint64_t>& keys, DBuf<uint64_t>& vals, int64_t nent, int64_t nrows, int cbits,
                    CsrOut& out, cudaStream_t s, int64_t* counter, const int64_t* grouped, int64_t ngroups) {
  if (grouped)
    sort_within_rows(keys, vals, nent, grouped, ngroups, cbits, s);
  else
    radix_sort_pairs(keys.get(), vals.get(), nent, bits_for(nrows) + cbits, s);
  int64_t nseg = 0;
  DBuf<uint8_t> head(nent, s);
  DBuf<int64_t> segid(nent + 1, s);
  const int g = grid_for(nent, 256, kSMs * 16);
  if (nent > 0) {
    k_seg_heads<<<g, 256, 0, s>>>(keys.get(), nent, head.get());
    LG_LAUNCH_CHECK();
  }
  exclusive_scan_flags(head.get(), segid.get(), nent, s);
  LG_CUDA(cudaMemcpyAsync(&nseg, segid.get() + nent, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  LG_CUDA(cudaStreamSynchronize(s));
  DBuf<int64_t> start(nseg, s);
  DBuf<uint64_t> segkey(nseg, s);
  out.col.alloc(nseg, s, counter);
  out.w.alloc(nseg, s, counter);
  out.rowptr.alloc(nrows + 1, s, counter);
  out.nnz = nseg;
  if (nent > 0) {
    k_seg_starts<<<g, 256, 0, s>>>(head.get(), segid.get(), nent, start.get());
    LG_LAUNCH_CHECK();
    k_seg_sum<<<grid_for(nseg, 256, kSMs * 16), 256, 0, s>>>(keys.get(), vals.get(), start.get(), nseg, nent,
                                                            (1ull << cbits) - 1ull, out.col.get(), out.w.get(),
                                                            segkey.get());
    LG_LAUNCH_CHECK();
  }
  k_rowptr_from_keys<<<grid_for(nrows + 1, 256, kSMs * 16), 256, 0, s>>>(segkey.get(), nseg, cbits, nrows,
                                                                        out.rowptr.get());
  LG_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// Row plan.
// ---------------------------------------------------------------------------
__global__ void k_plan_count(int64_t n, const int64_t* __restrict__ rowptr, int64_t* __restrict__ nch,
                             uint8_t* __restrict__ islong) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t deg = rowptr[i + 1] - rowptr[i];
    const bool l = deg > kChunk;
    islong[i] = l;
    nch[i] = l ? (deg + kChunk - 1) / kChunk : 0;
  }
}

__global__ void k_plan_fill(int64_t n, const int64_t* __restrict__ rowptr, const uint8_t* __restrict__ islong,
                            const int64_t* __restrict__ cstart, const int64_t* __restrict__ lidx, int32_t* chunk_row,
                            int64_t* chunk_beg, int32_t* chunk_lrow, int32_t* lrow_first, int32_t* lrow_count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (!islong[i]) continue;
    const int64_t lr = lidx[i], c0 = cstart[i], cnt = cstart[i + 1] - cstart[i];
    lrow_first[lr] = (int32_t)c0;
    lrow_count[lr] = (int32_t)cnt;
    for (int64_t q = 0; q < cnt; ++q) {
      chunk_row[c0 + q] = (int32_t)i;
      chunk_beg[c0 + q] = rowptr[i] + q * kChunk;
      chunk_lrow[c0 + q] = (int32_t)lr;
    }
  }
}

// Class of each row: the smallest c with deg <= E 2^c (capped at the last
// class); kClasses for rows cut into chunks.
__global__ void k_plan_class(int64_t n, const int64_t* __restrict__ rowptr, int E, uint64_t* __restrict__ key,
                             uint64_t* __restrict__ val) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t deg = rowptr[i + 1] - rowptr[i];
    int c = 0;
    while (c < kClasses - 1 && deg > (int64_t)E << c) ++c;
    key[i] = deg > kChunk ? (uint64_t)kClasses : (uint64_t)c;
    val[i] = (uint64_t)i;
  }
}

__global__ void k_plan_lists(int64_t n, const uint64_t* __restrict__ key, const uint64_t* __restrict__ val,
                             int32_t* __restrict__ rows, int64_t* __restrict__ off) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    rows[i] = (int32_t)val[i];
    if (i == 0 || key[i] != key[i - 1])
      for (uint64_t c = (i == 0 ? 0 : key[i - 1] + 1); c <= key[i]; ++c) off[c] = i;
    if (i == n - 1)
      for (uint64_t c = key[i] + 1; c <= (uint64_t)kClasses; ++c) off[c] = n;
  }
}

void bin_rows(RowPlanStore& ps, int64_t n, const int64_t* rowptr, int E, cudaStream_t s) {
  RowPlan& p = ps.plan;
  p.E = E;
  int64_t off[kClasses + 1] = {0};
  if (n > 0) {
    DBuf<uint64_t> key(n, s), val(n, s);
    DBuf<int64_t> doff(kClasses + 1, s);
    const int g = grid_for(n, 256, kSMs * 16);
    k_plan_class<<<g, 256, 0, s>>>(n, rowptr, E, key.get(), val.get());
    LG_LAUNCH_CHECK();
    radix_sort_pairs(key.get(), val.get(), n, 8, s);
    k_plan_lists<<<g, 256, 0, s>>>(n, key.get(), val.get(), ps.rows_by_class.get(), doff.get());
    LG_LAUNCH_CHECK();
    LG_CUDA(cudaMemcpyAsync(off, doff.get(), sizeof(off), cudaMemcpyDeviceToHost, s));
    LG_CUDA(cudaStreamSynchronize(s));
  }
  int blk = 0;
  for (int c = 0; c < kClasses; ++c) {
    p.cls_off[c] = off[c];
    p.blk_off[c] = blk;
    const int64_t rows = off[c + 1] - off[c];
    const int64_t per_block = class_rows_per_block(c);
    blk += (int)((rows + per_block - 1) / per_block);
  }
  p.cls_off[kClasses] = off[kClasses];
  p.blk_off[kClasses] = blk;
  p.rows_by_class = ps.rows_by_class.get();
}

RowBins bins_of(const RowPlan& p, int64_t n) {
  RowBins b;
  b.rows = p.rows_by_class;
  for (int c = 0; c <= kClasses; ++c) b.off[c] = p.cls_off[c];
  b.off[kClasses + 1] = n;
  int blk = (int)(n - p.cls_off[kClasses]);  // one block per long row
  for (int c = kClasses - 1; c >= 0; --c) {
    b.blk[c] = blk;
    const int64_t per = kEachThreads >> c;
    blk += (int)((b.off[c + 1] - b.off[c] + per - 1) / per);
  }
  b.grid = blk;
  return b;
}

void make_bins(RowBinsStore& b, int64_t n, const int64_t* rowptr, cudaStream_t s) {
  int64_t off[kClasses + 1] = {0};
  b.rows.alloc(n, s);
  if (n > 0) {
    DBuf<uint64_t> key(n, s), val(n, s);
    DBuf<int64_t> doff(kClasses + 1, s);
    const int g = grid_for(n, 256, kSMs * 16);
    k_plan_class<<<g, 256, 0, s>>>(n, rowptr, 4, key.get(), val.get());
    LG_LAUNCH_CHECK();
    radix_sort_pairs(key.get(), val.get(), n, 8, s);
    k_plan_lists<<<g, 256, 0, s>>>(n, key.get(), val.get(), b.rows.get(), doff.get());
    LG_LAUNCH_CHECK();
    LG_CUDA(cudaMemcpyAsync(off, doff.get(), sizeof(off), cudaMemcpyDeviceToHost, s));
    LG_CUDA(cudaStreamSynchronize(s));
  }
  RowPlan p;
  p.rows_by_class = b.rows.get();
  for (int c = 0; c <= kClasses; ++c) p.cls_off[c] = off[c];
  b.bins = bins_of(p, n);
}

__global__ void k_long_rows(int64_t nlong, const int32_t* __restrict__ rows, const int64_t* __restrict__ rowptr,
                            int64_t* __restrict__ span) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nlong; q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = rows[q];
    span[2 * q] = rowptr[r];
    span[2 * q + 1] = rowptr[r + 1];
  }
}

// Tiles of the column-segmented long-row pass (RowPlan::nseg_tiles), or
// none. Staging the whole vector costs ncols * sizeof(T) per tile against
// the tile's entries * (4 + sizeof(T)) bytes streamed, so a tile takes at
// least 7 ncols entries (staging under a tenth of the stream) and at most
// the long entries over 4 tiles per SM; with fewer than 2 tiles per SM, or
// long rows under a quarter of the entries, the long rows stay chunked.
// Long rows are cut into virtual rows of at most max(kChunk, TE / 128)
// entries (equal parts); a row's virtual rows share a tile, and a tile
// holds at most kSegMaxVrows of them and about TE entries.
static void plan_segments(RowPlanStore& ps, int64_t n, int64_t nnz, const int64_t* rowptr, int64_t ncols,
                          cudaStream_t s, int64_t* counter) {
  RowPlan& p = ps.plan;
  p.nseg_tiles = 0;
  p.ncols = ncols;
  const int64_t nlong = n - p.cls_off[kClasses];
  if (ncols <= 0 || nlong <= 0) return;
  std::vector<int64_t> span((size_t)(2 * nlong));
  {
    DBuf<int64_t> dspan((size_t)(2 * nlong), s);
    k_long_rows<<<grid_for(nlong, 256, kSMs * 8), 256, 0, s>>>(nlong, ps.rows_by_class.get() + p.cls_off[kClasses],
                                                               rowptr, dspan.get());
    LG_LAUNCH_CHECK();
    LG_CUDA(cudaMemcpyAsync(span.data(), dspan.get(), sizeof(int64_t) * 2 * nlong, cudaMemcpyDeviceToHost, s));
    LG_CUDA(cudaStreamSynchronize(s));
  }
  int64_t long_entries = 0;
  for (int64_t q = 0; q < nlong; ++q) long_entries += span[2 * q + 1] - span[2 * q];
  const int64_t te_min = 7 * ncols;
  const int64_t te = std::max<int64_t>(te_min, long_entries / (4 * kSMs));
  if (4 * long_entries < nnz || long_entries < 2 * kSMs * te_min) return;
  const int64_t vr = std::max<int64_t>(kChunk, te / 128);
  std::vector<int32_t> row_of, tile_off(1, 0);
  std::vector<int64_t> beg, end;
  std::vector<int32_t> rows(nlong);
  LG_CUDA(cudaMemcpyAsync(rows.data(), ps.rows_by_class.get() + p.cls_off[kClasses], sizeof(int32_t) * nlong,
                          cudaMemcpyDeviceToHost, s));
  LG_CUDA(cudaStreamSynchronize(s));
  int64_t tile_entries = 0;
  int tile_vrows = 0;
  for (int64_t q = 0; q < nlong; ++q) {
    const int64_t b = span[2 * q], e = span[2 * q + 1], deg = e - b;
    int64_t parts = (deg + vr - 1) / vr;
    if (parts > kSegMaxVrows) parts = kSegMaxVrows;  // a row never spans two tiles
    if (tile_vrows > 0 && (tile_vrows + parts > kSegMaxVrows || tile_entries + deg > te)) {
      tile_off.push_back((int32_t)row_of.size());
      tile_vrows = 0;
      tile_entries = 0;
    }
    for (int64_t k = 0; k < parts; ++k) {
      row_of.push_back(rows[q]);
      beg.push_back(b + deg * k / parts);
      end.push_back(b + deg * (k + 1) / parts);
    }
    tile_vrows += (int)parts;
    tile_entries += deg;
  }
  tile_off.push_back((int32_t)row_of.size());
  const size_t nv = row_of.size(), nt = tile_off.size() - 1;
  ps.seg_tile_off.alloc(nt + 1, s, counter);
  ps.vrow_row.alloc(nv, s, counter);
  ps.vrow_beg.alloc(nv, s, counter);
  ps.vrow_end.alloc(nv, s, counter);
  LG_CUDA(cudaMemcpyAsync(ps.seg_tile_off.get(), tile_off.data(), sizeof(int32_t) * (nt + 1), cudaMemcpyHostToDevice, s));
  LG_CUDA(cudaMemcpyAsync(ps.vrow_row.get(), row_of.data(), sizeof(int32_t) * nv, cudaMemcpyHostToDevice, s));
  LG_CUDA(cudaMemcpyAsync(ps.vrow_beg.get(), beg.data(), sizeof(int64_t) * nv, cudaMemcpyHostToDevice, s));
  LG_CUDA(cudaMemcpyAsync(ps.vrow_end.get(), end.data(), sizeof(int64_t) * nv, cudaMemcpyHostToDevice, s));
  LG_CUDA(cudaStreamSynchronize(s));  // the host vectors go out of scope
  p.nseg_tiles = (int)nt;
  p.seg_tile_off = ps.seg_tile_off.get();
  p.vrow_row = ps.vrow_row.get();
  p.vrow_beg = ps.vrow_beg.get();
  p.vrow_end = ps.vrow_end.get();
}

void build_row_plan(RowPlanStore& ps, int64_t n, int64_t nnz, const int64_t* rowptr, cudaStream_t s,
                    int64_t* counter, int64_t ncols) {
  RowPlan& p = ps.plan;
  DBuf<int64_t> nch(n + 1, s), lidx(n + 1, s);
  DBuf<uint8_t> islong(n, s);
  const int g = grid_for(n, 256, kSMs * 16);
  if (n > 0) {
    k_plan_count<<<g, 256, 0, s>>>(n, rowptr, nch.get(), islong.get());
    LG_LAUNCH_CHECK();
  }
  exclusive_scan(nch.get(), nch.get(), n, s);
  exclusive_scan_flags(islong.get(), lidx.get(), n, s);
  int64_t tot[2];
  LG_CUDA(cudaMemcpyAsync(&tot[0], nch.get() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  LG_CUDA(cudaMemcpyAsync(&tot[1], lidx.get() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  LG_CUDA(cudaStreamSynchronize(s));
  p.nchunks = tot[0];
  p.nlong = tot[1];
  ps.rows_by_class.alloc(n, s, counter);
  ps.chunk_row.alloc(p.nchunks, s, counter);
  ps.chunk_beg.alloc(p.nchunks, s, counter);
  ps.chunk_lrow.alloc(p.nchunks, s, counter);
  ps.lrow_first.alloc(p.nlong, s, counter);
  ps.lrow_count.alloc(p.nlong, s, counter);
  ps.partial.alloc((size_t)(p.nchunks > 0 ? p.nchunks : 1) * kMaxCols, s, counter);
  ps.ticket.alloc(p.nlong > 0 ? p.nlong : 1, s, counter);
  LG_CUDA(cudaMemsetAsync(ps.ticket.get(), 0, sizeof(unsigned) * (p.nlong > 0 ? p.nlong : 1), s));
  if (p.nlong > 0) {
    k_plan_fill<<<g, 256, 0, s>>>(n, rowptr, islong.get(), nch.get(), lidx.get(), ps.chunk_row.get(),
                                  ps.chunk_beg.get(), ps.chunk_lrow.get(), ps.lrow_first.get(), ps.lrow_count.get());
    LG_LAUNCH_CHECK();
  }
  p.chunk_row = ps.chunk_row.get();
  p.chunk_beg = ps.chunk_beg.get();
  p.chunk_lrow = ps.chunk_lrow.get();
  p.lrow_first = ps.lrow_first.get();
  p.lrow_count = ps.lrow_count.get();
  p.partial = ps.partial.get();
  p.ticket = ps.ticket.get();
  bin_rows(ps, n, rowptr, 4, s);
  plan_segments(ps, n, nnz, rowptr, ncols, s, counter);
}

}  // namespace lg
