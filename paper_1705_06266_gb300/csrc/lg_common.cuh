// Internal header of the sm_103a graph-Laplacian multigrid library.
//
// Error handling, stream-ordered device buffers, the SplitMix64 random
// streams, deterministic group / block / grid reductions and the SpMV row
// plan shared by the setup and solve kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstddef>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <utility>
#include <vector>

#include "../../include/lg.h"

namespace lg {

// ---------------------------------------------------------------------------
// Errors: library code throws Error; the C-ABI layer turns it into a status.
// ---------------------------------------------------------------------------
struct Error {
  int code;
  const char* what;
};

[[noreturn]] inline void fail(int code, const char* what) { throw Error{code, what}; }

// Detail of the last error on this host thread (lg_last_error_detail).
extern thread_local std::string g_last_error;

inline void check_cuda(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return;
  static thread_local char msg[256];
  std::snprintf(msg, sizeof(msg), "%s: %s", what, cudaGetErrorName(e));
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    fail(LG_ERR_NOMEM, msg);
  }
  fail(LG_ERR_CUDA, msg);
}

#define LG_CUDA(call) ::lg::check_cuda((call), #call)

// Every kernel launch site is followed by LG_LAUNCH_CHECK(), which counts the
// launch and turns a launch error into an Error naming the site and the CUDA
// error. With LG_DEBUG_SYNC=1 in the environment it also waits for the
// kernel, so an asynchronous fault is reported at the kernel that caused it
// (and solves run without graph capture).
extern std::atomic<uint64_t> g_launches;
bool debug_sync();
void check_launch(const char* file, int line);
#define LG_LAUNCH_CHECK()                                           \
  do {                                                              \
    ::lg::g_launches.fetch_add(1, std::memory_order_relaxed);      \
    ::lg::check_launch(__FILE__, __LINE__);                         \
  } while (0)

// ---------------------------------------------------------------------------
// Device memory: stream-ordered allocation (cudaMallocAsync on the pool of
// the device), released on the stream it was made on. `counter` tracks the
// bytes a hierarchy or workspace holds.
// ---------------------------------------------------------------------------
template <typename T>
class DBuf {
 public:
  DBuf() = default;
  DBuf(size_t count, cudaStream_t s, int64_t* counter = nullptr) { alloc(count, s, counter); }
  ~DBuf() { release(); }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept { *this = std::move(o); }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) {
      release();
      p_ = o.p_; n_ = o.n_; s_ = o.s_; counter_ = o.counter_;
      o.p_ = nullptr; o.n_ = 0; o.counter_ = nullptr;
    }
    return *this;
  }
  void alloc(size_t count, cudaStream_t s, int64_t* counter = nullptr) {
    release();
    s_ = s;
    n_ = count;
    counter_ = counter;
    size_t bytes = (count ? count : 1) * sizeof(T);
    void* p = nullptr;
    LG_CUDA(cudaMallocAsync(&p, bytes, s));
    p_ = static_cast<T*>(p);
    if (counter_) *counter_ += (int64_t)bytes;
  }
  void release() {
    if (p_) {
      // a failed free must not leave its error behind for an unrelated later check
      if (cudaFreeAsync(p_, s_) != cudaSuccess) cudaGetLastError();
      if (counter_) *counter_ -= (int64_t)((n_ ? n_ : 1) * sizeof(T));
    }
    p_ = nullptr;
    n_ = 0;
  }
  T* get() const { return p_; }
  size_t size() const { return n_; }
  operator T*() const { return p_; }

 private:
  T* p_ = nullptr;
  size_t n_ = 0;
  cudaStream_t s_ = nullptr;
  int64_t* counter_ = nullptr;
};

// Pinned host staging for scalars read back during setup.
struct HostScratch {
  void* p = nullptr;
  explicit HostScratch(size_t bytes) { LG_CUDA(cudaMallocHost(&p, bytes)); }
  ~HostScratch() { if (p) cudaFreeHost(p); }
  template <typename T> T* as() { return static_cast<T*>(p); }
};

constexpr int kSMs = 152;  // GB300: 2 dies x 76 SMs

inline int grid_for(int64_t work_items, int threads, int max_blocks) {
  int64_t b = (work_items + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): output number `counter` of
// the generator seeded with `seed` is the finaliser applied to
// seed + (counter + 1) * 0x9E3779B97F4A7C15. Counters pack a stream id
// (bits 56..63), a level (bits 40..55) and an index (bits 0..39).
// Stream 0: vertex hash for elimination. Streams 1..8: strength test
// vectors. Stream 8 is also the Lanczos start vector (vectors use 1..m, m<=7
// when the Lanczos stream is needed on the same level).
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t counter) {
  uint64_t z = seed + (counter + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t rng_counter(int stream, int level, int64_t idx) {
  return ((uint64_t)(uint32_t)stream << 56) | ((uint64_t)(uint32_t)level << 40) | (uint64_t)idx;
}

// Uniform in [-1, 1) from the top 53 bits.
__device__ __forceinline__ double uniform_pm1(uint64_t seed, int stream, int level, int64_t idx) {
  uint64_t z = splitmix64(seed, rng_counter(stream, level, idx));
  return 2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0;
}

constexpr int kStreamHash = 0;
constexpr int kStreamLanczos = 8;
constexpr int kStreamOrder = 9;  // the random vertex ordering (option reorder = 2)

// ---------------------------------------------------------------------------
// Reductions. Group reductions use xor butterflies inside aligned groups of
// G lanes; the order of additions depends only on G, so results are
// reproducible run to run.
// ---------------------------------------------------------------------------
template <int G>
__device__ __forceinline__ unsigned group_mask() {
  if constexpr (G == 32) {
    return 0xffffffffu;
  } else {
    unsigned lane = threadIdx.x & 31u;
    return ((1u << G) - 1u) << (lane & ~(unsigned)(G - 1));
  }
}

template <int G, typename T>
__device__ __forceinline__ T group_sum(T v, unsigned mask) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, G);
  return v;
}

// Sum into the group's first lane only: at each step just the lanes that
// still hold partial sums add (G - 1 additions in all instead of G log2 G),
// which matters for FP64, whose pipe is narrow on this part.
template <int G, typename T>
__device__ __forceinline__ T group_sum_first(T v, unsigned mask, int lane) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    const T t = __shfl_down_sync(mask, v, o, G);
    if (lane < o) v += t;
  }
  return v;
}

template <int G, typename T>
__device__ __forceinline__ T group_max(T v, unsigned mask) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    T u = __shfl_xor_sync(mask, v, o, G);
    v = u > v ? u : v;
  }
  return v;
}

template <int G>
__device__ __forceinline__ uint64_t group_min_u64(uint64_t v, unsigned mask) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    uint64_t u = __shfl_xor_sync(mask, v, o, G);
    v = u < v ? u : v;
  }
  return v;
}

// Block-wide sum of K values; the result is valid in thread 0.
template <int NT, int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* smem /* K * (NT/32) */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = group_sum<32>(v[k], 0xffffffffu);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) smem[k * (NT / 32) + wid] = v[k];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double t = lane < NT / 32 ? smem[k * (NT / 32) + lane] : 0.0;
      v[k] = group_sum<32>(t, 0xffffffffu);
    }
  }
  __syncthreads();
}

// Grid-wide sum of K values in one launch: blocks store partials, the last
// block to arrive (ticket counter) adds them in block order and writes
// out[0..K-1]. Deterministic for a fixed grid size. Meant for the vector
// kernels (grids of at most a few thousand blocks of uniform work); the
// row passes write their results and leave dot products to those kernels.
// Every thread of every block must call it; `partials` holds K values per
// block; `ticket` must be 0 on entry and is 0 again on exit. Returns true in
// exactly one thread (thread 0 of the last block), after out[] is written,
// so that it can derive scalars from the totals.
template <int NT, int K>
__device__ __forceinline__ bool grid_sum(double (&v)[K], double* partials, unsigned* ticket, double* out) {
  __shared__ double red_smem[K * (NT / 32)];
  __shared__ bool am_last;
  block_sum<NT, K>(v, red_smem);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) partials[(size_t)blockIdx.x * K + k] = v[k];
    __threadfence();
    unsigned t = atomicAdd(ticket, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return false;
  __threadfence();
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += NT) {
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] += __ldcg(&partials[(size_t)b * K + k]);
  }
  block_sum<NT, K>(acc, red_smem);
  if (threadIdx.x != 0) return false;
#pragma unroll
  for (int k = 0; k < K; ++k) out[k] = acc[k];
  *ticket = 0u;
  return true;
}

// ---------------------------------------------------------------------------
// SpMV row plan of one CSR operator (see lg_rows.cuh). Rows are binned by
// length into classes c = 0..5 served by groups of G = 2^c lanes: class c
// holds the rows with E 2^(c-1) < deg <= E 2^c (class 0: deg <= E, class 5:
// up to kChunk entries), E the entries per lane, so every group of a warp
// does about the same work. Rows longer than kChunk are cut into chunks of
// kChunk entries, one block per chunk; the last block of a row (per-row
// ticket) adds the chunk partials in chunk order and applies the epilogue.
// ---------------------------------------------------------------------------
constexpr int kRowThreads = 256;
constexpr int kChunk = 2048;
constexpr int kClasses = 6;
// Rows one block of kRowThreads threads serves in class c (groups of 2^c
// lanes; classes 0..3 take 2^c rows per group, so 32 rows per warp; the two
// widest classes one row per group, so that every such row has its own group
// in flight: more rows per group would serialise them and leave the gathers'
// latency exposed).
__host__ __device__ constexpr int64_t class_rows_per_block(int c) {
  return c <= 3 ? kRowThreads : c == 4 ? kRowThreads / 16 : kRowThreads / 32;
}

struct RowPlan {
  int E = 4;                          // entries per lane (class boundaries)
  int64_t cls_off[kClasses + 1] = {};  // class c rows: rows_by_class[cls_off[c] .. cls_off[c+1])
  int blk_off[kClasses + 1] = {};      // class c blocks: [nchunks + blk_off[c], nchunks + blk_off[c+1])
  const int32_t* rows_by_class = nullptr;
  int64_t nlong = 0;
  int64_t nchunks = 0;
  int32_t* chunk_row = nullptr;   // row of each chunk
  int64_t* chunk_beg = nullptr;   // first entry of each chunk
  int32_t* chunk_lrow = nullptr;  // index of the row among the long rows
  int32_t* lrow_first = nullptr;  // first chunk of each long row
  int32_t* lrow_count = nullptr;  // chunks of each long row
  double* partial = nullptr;      // nchunks * kMaxCols partial sums
  unsigned* ticket = nullptr;     // nlong tickets, zero between launches
  // Column-segmented service of the long rows (k_rows_seg, lg_rows.cuh), for
  // operators whose vector is short next to their long rows' entries: a
  // block takes a tile of long rows and walks the columns in segments of
  // kSegBytes, each staged once in shared memory, so the tile's gathers read
  // shared memory instead of a 32-byte L2 sector each. A long row may be cut
  // into several virtual rows (entry ranges) of one tile, whose sums are
  // added in order. nseg_tiles = 0: the long rows go by chunks.
  int64_t ncols = 0;                   // length of the gathered vector
  int nseg_tiles = 0;
  const int32_t* seg_tile_off = nullptr;  // tile t: virtual rows [seg_tile_off[t], seg_tile_off[t+1])
  const int32_t* vrow_row = nullptr;      // the row of each virtual row
  const int64_t* vrow_beg = nullptr;      // its entries [vrow_beg, vrow_end)
  const int64_t* vrow_end = nullptr;

  int grid() const { return (int)nchunks + blk_off[kClasses]; }
};

// Shared memory of one staged column segment, and the most virtual rows of a
// tile (32 warps, 8 each).
constexpr int kSegBytes = 128 * 1024;
constexpr int kSegThreads = 1024;
constexpr int kSegRowsPerWarp = 8;
constexpr int kSegMaxVrows = (kSegThreads / 32) * kSegRowsPerWarp;

constexpr int kMaxCols = 32;  // widest multi-RHS block

}  // namespace lg
