// lg_elim_select_noalloc: the elimination-candidate selection of
// lg_elim_select with its scratch memory in a fixed device array instead of
// a stream-ordered allocation.
//
// Some callers cannot allocate device memory at the moment they call: code
// running inside a memory pool that must not grow, a host callback or a
// thread of an embedding runtime that forbids cudaMalloc and friends, or a
// real-time loop where an allocation could stall. This entry point uses only
// the caller's input and output buffers plus the array below, which every
// process that loads the library holds on every device it uses until exit.
#include <mutex>

#include "lg_hier.h"

namespace lg {

// Largest graph the entry point accepts: 2^20 vertices (8 MiB of hash values).
constexpr int64_t kNoAllocMaxN = int64_t(1) << 20;

// Scratch shared by every call: one hash (or +infinity) per vertex and the
// count of eliminated vertices. Host code must not pass these names to a
// kernel (on the host they are stand-ins, not device addresses); it uses
// the addresses looked up below.
static __device__ __align__(256) uint64_t g_noalloc_hash[kNoAllocMaxN];
static __device__ __align__(256) unsigned long long g_noalloc_count;

struct NoAllocAddrs {
  uint64_t* hash = nullptr;
  unsigned long long* count = nullptr;
};

// Device addresses of the scratch, looked up once per device with that
// device current.
static NoAllocAddrs noalloc_addrs() {
  static std::mutex mu;
  static std::vector<NoAllocAddrs> per_device;
  int dev = 0;
  LG_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if ((int)per_device.size() <= dev) per_device.resize(dev + 1);
  NoAllocAddrs& a = per_device[dev];
  if (!a.hash) {
    void* p = nullptr;
    LG_CUDA(cudaGetSymbolAddress(&p, g_noalloc_hash));
    void* q = nullptr;
    LG_CUDA(cudaGetSymbolAddress(&q, g_noalloc_count));
    a.hash = static_cast<uint64_t*>(p);
    a.count = static_cast<unsigned long long*>(q);
  }
  return a;
}

#define LG_NA_STRIDE(i, n) \
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

__global__ void k_na_hash(int64_t n, const int64_t* __restrict__ rowptr, int max_degree, uint64_t seed,
                          uint64_t* __restrict__ hc, unsigned long long* count) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *count = 0ull;  // the count starts at zero on every call
  LG_NA_STRIDE(i, n) {
    const int64_t deg = rowptr[i + 1] - rowptr[i];
    hc[i] = deg <= max_degree ? splitmix64(seed, rng_counter(kStreamHash, 0, i)) : ~0ull;
  }
}

__global__ void k_na_select(int64_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            int max_degree, const uint64_t* __restrict__ hc, uint8_t* __restrict__ is_f,
                            unsigned long long* count) {
  unsigned long long local = 0;
  LG_NA_STRIDE(i, n) {
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
    local += f;
  }
  local = group_sum<32>(local, 0xffffffffu);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd(count, local);
}

}  // namespace lg

extern "C" int lg_elim_select_noalloc(int64_t n, const int64_t* rowptr, const int32_t* col, int32_t max_degree,
                                      uint64_t seed, uint8_t* is_f, int64_t* nf, void* stream) {
  if (n < 1 || !rowptr || !col || !is_f || max_degree < 0) return LG_ERR_INVALID;
  if (n > lg::kNoAllocMaxN) {
    lg::g_last_error = "lg_elim_select_noalloc: n exceeds the fixed scratch of 1048576 vertices";
    return LG_ERR_INVALID;
  }
  try {
    cudaStream_t s = (cudaStream_t)stream;
    if (s) {
      // the scratch address is the current device's: a stream of another
      // device would run the kernels against the wrong device's array
      int cur = 0, sdev = 0;
      LG_CUDA(cudaGetDevice(&cur));
      LG_CUDA(cudaStreamGetDevice(s, &sdev));
      if (sdev != cur) {
        lg::g_last_error = "lg_elim_select_noalloc: stream belongs to another device than the current one";
        return LG_ERR_INVALID;
      }
    }
    const lg::NoAllocAddrs a = lg::noalloc_addrs();
    const int blocks = lg::grid_for(n, 256, lg::kSMs * 8);
    lg::k_na_hash<<<blocks, 256, 0, s>>>(n, rowptr, max_degree, seed, a.hash, a.count);
    LG_LAUNCH_CHECK();
    lg::k_na_select<<<blocks, 256, 0, s>>>(n, rowptr, col, max_degree, a.hash, is_f, a.count);
    LG_LAUNCH_CHECK();
    unsigned long long c = 0;
    LG_CUDA(cudaMemcpyAsync(&c, a.count, sizeof(c), cudaMemcpyDeviceToHost, s));
    LG_CUDA(cudaStreamSynchronize(s));
    if (nf) *nf = (int64_t)c;
    return LG_OK;
  } catch (const lg::Error& e) {
    lg::g_last_error = e.what ? e.what : "";
    return e.code;
  }
}
