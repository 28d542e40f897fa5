// sem_dot_static: a dot product that needs no context and allocates no memory.
//
// Some callers cannot allocate device memory: a host framework that owns a
// fixed device-memory budget and hands the library only pointers into it, code
// that must not pay for cudaMalloc's device-wide synchronisation in a latency-
// critical loop, or a caller that has no libsem context at all. For them this
// entry point keeps its scratch (one partial sum per block plus a completion
// counter) in a file-scope static device array instead of memory from
// cudaMalloc. The array exists once per device that loads the library and
// stays allocated until the process exits.
//
// The kernel is a variant of the deterministic last-block reduction used for
// the Krylov dot products: block q sums the elements of tile q in a fixed
// order, the last block to finish adds the block partials in index order.
#include <mutex>

#include "sem_internal.cuh"

namespace {

constexpr int DS_THREADS = 256;
constexpr int64_t DS_TILE = 8192;          // elements per block
constexpr int DS_MAX_BLOCKS = 8192;        // block partials the static scratch holds
constexpr int64_t DS_MAX_N = DS_TILE * DS_MAX_BLOCKS;   // 67,108,864 elements

struct DotScratch {
  double part[DS_MAX_BLOCKS];
  unsigned int ticket;
};

// 64 KiB + 4 bytes per device; host code only ever sees its device address
// through cudaGetSymbolAddress (the name itself is a host-side stand-in).
static __device__ __align__(256) DotScratch g_dot_scratch;

std::mutex g_addr_mutex;
DotScratch* g_addr[sem::MAX_DEVICES] = {};

__global__ void __launch_bounds__(DS_THREADS)
    k_dot_static(int64_t n, const double* __restrict__ a, const double* __restrict__ b,
                 const uint8_t* __restrict__ mask, DotScratch* S, double* out) {
  __shared__ double s_w[DS_THREADS / 32];
  __shared__ bool s_last;
  const int64_t lo = (int64_t)blockIdx.x * DS_TILE;
  const int64_t hi = min(n, lo + DS_TILE);
  double acc = 0.0;
  for (int64_t l = lo + threadIdx.x; l < hi; l += DS_THREADS)
    if (!mask || mask[l]) acc = fma(a[l], b[l], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s_w[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < DS_THREADS / 32; ++w) t += s_w[w];
    S->part[blockIdx.x] = t;
    __threadfence();
    s_last = (atomicAdd(&S->ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double t = 0.0;
  for (unsigned q = threadIdx.x; q < gridDim.x; q += DS_THREADS) t += __ldcg(&S->part[q]);
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  __syncthreads();
  if (lane == 0) s_w[warp] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < DS_THREADS / 32; ++w) tot += s_w[w];
    *out = tot;
    S->ticket = 0u;
  }
}

// Device address of the static scratch on the current device, looked up once
// per device (with that device current) and cached.
int scratch_address(DotScratch** out) {
  int dev = -1;
  SEM_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= sem::MAX_DEVICES) {
    sem::set_detail("sem_dot_static: device ordinal %d out of range", dev);
    return SEM_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_dot_scratch);
    if (e != cudaSuccess || !p) {
      sem::set_detail("sem_dot_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return SEM_ECUDA;
    }
    g_addr[dev] = static_cast<DotScratch*>(p);
  }
  *out = g_addr[dev];
  return SEM_OK;
}

}  // namespace

extern "C" int sem_dot_static(const double* a, const double* b, const uint8_t* mask, int64_t n, double* out,
                              void* stream) {
  if (!a || !b || !out || n < 0) {
    sem::set_detail("sem_dot_static: NULL vector/output or negative length");
    return SEM_EINVAL;
  }
  if (n > DS_MAX_N) {
    sem::set_detail("sem_dot_static: n = %lld exceeds the static scratch capacity of %lld elements",
                    (long long)n, (long long)DS_MAX_N);
    return SEM_EINVAL;
  }
  DotScratch* S = nullptr;
  SEM_TRY(scratch_address(&S));
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0) {
    SEM_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(double), s));
    return SEM_OK;
  }
  // the completion counter must start at zero (the previous call leaves it at zero;
  // clearing it here also recovers from an interrupted call)
  SEM_CUDA_TRY(cudaMemsetAsync(&S->ticket, 0, sizeof(unsigned int), s));
  const unsigned nblk = (unsigned)((n + DS_TILE - 1) / DS_TILE);
  k_dot_static<<<nblk, DS_THREADS, 0, s>>>(n, a, b, mask, S, out);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}
