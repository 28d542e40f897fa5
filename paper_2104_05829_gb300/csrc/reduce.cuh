// Deterministic block reductions shared by the vector kernels (blas.cu, proj.cu).
//
// A fixed grid of RED_BLOCKS blocks walks the vector with a fixed stride; each
// block reduces its NS running sums in a fixed shuffle tree and stores them in
// part[s * gridDim.x + blockIdx.x]; the last block to finish (atomic ticket)
// adds the block partials in index order and calls fin(totals). The result
// does not depend on block scheduling. Nothing spins.
#pragma once

#include <cstdint>
#include <initializer_list>

#include "sem_internal.cuh"

namespace sem {

template <int NS>
struct Sums {
  double v[NS];
};

template <int NS>
__device__ __forceinline__ void warp_sum(Sums<NS>& a) {
#pragma unroll
  for (int s = 0; s < NS; ++s)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a.v[s] += __shfl_xor_sync(0xffffffffu, a.v[s], o);
}

// Block-reduce `a`, publish the block partial, and let the last block combine
// all partials in index order and call fin(totals).
template <int NS, class Fin>
__device__ void reduce_finish(Sums<NS> a, double* part, unsigned* ticket, Fin fin) {
  __shared__ double s_w[RED_THREADS / 32][NS];
  __shared__ bool s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  warp_sum(a);
  if (lane == 0)
#pragma unroll
    for (int s = 0; s < NS; ++s) s_w[warp][s] = a.v[s];
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      double t = 0;
      for (int w = 0; w < RED_THREADS / 32; ++w) t += s_w[w][s];
      part[s * gridDim.x + blockIdx.x] = t;
    }
    __threadfence();
    const unsigned t = atomicAdd(ticket, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  Sums<NS> b;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    double t = 0;
    for (unsigned q0 = threadIdx.x; q0 < gridDim.x; q0 += blockDim.x * 8) {
      double v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const unsigned q = q0 + blockDim.x * k;
        v[k] = q < gridDim.x ? __ldcg(part + s * gridDim.x + q) : 0.0;
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) t += v[k];
    }
    b.v[s] = t;
  }
  warp_sum(b);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int s = 0; s < NS; ++s) s_w[warp][s] = b.v[s];
  __syncthreads();
  if (threadIdx.x == 0) {
    Sums<NS> tot;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      double t = 0;
      for (int w = 0; w < RED_THREADS / 32; ++w) t += s_w[w][s];
      tot.v[s] = t;
    }
    fin(tot);
    *ticket = 0u;
  }
}

#define GRID_LOOP(l, n) \
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < (n); l += (int64_t)gridDim.x * blockDim.x)

// Grid-stride loop that takes U points a grid stride apart per trip: ld(l) for all
// U points first, then op(l, loaded) for each in order, so a thread keeps U points'
// loads in flight while earlier arithmetic (on GB300 often the narrow FP64 pipe)
// runs. The tail takes one point per trip. Each thread visits its points in a
// fixed order, so sums stay deterministic.
template <int U, class Ld, class Op>
__device__ __forceinline__ void grid_loop_u(int64_t n, Ld ld, Op op) {
  using V = decltype(ld(int64_t(0)));
  const int64_t S = (int64_t)gridDim.x * blockDim.x;
  int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; l + (U - 1) * S < n; l += U * S) {
    V v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = ld(l + u * S);
#pragma unroll
    for (int u = 0; u < U; ++u) op(l + u * S, v[u]);
  }
  for (; l < n; l += S) op(l, ld(l));
}

// Grid-stride loop over n floats in chunks of four: op4(i) handles elements 4i .. 4i+3 (the
// caller's pointers are 16-byte aligned), op1(l) each element of the tail.
template <class Op4, class Op1>
__device__ __forceinline__ void grid_loop_f4(int64_t n, Op4 op4, Op1 op1) {
  const int64_t n4 = n / 4, S = (int64_t)gridDim.x * blockDim.x, t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t i = t0; i < n4; i += S) op4(i);
  for (int64_t l = 4 * n4 + t0; l < n; l += S) op1(l);
}

__device__ __forceinline__ float4 ld4(const float* p, int64_t i) { return reinterpret_cast<const float4*>(p)[i]; }
__device__ __forceinline__ void st4(float* p, int64_t i, float4 v) { reinterpret_cast<float4*>(p)[i] = v; }

// FP32 vector kernels in chunks of four where the vectors allow it
constexpr bool kVec4 = true;

// true when every non-null pointer is 16-byte aligned
inline bool aligned16(std::initializer_list<const void*> ps) {
  for (const void* p : ps)
    if (p && ((uintptr_t)p & 15)) return false;
  return true;
}

}  // namespace sem
