// sem_measure_peaks: arithmetic peaks of the current device, measured with plain
// kernels and CUDA events. The paper has no counterpart; the library's roofline
// reports use these figures as the denominators of its arithmetic-bound kernels.
//
// * FP64 FMA: every thread runs 8 independent fma chains (2 flops per fma).
// * FP64 MMA: every warp runs 4 independent m16n8k8 mma.sync accumulations with an
//   operand that changes each round (constant operands can run faster than real data).
// * FP32 FMA: 8 independent chains of float fma per thread.
// Each kernel is launched once to warm up, then timed once; grids cover every SM
// several times over.
#include "sem_internal.cuh"

namespace sem {

namespace {

constexpr int PK_THREADS = 256;

__global__ void __launch_bounds__(PK_THREADS) k_peak_dfma(int iters, double b, double c, double* out) {
  double a[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) a[q] = threadIdx.x * 1e-3 + q;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = fma(a[q], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += a[q];
  out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PK_THREADS) k_peak_ffma(int iters, float b, float c, float* out) {
  float a[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) a[q] = threadIdx.x * 1e-3f + q;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = fmaf(a[q], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += a[q];
  out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}

__device__ __forceinline__ void mma_m16n8k8_f64(double (&d)[4], const double (&a)[4], const double (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+d"(d[0]), "+d"(d[1]), "+d"(d[2]), "+d"(d[3])
      : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(b[0]), "d"(b[1]));
}

__global__ void __launch_bounds__(PK_THREADS) k_peak_dmma(int iters, double* out) {
  double a[4], b[2], acc[4][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) a[q] = 0.5 + 1e-3 * (threadIdx.x + q);
  b[0] = 0.25;
  b[1] = 0.75;
#pragma unroll
  for (int q = 0; q < 4; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < 4; ++q) mma_m16n8k8_f64(acc[q], a, b);
    a[0] += 1e-12;
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < 4; ++q) s += acc[q][0] + acc[q][1] + acc[q][2] + acc[q][3];
  out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}

template <typename F>
int time_launch(F&& launch, float* ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SEM_CUDA_TRY(cudaEventCreate(&e0));
  const cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    SEM_CUDA_TRY(ce);
  }
  launch();   // warm-up
  cudaEventRecord(e0, 0);
  launch();
  cudaEventRecord(e1, 0);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  SEM_CUDA_TRY(e);
  return SEM_OK;
}

}  // namespace

}  // namespace sem

using namespace sem;

extern "C" int sem_measure_peaks(double* out) {
  if (!out) {
    set_detail("sem_measure_peaks: NULL output");
    return SEM_EINVAL;
  }
  int dev = 0, nsm = 0;
  SEM_CUDA_TRY(cudaGetDevice(&dev));
  SEM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = nsm * 8;
  const size_t n = (size_t)blocks * PK_THREADS;
  void* buf = nullptr;
  if (cudaMalloc(&buf, n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    set_detail("sem_measure_peaks: cudaMalloc failed");
    return SEM_ENOMEM;
  }
  const double threads = (double)n, warps = threads / 32.0;
  float ms = 0.f;
  int rc = SEM_OK;
  const int it64 = 4096, itmma = 256, it32 = 65536;
  if (rc == SEM_OK)
    rc = time_launch([&] { k_peak_dfma<<<blocks, PK_THREADS>>>(it64, 0.999, 1e-3, (double*)buf); }, &ms);
  if (rc == SEM_OK) out[0] = threads * it64 * 8 * 2.0 / (ms * 1e-3) / 1e12;
  if (rc == SEM_OK) rc = time_launch([&] { k_peak_dmma<<<blocks, PK_THREADS>>>(itmma, (double*)buf); }, &ms);
  if (rc == SEM_OK) out[1] = warps * itmma * 4 * (2.0 * 16 * 8 * 8) / (ms * 1e-3) / 1e12;
  if (rc == SEM_OK)
    rc = time_launch([&] { k_peak_ffma<<<blocks, PK_THREADS>>>(it32, 0.999f, 1e-3f, (float*)buf); }, &ms);
  if (rc == SEM_OK) out[2] = threads * it32 * 8 * 2.0 / (ms * 1e-3) / 1e12;
  cudaFree(buf);
  return rc;
}
