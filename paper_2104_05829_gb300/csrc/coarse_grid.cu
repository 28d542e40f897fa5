// Coarsest-level Jacobi-PCG (order 1) in one cooperative launch over the whole GPU.
//
// The coarse problem (a few hundred thousand local points) is latency-bound:
// a kernel per Krylov step pays launch gaps, and a single cluster has too few
// SMs. Here every SM takes a slice of whole elements; per-point Krylov vectors
// (x, r, p, the Jacobi weights and flags) live in registers for the whole
// solve, each block's geometric factors are staged once in shared memory, and
// phases are separated by a grid barrier. The iteration is the Chronopoulos-Gear
// form of Jacobi-PCG (the same iterates in exact arithmetic, one reduction per
// iteration), which needs two barriers:
//   1. x, r, p and s = A p updated with the previous scalars; u = D^-1 r;
//      (r, u) and (r, r); element operator w_L = A_L u (registers + shared
//      memory, warp shuffles); barrier;
//   2. gather-scatter of the shared nodes (segments split across blocks) with
//      the (w, u) products of their owner copies; barrier; the three sums give
//      the convergence test, beta = (r, u)_new / (r, u) and
//      alpha = (r, u)_new / ((w, u) - beta (r, u)_new / alpha_old).
// Sums: per-thread partials (FP32 in the FP32 solve), block sums in FP64
// written to a partial array; after the barrier every block adds all block
// partials in the same fixed order, so all blocks hold the same bits and take
// the same branches. The grid barrier has no contended counter: each block
// publishes an epoch in its own flag, block 0 waits for all flags in parallel
// and releases the epoch. Waits are bounded: a block that waits longer than
// about a second sets an error flag, after which every barrier returns at once
// and the solve reports a breakdown.
// As in the multi-kernel solve: x0 = 0, r = b, stop when (r, r) <= tol^2 (b, b)
// or after maxit iterations.
#include <algorithm>

#include "sem_internal.cuh"
#include "spin.cuh"

namespace sem {

namespace {

constexpr int GT_THREADS = 256;
constexpr int NPC = 2;              // order 1
constexpr int NPC3 = 8;

struct GridArgs {
  int E;
  int64_t nseg;
  const void* G;                    // [E][7][8]
  const void* b;
  void* x;
  void* p_glob;                     // p at every point, read by the gather-scatter phase
  void* w;
  const void* dinv;
  const uint8_t* own;
  const int32_t* mult;
  const int32_t* seg_off;
  const int32_t* seg_idx;
  const uint8_t* seg_dir;
  double h1, h2;
  double tol;
  int maxit;
  int epb;                          // elements per block
  int spb;                          // gather-scatter segments per block (upper bound, staged in shared memory)
  double* part;                     // [3][gridDim.x] block partials
  unsigned* bar;                    // [gridDim.x] arrival epochs, then [1] the released epoch
  int* err;                         // barrier timeout flag
  double* sc;                       // outputs: S_ITER, S_TOTAL, S_RR, S_BB, S_DONE, S_BREAK
};

// factor value in the arithmetic type (FP64 factors stay FP64)
__device__ __forceinline__ double fval(double v) { return v; }
__device__ __forceinline__ float fval(float v) { return v; }
__device__ __forceinline__ float fval(__nv_bfloat16 v) { return __bfloat162float(v); }

// Grid barrier without a contended counter: every block publishes the barrier's
// epoch in its own flag; block 0's threads wait for all flags in parallel and
// then publish the epoch in `gen`, which the other blocks wait for. Epochs grow
// by one per barrier from 0 (flags and gen are zeroed before the launch).
// Waits are bounded (wait_at_least); after a timeout every barrier returns at once.
__device__ void grid_barrier(unsigned* flags, unsigned* gen, int* err, unsigned& epoch) {
  ++epoch;
  __syncthreads();
  const bool live = *(volatile int*)err == 0;
  if (threadIdx.x == 0 && live) {
    __threadfence();
    atomicExch(flags + blockIdx.x, epoch);
  }
  if (blockIdx.x == 0) {
    if (live)
      for (unsigned q = threadIdx.x; q < gridDim.x; q += blockDim.x) wait_at_least(flags + q, epoch, err);
    __syncthreads();
    if (threadIdx.x == 0 && live) {
      __threadfence();
      atomicExch(gen, epoch);
    }
  } else if (threadIdx.x == 0 && live) {
    wait_at_least(gen, epoch, err);
  }
  if (threadIdx.x == 0) __threadfence();
  __syncthreads();
}

// Block sum of NS values into part[s * nblk + blockIdx.x] (FP64), lane 0 of warp 0 writes.
template <int NS, typename T>
__device__ void block_partial(T (&v)[NS], double* part) {
  __shared__ double s_w[GT_THREADS / 32][NS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < NS; ++s)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[s] += __shfl_xor_sync(0xffffffffu, v[s], o);
  if (lane == 0)
#pragma unroll
    for (int s = 0; s < NS; ++s) s_w[warp][s] = (double)v[s];
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      double t = 0;
      for (int q = 0; q < GT_THREADS / 32; ++q) t += s_w[q][s];
      __stcg(part + s * gridDim.x + blockIdx.x, t);
    }
}

// Totals of the block partials, identical in every block (warp 0 reads them all
// in a fixed lane-strided order and reduces in a fixed shuffle tree). The loads of
// a lane are issued eight at a time before they are added (in the same order).
template <int NS>
__device__ void grid_totals(const double* part, double* tot) {
  if (threadIdx.x < 32) {
    const unsigned G = gridDim.x;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      double t = 0;
      for (unsigned q0 = threadIdx.x; q0 < G; q0 += 32 * 8) {
        double v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const unsigned q = q0 + 32 * k;
          v[k] = q < G ? __ldcg(part + s * G + q) : 0.0;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k)
          if (q0 + 32 * k < G) t += v[k];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (threadIdx.x == 0) tot[s] = t;
    }
  }
  __syncthreads();
}

template <typename T, typename GT, int PPT, bool SMEM_G>
__global__ void __launch_bounds__(GT_THREADS) k_coarse_grid(GridArgs a, Mat64 D) {
  extern __shared__ __align__(16) unsigned char s_raw[];
  GT* sG = reinterpret_cast<GT*>(s_raw);
  // after the factors: this block's segments (offsets, copies, Dirichlet flags)
  const size_t g_bytes = SMEM_G ? ((size_t)a.epb * 7 * NPC3 * sizeof(GT) + 15) / 16 * 16 : 0;
  int32_t* s_off = reinterpret_cast<int32_t*>(s_raw + g_bytes);    // [spb + 1]
  int32_t* s_idx = s_off + a.spb + 1;                               // [8 * spb]
  uint8_t* s_dir = reinterpret_cast<uint8_t*>(s_idx + 8 * a.spb);  // [spb]
  __shared__ double tot[3];
  __shared__ int s_flag;     // 0 go on, 1 converged, 2 breakdown, 3 iteration cap
  __shared__ T s_al, s_be;   // alpha and beta, computed once per block by thread 0
  const T* b = static_cast<const T*>(a.b);
  T* xg = static_cast<T*>(a.x);
  T* pg = static_cast<T*>(a.p_glob);
  T* w = static_cast<T*>(a.w);
  const T* dv = static_cast<const T*>(a.dinv);
  const GT* G = static_cast<const GT*>(a.G);
  const int e0 = min(a.E, (int)blockIdx.x * a.epb), e1 = min(a.E, e0 + a.epb);
  const int64_t p0 = (int64_t)e0 * NPC3;
  const int npts = (e1 - e0) * NPC3;
  // stage this block's factors (or read them from global memory when they do not fit)
  if (SMEM_G)
    for (int q = threadIdx.x; q < (e1 - e0) * 7 * NPC3; q += GT_THREADS) sG[q] = G[(int64_t)e0 * 7 * NPC3 + q];
  const GT* gb = SMEM_G ? sG : G + (int64_t)e0 * 7 * NPC3;
  // per-thread points: c-th point is p0 + threadIdx.x + c * GT_THREADS
  const int lq = threadIdx.x & 7;
  const int i = lq & 1, j = (lq >> 1) & 1, k = lq >> 2;
  const T d00 = (T)D.a[0], d01 = (T)D.a[1], d10 = (T)D.a[2], d11 = (T)D.a[3];
  const T di_s = i ? d11 : d00, di_o = i ? d10 : d01;
  const T dj_s = j ? d11 : d00, dj_o = j ? d10 : d01;
  const T dk_s = k ? d11 : d00, dk_o = k ? d10 : d01;
  const T ti_o = i ? d01 : d10, tj_o = j ? d01 : d10, tk_o = k ? d01 : d10;
  const T h1 = (T)a.h1, h2 = (T)a.h2;
  // Chronopoulos-Gear form of Jacobi-PCG (one reduction per iteration): with
  // u = D^-1 r and w = A u, gamma = (r, u), delta = (w, u);
  //   p = u + beta p, s = w + beta s (= A p), x += alpha p, r -= alpha s,
  //   beta = gamma_new / gamma, alpha = gamma_new / (delta - beta gamma_new / alpha_old).
  T x[PPT], r[PPT], p[PPT], sv[PPT], dinv[PPT];
  unsigned solo = 0, own = 0, live = 0;   // bit c: point c is an owner / an owner of a one-copy node / exists
#pragma unroll
  for (int c = 0; c < PPT; ++c) {
    const int lp = threadIdx.x + c * GT_THREADS;
    x[c] = r[c] = p[c] = sv[c] = dinv[c] = T(0);
    if (lp < npts) {
      const int64_t l = p0 + lp;
      live |= 1u << c;
      dinv[c] = dv[l];
      r[c] = b[l];
      if (a.own[l]) {
        own |= 1u << c;
        if (a.mult[l] == 1) solo |= 1u << c;
      }
    }
  }
  const int64_t s0 = a.nseg * blockIdx.x / gridDim.x, s1 = a.nseg * (blockIdx.x + 1) / gridDim.x;
  // stage the block's gather-scatter segments once (they never change); a block whose
  // segments hold more copies than the staging room reads them from global memory
  const int ns = (int)(s1 - s0);
  const int c0 = a.nseg > 0 ? a.seg_off[s0] : 0;
  const bool staged = ns <= a.spb && a.nseg > 0 && a.seg_off[s1] - c0 <= 8 * a.spb;
  if (staged) {
    for (int q = threadIdx.x; q <= ns; q += GT_THREADS) s_off[q] = a.seg_off[s0 + q] - c0;
    for (int q = threadIdx.x; q < a.seg_off[s1] - c0; q += GT_THREADS) s_idx[q] = a.seg_idx[c0 + q];
    for (int q = threadIdx.x; q < ns; q += GT_THREADS) s_dir[q] = a.seg_dir[s0 + q];
  }
  __syncthreads();
  const int32_t* g_off = staged ? s_off : a.seg_off + s0;    // offsets relative to g_idx
  const int32_t* g_idx = staged ? s_idx : a.seg_idx;
  const uint8_t* g_dir = staged ? s_dir : a.seg_dir + s0;
  unsigned epoch = 0;                 // barriers passed
  // scalar state, held by thread 0 only (FP64 division is slow on this part)
  double bb = 0, rr = 0, gam = 0, alpha_old = 0, tol2 = 0;
  int flag = 0, it = 0;               // flag: 0 go on, 1 converged, 2 breakdown, 3 iteration cap
  T al = T(0), be = T(0);
  bool first = true;
  while (true) {
    // update with the scalars of the previous pass (none in the first pass)
    if (!first) {
#pragma unroll
      for (int c = 0; c < PPT; ++c) {
        if (!((live >> c) & 1u)) continue;
        const int64_t l = p0 + threadIdx.x + c * GT_THREADS;
        p[c] = fma(be, p[c], dinv[c] * r[c]);
        sv[c] = fma(be, sv[c], __ldcg(w + l));
        x[c] = fma(al, p[c], x[c]);
        r[c] = fma(-al, sv[c], r[c]);
      }
    }
    // u = D^-1 r; (r, u), (r, r); w = A_L u; (w, u) on one-copy owners
    T acc[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int c = 0; c < PPT; ++c) {
      const int lp = threadIdx.x + c * GT_THREADS;
      const bool lv = (live >> c) & 1u;
      const T u = dinv[c] * r[c];
      if (lv) {
        __stcg(pg + p0 + lp, u);
        if ((own >> c) & 1u) {
          acc[0] = fma(r[c], u, acc[0]);
          acc[1] = fma(r[c], r[c], acc[1]);
        }
      }
      const T ur = di_s * u + di_o * __shfl_xor_sync(0xffffffffu, u, 1);
      const T us = dj_s * u + dj_o * __shfl_xor_sync(0xffffffffu, u, 2);
      const T ut = dk_s * u + dk_o * __shfl_xor_sync(0xffffffffu, u, 4);
      T wr = T(0), ws = T(0), wt = T(0), bu = T(0);
      if (lv) {
        const int le = lp >> 3;
        const GT* g = gb + le * 7 * NPC3 + lq;
        const T g11 = (T)fval(g[0]), g12 = (T)fval(g[8]), g13 = (T)fval(g[16]);
        const T g22 = (T)fval(g[24]), g23 = (T)fval(g[32]), g33 = (T)fval(g[40]);
        wr = h1 * (g11 * ur + g12 * us + g13 * ut);
        ws = h1 * (g12 * ur + g22 * us + g23 * ut);
        wt = h1 * (g13 * ur + g23 * us + g33 * ut);
        bu = h2 * (T)fval(g[48]) * u;
      }
      T wv = bu + di_s * wr + ti_o * __shfl_xor_sync(0xffffffffu, wr, 1);
      wv += dj_s * ws + tj_o * __shfl_xor_sync(0xffffffffu, ws, 2);
      wv += dk_s * wt + tk_o * __shfl_xor_sync(0xffffffffu, wt, 4);
      if (lv) {
        __stcg(w + p0 + lp, wv);
        if ((solo >> c) & 1u) acc[2] = fma(u, wv, acc[2]);
      }
    }
    grid_barrier(a.bar, a.bar + gridDim.x, a.err, epoch);
    // gather-scatter of shared / Dirichlet nodes, with (w, u) at their owner copies
    for (int sg = threadIdx.x; sg < ns; sg += GT_THREADS) {
      const int bgn = g_off[sg], end = g_off[sg + 1], m = end - bgn;
      if (g_dir[sg]) {
        for (int q = bgn; q < end; ++q) __stcg(w + g_idx[q], T(0));
      } else if (m <= 8) {
        // every load of the node's copies (and of u at its owner) in flight at once
        int id[8];
        T v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) id[t] = t < m ? g_idx[bgn + t] : 0;
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = t < m ? __ldcg(w + id[t]) : T(0);
        const T uo = __ldcg(pg + id[0]);
        T sum = v[0];
#pragma unroll
        for (int t = 1; t < 8; ++t)
          if (t < m) sum += v[t];
        if (m > 1)
#pragma unroll
          for (int t = 0; t < 8; ++t)
            if (t < m) __stcg(w + id[t], sum);
        acc[2] = fma(uo, sum, acc[2]);
      } else {
        T sum = __ldcg(w + g_idx[bgn]);
        for (int q = bgn + 1; q < end; ++q) sum += __ldcg(w + g_idx[q]);
        for (int q = bgn; q < end; ++q) __stcg(w + g_idx[q], sum);
        acc[2] = fma(__ldcg(pg + g_idx[bgn]), sum, acc[2]);
      }
    }
    block_partial<3>(acc, a.part);
    grid_barrier(a.bar, a.bar + gridDim.x, a.err, epoch);
    grid_totals<3>(a.part, tot);
    if (threadIdx.x == 0) {
      const double gnew = tot[0], del = tot[2];
      rr = tot[1];
      if (first) {
        bb = rr;
        tol2 = a.tol * a.tol * bb;
      } else {
        ++it;
      }
      int f = 0;
      double alpha = 0, beta = 0;
      if (*(volatile int*)a.err != 0 || !isfinite(rr)) f = 2;
      else if (rr <= tol2) f = 1;
      else if (it >= a.maxit) f = 3;
      else {
        beta = first ? 0.0 : gnew / gam;
        const double den = first ? del : del - beta * gnew / alpha_old;
        alpha = gnew / den;
        if (!(den > 0.0) || !(gnew > 0.0) || !isfinite(alpha)) f = 2;
      }
      gam = gnew;
      alpha_old = alpha;
      s_flag = f;
      s_al = (T)alpha;
      s_be = (T)beta;
    }
    __syncthreads();
    flag = s_flag;
    al = s_al;
    be = s_be;
    first = false;
    if (flag != 0) break;
  }
#pragma unroll
  for (int c = 0; c < PPT; ++c)
    if ((live >> c) & 1u) xg[p0 + threadIdx.x + c * GT_THREADS] = x[c];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.sc[S_ITER] = it;
    a.sc[S_TOTAL] += it;
    a.sc[S_RR] = rr;
    a.sc[S_BB] = bb;
    a.sc[S_BREAK] = flag == 2 ? 1 : 0;
    a.sc[S_DONE] = 1;
  }
}

struct GridPlan {
  int grid = 0, epb = 0, spb = 0;
  size_t smem = 0;
  const void* f = nullptr;
};

// A plan for PPT points per thread: the grid it needs must be co-resident and at
// most two blocks per SM (fewer arrivals per barrier).
// shared memory of a block: factors (when staged) and the segment staging room
template <typename GT, bool SMEM_G>
size_t grid_smem(int epb, int spb) {
  const size_t g = SMEM_G ? ((size_t)epb * 7 * NPC3 * sizeof(GT) + 15) / 16 * 16 : 0;
  return g + (size_t)(spb + 1) * 4 + (size_t)8 * spb * 4 + (size_t)spb;
}

template <typename T, typename GT, int PPT, bool SMEM_G>
bool plan_for(int E, int64_t nseg, int nsm, GridPlan* out) {
  const int epb = (PPT * GT_THREADS) / NPC3;                 // elements one block can hold
  const int grid = (E + epb - 1) / epb;
  const int spb = (int)((nseg + grid - 1) / grid) + 1;
  const size_t smem = grid_smem<GT, SMEM_G>(epb, spb);
  if (smem > 200 * 1024) return false;
  const void* f = (const void*)k_coarse_grid<T, GT, PPT, SMEM_G>;
  if (smem > 48 * 1024 && cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, GT_THREADS, smem) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (per_sm < 1 || grid > std::min(per_sm, 2) * nsm) return false;
  out->grid = grid;
  out->epb = (E + grid - 1) / grid;                          // spread the elements evenly
  out->spb = spb;
  out->smem = grid_smem<GT, SMEM_G>(out->epb, spb);
  out->f = f;
  return true;
}

template <typename T, typename GT>
bool make_plan(int E, int64_t nseg, int nsm, GridPlan* pl) {
  if (plan_for<T, GT, 1, true>(E, nseg, nsm, pl) || plan_for<T, GT, 2, true>(E, nseg, nsm, pl) ||
      plan_for<T, GT, 4, true>(E, nseg, nsm, pl) || plan_for<T, GT, 8, true>(E, nseg, nsm, pl) ||
      plan_for<T, GT, 16, true>(E, nseg, nsm, pl) || plan_for<T, GT, 8, false>(E, nseg, nsm, pl) ||
      plan_for<T, GT, 16, false>(E, nseg, nsm, pl))
    return true;
  if constexpr (sizeof(T) == 4) return plan_for<T, GT, 32, false>(E, nseg, nsm, pl);   // FP64 would spill
  return false;
}

template <typename T, typename GT>
int launch_grid(const Level& L, const GT* G, const void* b, void* x, void* pglob, void* w, const void* dinv,
                double h1, double h2, double tol, int maxit, double* sc, double* part, unsigned* bar, int* err,
                cudaStream_t s, bool* used) {
  *used = false;
  int dev = 0, nsm = 0;
  SEM_CUDA_TRY(cudaGetDevice(&dev));
  SEM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  GridPlan pl;
  if (!make_plan<T, GT>(L.E, L.n_seg, nsm, &pl)) return SEM_OK;   // does not fit: the caller falls back
  if (pl.grid > COARSE_GRID_MAX) return SEM_OK;
  GridArgs a{};
  a.E = L.E;
  a.nseg = L.n_seg;
  a.G = G;
  a.b = b;
  a.x = x;
  a.p_glob = pglob;
  a.w = w;
  a.dinv = dinv;
  a.own = L.owner;
  a.mult = L.mult;
  a.seg_off = L.seg_off;
  a.seg_idx = L.seg_idx;
  a.seg_dir = L.seg_dir;
  a.h1 = h1;
  a.h2 = h2;
  a.tol = tol;
  a.maxit = maxit;
  a.epb = pl.epb;
  a.spb = pl.spb;
  a.part = part;
  a.bar = bar;
  a.err = err;
  a.sc = sc;
  Mat64 D = L.D;
  void* args[] = {&a, &D};
  SEM_CUDA_TRY(cudaMemsetAsync(bar, 0, (pl.grid + 1) * sizeof(unsigned), s));
  SEM_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
  SEM_CUDA_TRY(cudaLaunchCooperativeKernel(pl.f, dim3(pl.grid), dim3(GT_THREADS), args, pl.smem, s));
  *used = true;
  return SEM_OK;
}

}  // namespace

// Whole-GPU coarse solve at order 1 (FP64, FP32 or BF16-factor V-cycles);
// *used = false when it does not apply (another order, or the grid does not fit).
// Scratch: part [3 * grid] doubles, bar [2] unsigned, err [1] int (Level-owned).
int coarse_grid_solve(const Level& L, int prec, const void* b, void* x, void* p, void* w, const void* dinv,
                      double h1, double h2, double tol, int maxit, double* sc, double* part, unsigned* bar, int* err,
                      cudaStream_t s, bool* used) {
  *used = false;
  if (L.NP != NPC) return SEM_OK;
  if (prec == SEM_FP64)
    return launch_grid<double, double>(L, L.G, b, x, p, w, dinv, h1, h2, tol, maxit, sc, part, bar, err, s, used);
  if (prec == SEM_FP32)
    return launch_grid<float, float>(L, L.G32, b, x, p, w, dinv, h1, h2, tol, maxit, sc, part, bar, err, s, used);
  return launch_grid<float, __nv_bfloat16>(L, L.G16, b, x, p, w, dinv, h1, h2, tol, maxit, sc, part, bar, err, s,
                                           used);
}

}  // namespace sem
