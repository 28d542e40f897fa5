// Coarsest-level Jacobi-PCG in one launch on one thread-block cluster.
//
// The coarse problem of the p-multigrid V-cycle (order 1 by default, a few
// hundred thousand local points) is too small to fill the GPU, and a kernel
// per Krylov step makes its iterations launch- and latency-bound. Here the
// whole solve is one kernel on a single cluster of up to 16 CTAs:
//  - phases (element operator, gather-scatter, vector updates) are separated
//    by the hardware cluster barrier (barrier.cluster arrive/wait);
//  - every dot product is reduced block-wise, the block partials are
//    published in shared memory and one warp of every CTA reads all of them
//    through distributed shared memory and adds them in a fixed order, so all
//    CTAs hold the same bits and take the same branch (convergence, breakdown);
//  - vectors live in global memory (they fit in L2).
// The algorithm is the multi-kernel one: x0 = 0, r = b, z = D^-1 r, stop when
// (r,r) <= tol^2 (b,b) or after maxit iterations. It serves the FP32 and
// BF16-factor V-cycles at order 1 (one element per thread fits in registers);
// per-thread sums are FP32, block and cluster sums FP64. The FP64 V-cycle keeps
// the multi-kernel solve, which spreads its FP64 work over every SM.
// w is written by one CTA (element operator, gather-scatter) and read by
// others, so its accesses bypass L1 (__ldcg/__stcg); each CTA's point range is
// exactly the points of its elements, so x, r, p stay CTA-local.
#include <cooperative_groups.h>

#include "sem_internal.cuh"

namespace cg = cooperative_groups;

namespace sem {

namespace {

constexpr int CT = 1024;   // threads per CTA
constexpr int NP = 2;      // order 1
constexpr int NP3 = NP * NP * NP;

struct CoarseArgs {
  int E;
  int64_t nseg;
  const void* G;          // factors [E][7][8] (FP32 or BF16)
  const float* b;
  float* x;
  float* r;
  float* p;
  float* w;
  const float* dinv;
  const uint8_t* own;
  const int32_t* seg_off;
  const int32_t* seg_idx;
  const uint8_t* seg_dir;
  float h1, h2;
  double tol;
  int maxit;
  double* sc;             // outputs: S_ITER, S_TOTAL, S_RR, S_BB, S_DONE, S_BREAK
};

__device__ __forceinline__ float gload(const float* G, int64_t q) { return G[q]; }
__device__ __forceinline__ float gload(const __nv_bfloat16* G, int64_t q) { return __bfloat162float(G[q]); }

// Cluster-wide sums of per-thread FP32 partials, identical in every CTA: FP32
// warp trees, the 32 warp partials of the block in FP64 by warp 0, then warp 0
// fetches the block partials of all CTAs through distributed shared memory
// (lane q reads CTA q) and adds them in a fixed shuffle tree. The totals land in
// `tot` (shared). The two slot buffers alternate, so one cluster barrier per sum
// suffices: a slot is rewritten only after the next sum's barrier, which every
// CTA reaches after reading it. FP64 work stays in one warp per CTA.
template <int NS>
__device__ void cluster_sum(float (&v)[NS], double (*slots)[2][4], double* tot, int& parity,
                            cg::cluster_group& cl) {
  __shared__ float s_w[CT / 32][NS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < NS; ++s)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[s] += __shfl_xor_sync(0xffffffffu, v[s], o);
  if (lane == 0)
#pragma unroll
    for (int s = 0; s < NS; ++s) s_w[warp][s] = v[s];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      double t = (double)s_w[lane][s];   // CT / 32 == 32 warps: one partial per lane
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) (*slots)[parity][s] = t;
    }
  }
  cl.sync();
  if (warp == 0) {
    const unsigned ncta = cl.num_blocks();
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      double t = 0.0;
      if ((unsigned)lane < ncta) {
        double(*rs)[2][4] = cl.map_shared_rank(slots, (unsigned)lane);
        t = (*rs)[parity][s];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) tot[s] = t;
    }
  }
  parity ^= 1;
  __syncthreads();   // tot visible; s_w free for the next sum
}

// w = A_L p for the points [p0, p1) (whole elements), one point per thread.
// At order 1 the 8 points of an element are 8 consecutive lanes of a warp and
// the neighbour of point (i, j, k) along r, s, t is the lane with bit 0, 1 or
// 2 flipped, so every contraction is one shuffle: (D v)_a = D[a][a] v_a + D[a][1-a] v_partner.
template <typename GT>
__device__ void element_ax(const CoarseArgs& a, const Mat32& D, int64_t p0, int64_t p1) {
  const GT* G = static_cast<const GT*>(a.G);
  const int q = threadIdx.x & 7;                 // point within the element
  const int i = q & 1, j = (q >> 1) & 1, k = q >> 2;
  const float d00 = D.a[0], d01 = D.a[1], d10 = D.a[2], d11 = D.a[3];
  const float di_s = i ? d11 : d00, di_o = i ? d10 : d01;   // D[i][i], D[i][1-i]
  const float dj_s = j ? d11 : d00, dj_o = j ? d10 : d01;
  const float dk_s = k ? d11 : d00, dk_o = k ? d10 : d01;
  const float ti_o = i ? d01 : d10, tj_o = j ? d01 : d10, tk_o = k ? d01 : d10;   // D[1-a][a]
  // CT is a multiple of 8, and p0, p1 are multiples of 8: every warp pass covers whole elements
  for (int64_t l = p0 + threadIdx.x; l < p1 + ((p1 - p0) % CT ? CT - (p1 - p0) % CT : 0); l += CT) {
    const bool live = l < p1;
    const float u = live ? a.p[l] : 0.f;
    const float ur = di_s * u + di_o * __shfl_xor_sync(0xffffffffu, u, 1);
    const float us = dj_s * u + dj_o * __shfl_xor_sync(0xffffffffu, u, 2);
    const float ut = dk_s * u + dk_o * __shfl_xor_sync(0xffffffffu, u, 4);
    float wr = 0.f, ws = 0.f, wt = 0.f, bu = 0.f;
    if (live) {
      const int64_t e = l >> 3;
      const int64_t gb = e * 7 * NP3 + q;
      const float g11 = gload(G, gb), g12 = gload(G, gb + NP3), g13 = gload(G, gb + 2 * NP3);
      const float g22 = gload(G, gb + 3 * NP3), g23 = gload(G, gb + 4 * NP3), g33 = gload(G, gb + 5 * NP3);
      wr = a.h1 * (g11 * ur + g12 * us + g13 * ut);
      ws = a.h1 * (g12 * ur + g22 * us + g23 * ut);
      wt = a.h1 * (g13 * ur + g23 * us + g33 * ut);
      bu = a.h2 * gload(G, gb + 6 * NP3) * u;
    }
    float acc = bu + di_s * wr + ti_o * __shfl_xor_sync(0xffffffffu, wr, 1);
    acc += dj_s * ws + tj_o * __shfl_xor_sync(0xffffffffu, ws, 2);
    acc += dk_s * wt + tk_o * __shfl_xor_sync(0xffffffffu, wt, 4);
    if (live) __stcg(a.w + l, acc);
  }
}

template <typename GT>
__global__ void __maxnreg__(64) k_coarse_pcg(CoarseArgs a, Mat32 D) {
  cg::cluster_group cl = cg::this_cluster();
  __shared__ double slots[2][4];
  __shared__ double tot[4];
  __shared__ float s_alpha, s_beta;
  __shared__ int s_flag;   // 0 go on, 1 converged, 2 breakdown
  int parity = 0;
  const unsigned rank = cl.block_rank(), ncta = cl.num_blocks();
  const int e0 = (int)((int64_t)a.E * rank / ncta), e1 = (int)((int64_t)a.E * (rank + 1) / ncta);
  const int64_t p0 = (int64_t)e0 * NP3, p1 = (int64_t)e1 * NP3;
  const int64_t s0 = a.nseg * rank / ncta, s1 = a.nseg * (rank + 1) / ncta;
  const bool lead = threadIdx.x == 0;
  // scalars kept by the lead thread only (identical in every CTA)
  double bb = 0, rz = 0, rr = 0, tol2 = 0;

  // start: x = 0, r = b, p = D^-1 r; (b,b), (r,z)
  float f2[2] = {0.f, 0.f};
  for (int64_t l = p0 + threadIdx.x; l < p1; l += CT) {
    const float bl = a.b[l];
    a.x[l] = 0.f;
    a.r[l] = bl;
    const float zl = a.dinv[l] * bl;
    a.p[l] = zl;
    if (a.own[l]) {
      f2[0] = fmaf(bl, bl, f2[0]);
      f2[1] = fmaf(bl, zl, f2[1]);
    }
  }
  cluster_sum<2>(f2, &slots, tot, parity, cl);
  if (lead) {
    bb = tot[0];
    rz = tot[1];
    rr = bb;
    tol2 = a.tol * a.tol * bb;
    s_flag = rr <= tol2 ? 1 : 0;
  }
  __syncthreads();
  int it = 0;
  while (s_flag == 0 && it < a.maxit) {
    cl.sync();   // p complete in every CTA
    element_ax<GT>(a, D, p0, p1);
    cl.sync();   // w complete before the gather-scatter reads other CTAs' copies
    for (int64_t sg = s0 + threadIdx.x; sg < s1; sg += CT) {
      const int bgn = a.seg_off[sg], end = a.seg_off[sg + 1];
      if (a.seg_dir[sg]) {
        for (int q = bgn; q < end; ++q) __stcg(a.w + a.seg_idx[q], 0.f);
      } else if (end - bgn > 1) {
        float sum = __ldcg(a.w + a.seg_idx[bgn]);
        for (int q = bgn + 1; q < end; ++q) sum += __ldcg(a.w + a.seg_idx[q]);
        for (int q = bgn; q < end; ++q) __stcg(a.w + a.seg_idx[q], sum);
      }
    }
    cl.sync();   // assembled w visible
    float g[1] = {0.f};
    for (int64_t l = p0 + threadIdx.x; l < p1; l += CT)
      if (a.own[l]) g[0] = fmaf(a.p[l], __ldcg(a.w + l), g[0]);
    cluster_sum<1>(g, &slots, tot, parity, cl);
    if (lead) {
      const double pw = tot[0];
      if (!(pw > 0.0) || !isfinite(pw)) s_flag = 2;
      else s_alpha = (float)(rz / pw);
    }
    __syncthreads();
    if (s_flag != 0) break;
    const float at = s_alpha;
    float q2[2] = {0.f, 0.f};
    for (int64_t l = p0 + threadIdx.x; l < p1; l += CT) {
      a.x[l] = fmaf(at, a.p[l], a.x[l]);
      const float rl = fmaf(-at, __ldcg(a.w + l), a.r[l]);
      a.r[l] = rl;
      if (a.own[l]) {
        q2[0] = fmaf(rl, rl, q2[0]);
        q2[1] = fmaf(rl, a.dinv[l] * rl, q2[1]);
      }
    }
    cluster_sum<2>(q2, &slots, tot, parity, cl);
    ++it;
    if (lead) {
      rr = tot[0];
      const double beta = tot[1] / rz;
      rz = tot[1];
      s_beta = (float)beta;
      s_flag = !isfinite(rr) ? 2 : (rr <= tol2 ? 1 : 0);
    }
    __syncthreads();
    if (s_flag != 0) break;
    const float bt = s_beta;
    for (int64_t l = p0 + threadIdx.x; l < p1; l += CT) a.p[l] = fmaf(bt, a.p[l], a.dinv[l] * a.r[l]);
  }
  cl.sync();
  if (rank == 0 && lead) {
    a.sc[S_ITER] = it;
    a.sc[S_TOTAL] += it;
    a.sc[S_RR] = rr;
    a.sc[S_BB] = bb;
    a.sc[S_BREAK] = s_flag == 2 ? 1 : 0;
    a.sc[S_DONE] = 1;
  }
}

cudaLaunchConfig_t cluster_cfg(int cl, cudaStream_t s, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cl);
  cfg.blockDim = dim3(CT);
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// Largest cluster (16, 8, 4, 2 CTAs) the device can schedule for this kernel.
template <typename GT>
int cluster_size(cudaStream_t s) {
  static int cached[2] = {-1, -1};
  int& c = cached[sizeof(GT) == 4 ? 0 : 1];
  if (c >= 0) return c;
  const void* f = (const void*)k_coarse_pcg<GT>;
  c = 0;
  for (int cl : {16, 8, 4, 2}) {
    if (cl > 8 && cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_cfg(cl, s, attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, f, &cfg) == cudaSuccess && n >= 1) {
      c = cl;
      break;
    }
    cudaGetLastError();
  }
  return c;
}

template <typename GT>
int launch_coarse(const Level& L, const GT* G, const float* b, float* x, float* r, float* p, float* w,
                  const float* dinv, double h1, double h2, double tol, int maxit, double* sc, cudaStream_t s,
                  bool* used) {
  *used = false;
  const int cl = cluster_size<GT>(s);
  if (cl == 0) return SEM_OK;
  CoarseArgs a{};
  a.E = L.E;
  a.nseg = L.n_seg;
  a.G = G;
  a.b = b;
  a.x = x;
  a.r = r;
  a.p = p;
  a.w = w;
  a.dinv = dinv;
  a.own = L.owner;
  a.seg_off = L.seg_off;
  a.seg_idx = L.seg_idx;
  a.seg_dir = L.seg_dir;
  a.h1 = (float)h1;
  a.h2 = (float)h2;
  a.tol = tol;
  a.maxit = maxit;
  a.sc = sc;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = cluster_cfg(cl, s, attr);
  SEM_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_coarse_pcg<GT>, a, L.Df));
  *used = true;
  return SEM_OK;
}

}  // namespace

// One-launch coarse solve for the FP32 / BF16-factor V-cycle at order 1;
// *used = false when it does not apply (FP64, another order, no cluster fits).
int coarse_cluster_solve(const Level& L, int prec, const void* b, void* x, void* r, void* p, void* w,
                         const void* dinv, double h1, double h2, double tol, int maxit, double* sc,
                         cudaStream_t s, bool* used) {
  *used = false;
  if (L.NP != NP || prec == SEM_FP64) return SEM_OK;
  if (prec == SEM_FP32)
    return launch_coarse<float>(L, L.G32, (const float*)b, (float*)x, (float*)r, (float*)p, (float*)w,
                                (const float*)dinv, h1, h2, tol, maxit, sc, s, used);
  return launch_coarse<__nv_bfloat16>(L, L.G16, (const float*)b, (float*)x, (float*)r, (float*)p, (float*)w,
                                      (const float*)dinv, h1, h2, tol, maxit, sc, s, used);
}

}  // namespace sem
