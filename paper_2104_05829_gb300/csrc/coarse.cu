// Coarsest-level Jacobi-PCG (order 1) in one launch on one thread-block
// cluster, with the whole problem resident on chip.
//
// When the coarse problem fits one cluster of 8 or 16 CTAs, its state never
// leaves the SMs during the solve: each CTA owns a slice of whole elements, the
// per-point Krylov vectors (x, r, p, the Jacobi weights) sit in registers, the
// CTA's geometric factors and its operator output w in shared memory, and the
// gather-scatter reads and writes the copies held by other CTAs through
// distributed shared memory. An iteration:
//   1. w = A_L p on the CTA's elements (warp shuffles inside 8-lane element groups);
//   2. cluster barrier; gather-scatter of the shared and Dirichlet nodes (the
//      CTA's share of the segments; a copy is addressed as (CTA rank, offset));
//   3. cluster barrier; (p, w) over owner points; alpha; x, r update;
//      (r, r), (r, D^-1 r); beta and the convergence test; p update.
// Dot products: per-thread FP32 sums, FP64 block sums published in shared
// memory, and one warp per CTA adding all CTAs' block sums in a fixed order
// through distributed shared memory, so every CTA holds the same bits and takes
// the same branches. Phases are separated by the hardware cluster barrier.
// The algorithm is the multi-kernel one: x0 = 0, r = b, z = D^-1 r, stop when
// (r, r) <= tol^2 (b, b) or after maxit iterations. It serves the FP32 and
// BF16-factor V-cycles at order 1.
#include <cooperative_groups.h>

#include <algorithm>

#include "sem_internal.cuh"

namespace cg = cooperative_groups;

namespace sem {

namespace {

constexpr int CT = 512;     // threads per CTA
constexpr int NPO = 2;      // order 1
constexpr int P8 = 8;       // points per element

struct CoarseArgs {
  int E;
  int epc;                  // elements per CTA
  int64_t nseg;
  const void* G;            // factors [E][7][8] (FP32 or BF16)
  const float* b;
  float* x;
  const float* dinv;
  const uint8_t* own;
  const int32_t* seg_off;
  const int32_t* seg_loc;   // (CTA rank << 24 | offset) of every copy, in segment order
  const uint8_t* seg_dir;
  float h1, h2;
  double tol;
  int maxit;
  double* sc;               // outputs: S_ITER, S_TOTAL, S_RR, S_BB, S_DONE, S_BREAK
};

__device__ __forceinline__ float gval(float v) { return v; }
__device__ __forceinline__ float gval(__nv_bfloat16 v) { return __bfloat162float(v); }

// Cluster-wide sums of per-thread FP32 partials, identical in every CTA: FP32
// warp trees, the warp partials of the block in FP64 by warp 0, then warp 0
// fetches the block partials of all CTAs through distributed shared memory
// (lane q reads CTA q) and adds them in a fixed shuffle tree. The two slot
// buffers alternate, so one cluster barrier per sum suffices: a slot is
// rewritten only after the next sum's barrier, which every CTA reaches after
// reading it.
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
      double t = lane < CT / 32 ? (double)s_w[lane][s] : 0.0;
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

// address of a copy's operator output in the shared memory of the CTA that owns it
__device__ __forceinline__ float* w_at(cg::cluster_group& cl, float* sw, int32_t loc) {
  return cl.map_shared_rank(sw + (loc & 0xffffff), (unsigned)loc >> 24);
}

// loc[q] = (rank << 24) | offset for copy q: local point l lies in element l / 8,
// which CTA (l / 8) / epc holds at offset l - rank * epc * 8
__global__ void k_cluster_loc(int64_t n, const int32_t* __restrict__ idx, int epc, int32_t* __restrict__ loc) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int l = idx[q];
  const int rk = (l >> 3) / epc;
  loc[q] = (rk << 24) | (l - rk * epc * P8);
}

template <typename GT, int PPT>
__global__ void __launch_bounds__(CT) k_coarse_cluster(CoarseArgs a, Mat32 D) {
  extern __shared__ __align__(16) unsigned char s_raw[];
  cg::cluster_group cl = cg::this_cluster();
  const int epc = a.epc;
  float* sw = reinterpret_cast<float*>(s_raw);                                  // [epc * 8] operator output
  GT* sG = reinterpret_cast<GT*>(s_raw + (size_t)epc * P8 * sizeof(float));     // [epc][7][8] factors
  __shared__ double slots[2][4];
  __shared__ double tot[4];
  __shared__ float s_scal;   // alpha or beta, computed once per CTA by thread 0
  __shared__ int s_flag;     // 0 go on, 1 converged, 2 breakdown
  int parity = 0;
  const unsigned rank = cl.block_rank(), ncta = cl.num_blocks();
  const int e0 = min(a.E, (int)rank * epc), e1 = min(a.E, e0 + epc);
  const int npts = (e1 - e0) * P8;
  const int64_t p0 = (int64_t)e0 * P8;
  const GT* G = static_cast<const GT*>(a.G);
  for (int q = threadIdx.x; q < (e1 - e0) * 7 * P8; q += CT) sG[q] = G[(int64_t)e0 * 7 * P8 + q];
  const int64_t s0 = a.nseg * rank / ncta, s1 = a.nseg * (rank + 1) / ncta;
  const int lq = threadIdx.x & 7;
  const int i = lq & 1, j = (lq >> 1) & 1, k = lq >> 2;
  const float d00 = D.a[0], d01 = D.a[1], d10 = D.a[2], d11 = D.a[3];
  const float di_s = i ? d11 : d00, di_o = i ? d10 : d01;   // D[i][i], D[i][1-i]
  const float dj_s = j ? d11 : d00, dj_o = j ? d10 : d01;
  const float dk_s = k ? d11 : d00, dk_o = k ? d10 : d01;
  const float ti_o = i ? d01 : d10, tj_o = j ? d01 : d10, tk_o = k ? d01 : d10;   // D[1-a][a]
  float x[PPT], r[PPT], p[PPT], dinv[PPT];
  unsigned own = 0, live = 0;   // bit c: point c is an owner / exists
  float f2[2] = {0.f, 0.f};
#pragma unroll
  for (int c = 0; c < PPT; ++c) {
    const int lp = threadIdx.x + c * CT;
    x[c] = r[c] = p[c] = dinv[c] = 0.f;
    if (lp < npts) {
      const int64_t l = p0 + lp;
      live |= 1u << c;
      const float bl = a.b[l];
      dinv[c] = a.dinv[l];
      r[c] = bl;
      p[c] = dinv[c] * bl;
      if (a.own[l]) {
        own |= 1u << c;
        f2[0] = fmaf(bl, bl, f2[0]);
        f2[1] = fmaf(bl, p[c], f2[1]);
      }
    }
  }
  cluster_sum<2>(f2, &slots, tot, parity, cl);   // its barriers also order the factor staging
  // the FP64 scalar recurrences run in thread 0 only (FP64 division is slow on this part)
  double bb = tot[0], rz = tot[1], rr = bb;
  const double tol2 = a.tol * a.tol * bb;
  int flag = rr <= tol2 ? 1 : 0;
  int it = 0;
  while (flag == 0 && it < a.maxit) {
    // 1. w = A_L p on this CTA's elements, into shared memory
#pragma unroll
    for (int c = 0; c < PPT; ++c) {
      const int lp = threadIdx.x + c * CT;
      const bool lv = (live >> c) & 1u;
      const float u = p[c];
      const float ur = di_s * u + di_o * __shfl_xor_sync(0xffffffffu, u, 1);
      const float us = dj_s * u + dj_o * __shfl_xor_sync(0xffffffffu, u, 2);
      const float ut = dk_s * u + dk_o * __shfl_xor_sync(0xffffffffu, u, 4);
      float wr = 0.f, ws = 0.f, wt = 0.f, bu = 0.f;
      if (lv) {
        const GT* g = sG + (lp >> 3) * 7 * P8 + lq;
        const float g11 = gval(g[0]), g12 = gval(g[8]), g13 = gval(g[16]);
        const float g22 = gval(g[24]), g23 = gval(g[32]), g33 = gval(g[40]);
        wr = a.h1 * (g11 * ur + g12 * us + g13 * ut);
        ws = a.h1 * (g12 * ur + g22 * us + g23 * ut);
        wt = a.h1 * (g13 * ur + g23 * us + g33 * ut);
        bu = a.h2 * gval(g[48]) * u;
      }
      float acc = bu + di_s * wr + ti_o * __shfl_xor_sync(0xffffffffu, wr, 1);
      acc += dj_s * ws + tj_o * __shfl_xor_sync(0xffffffffu, ws, 2);
      acc += dk_s * wt + tk_o * __shfl_xor_sync(0xffffffffu, wt, 4);
      if (lv) sw[lp] = acc;
    }
    cl.sync();   // every CTA's w complete
    // 2. gather-scatter over distributed shared memory
    for (int64_t sg = s0 + threadIdx.x; sg < s1; sg += CT) {
      const int bgn = a.seg_off[sg], end = a.seg_off[sg + 1];
      if (a.seg_dir[sg]) {
        for (int q = bgn; q < end; ++q) *w_at(cl, sw, a.seg_loc[q]) = 0.f;
      } else if (end - bgn > 1) {
        float* at[8];
        const int m = end - bgn;
        float sum = 0.f;
        if (m <= 8) {
#pragma unroll
          for (int t = 0; t < 8; ++t)
            if (t < m) at[t] = w_at(cl, sw, a.seg_loc[bgn + t]);
#pragma unroll
          for (int t = 0; t < 8; ++t)
            if (t < m) sum += *at[t];
#pragma unroll
          for (int t = 0; t < 8; ++t)
            if (t < m) *at[t] = sum;
        } else {
          for (int q = bgn; q < end; ++q) sum += *w_at(cl, sw, a.seg_loc[q]);
          for (int q = bgn; q < end; ++q) *w_at(cl, sw, a.seg_loc[q]) = sum;
        }
      }
    }
    cl.sync();   // assembled w visible in every CTA
    // 3. alpha = (r, z) / (p, w); x, r; beta
    float g1[1] = {0.f};
#pragma unroll
    for (int c = 0; c < PPT; ++c)
      if ((own >> c) & 1u) g1[0] = fmaf(p[c], sw[threadIdx.x + c * CT], g1[0]);
    cluster_sum<1>(g1, &slots, tot, parity, cl);
    if (threadIdx.x == 0) {
      const double pw = tot[0];
      const bool bad = !(pw > 0.0) || !isfinite(pw);
      s_flag = bad ? 2 : 0;
      s_scal = bad ? 0.f : (float)(rz / pw);
    }
    __syncthreads();
    if (s_flag != 0) {
      flag = 2;
      break;
    }
    const float at = s_scal;
    float q2[2] = {0.f, 0.f};
#pragma unroll
    for (int c = 0; c < PPT; ++c) {
      if (!((live >> c) & 1u)) continue;
      x[c] = fmaf(at, p[c], x[c]);
      r[c] = fmaf(-at, sw[threadIdx.x + c * CT], r[c]);
      if ((own >> c) & 1u) {
        q2[0] = fmaf(r[c], r[c], q2[0]);
        q2[1] = fmaf(r[c], dinv[c] * r[c], q2[1]);
      }
    }
    cluster_sum<2>(q2, &slots, tot, parity, cl);
    ++it;
    if (threadIdx.x == 0) {
      rr = tot[0];
      s_scal = (float)(tot[1] / rz);
      rz = tot[1];
      s_flag = !isfinite(rr) ? 2 : (rr <= tol2 ? 1 : 0);
    }
    __syncthreads();
    flag = s_flag;
    if (flag != 0) break;
    const float bt = s_scal;
#pragma unroll
    for (int c = 0; c < PPT; ++c) p[c] = fmaf(bt, p[c], dinv[c] * r[c]);
  }
#pragma unroll
  for (int c = 0; c < PPT; ++c)
    if ((live >> c) & 1u) a.x[p0 + threadIdx.x + c * CT] = x[c];
  cl.sync();   // no CTA leaves while another may still read its shared memory
  if (rank == 0 && threadIdx.x == 0) {
    a.sc[S_ITER] = it;
    a.sc[S_TOTAL] += it;
    a.sc[S_RR] = rr;
    a.sc[S_BB] = bb;
    a.sc[S_BREAK] = flag == 2 ? 1 : 0;
    a.sc[S_DONE] = 1;
  }
}

cudaLaunchConfig_t cluster_cfg(int cl, size_t smem, cudaStream_t s, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cl);
  cfg.blockDim = dim3(CT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

struct ClusterPlan {
  int cl = 0, epc = 0;
  size_t smem = 0;
  const void* f = nullptr;
};

// Can PPT points per thread hold E elements on a cluster of `cl` CTAs, with each
// CTA's factors and operator output in its shared memory?
template <typename GT, int PPT>
bool try_plan(int E, int cl, ClusterPlan* pl) {
  const int epc = (E + cl - 1) / cl;
  if ((int64_t)epc * P8 > (int64_t)CT * PPT) return false;
  const size_t smem = (size_t)epc * P8 * sizeof(float) + (size_t)epc * 7 * P8 * sizeof(GT);
  if (smem > 220 * 1024) return false;
  const void* f = (const void*)k_coarse_cluster<GT, PPT>;
  if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      (cl > 8 && cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = cluster_cfg(cl, smem, nullptr, attr);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, f, &cfg) != cudaSuccess || n < 1) {
    cudaGetLastError();
    return false;
  }
  pl->cl = cl;
  pl->epc = epc;
  pl->smem = smem;
  pl->f = f;
  return true;
}

template <typename GT>
bool cluster_plan(int E, ClusterPlan* pl) {
  for (int cl : {8, 16}) {
    if (try_plan<GT, 2>(E, cl, pl) || try_plan<GT, 4>(E, cl, pl) || try_plan<GT, 8>(E, cl, pl) ||
        try_plan<GT, 16>(E, cl, pl))
      return true;
  }
  return false;
}

template <typename GT>
int launch_coarse(const Level& L, const GT* G, const float* b, float* x, const float* dinv, double h1, double h2,
                  double tol, int maxit, double* sc, cudaStream_t s, bool* used) {
  *used = false;
  // the plan depends only on E and the factor type; remember the last one per type
  static ClusterPlan cached[2];
  static int cached_E[2] = {-1, -1};
  const int slot = sizeof(GT) == 4 ? 0 : 1;
  if (cached_E[slot] != L.E) {
    cached[slot] = ClusterPlan();
    if (!cluster_plan<GT>(L.E, &cached[slot])) cached[slot].cl = 0;
    cached_E[slot] = L.E;
  }
  const ClusterPlan pl = cached[slot];
  if (pl.cl == 0) return SEM_OK;
  if (pl.epc * P8 >= (1 << 24)) return SEM_OK;
  Level& Lm = const_cast<Level&>(L);
  if (!Lm.cl_loc || Lm.cl_loc_epc != pl.epc) {
    if (!Lm.cl_loc && cudaMalloc(&Lm.cl_loc, (size_t)std::max<int64_t>(L.n_seg_idx, 1) * sizeof(int32_t)) != cudaSuccess) {
      Lm.cl_loc = nullptr;
      cudaGetLastError();
      set_detail("cudaMalloc of the coarse gather-scatter locations failed");
      return SEM_ENOMEM;
    }
    if (L.n_seg_idx > 0) {
      k_cluster_loc<<<(unsigned)((L.n_seg_idx + 255) / 256), 256, 0, s>>>(L.n_seg_idx, L.seg_idx, pl.epc, Lm.cl_loc);
      SEM_LAUNCH_CHECK();
    }
    Lm.cl_loc_epc = pl.epc;
  }
  CoarseArgs a{};
  a.E = L.E;
  a.epc = pl.epc;
  a.nseg = L.n_seg;
  a.G = G;
  a.b = b;
  a.x = x;
  a.dinv = dinv;
  a.own = L.owner;
  a.seg_off = L.seg_off;
  a.seg_loc = L.cl_loc;
  a.seg_dir = L.seg_dir;
  a.h1 = (float)h1;
  a.h2 = (float)h2;
  a.tol = tol;
  a.maxit = maxit;
  a.sc = sc;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = cluster_cfg(pl.cl, pl.smem, s, attr);
  Mat32 D = L.Df;
  void* args[] = {&a, &D};
  SEM_CUDA_TRY(cudaLaunchKernelExC(&cfg, pl.f, args));
  *used = true;
  return SEM_OK;
}

}  // namespace

// One-launch, on-chip coarse solve for the FP32 / BF16-factor V-cycle at order 1;
// *used = false when it does not apply (FP64, another order, or the problem does
// not fit one cluster). r, p, w are not needed: the solve keeps them on chip.
int coarse_cluster_solve(const Level& L, int prec, const void* b, void* x, void* r, void* p, void* w,
                         const void* dinv, double h1, double h2, double tol, int maxit, double* sc,
                         cudaStream_t s, bool* used) {
  (void)r;
  (void)p;
  (void)w;
  *used = false;
  if (L.NP != NPO || prec == SEM_FP64) return SEM_OK;
  if (prec == SEM_FP32)
    return launch_coarse<float>(L, L.G32, (const float*)b, (float*)x, (const float*)dinv, h1, h2, tol, maxit, sc,
                                s, used);
  return launch_coarse<__nv_bfloat16>(L, L.G16, (const float*)b, (float*)x, (const float*)dinv, h1, h2, tol, maxit,
                                      sc, s, used);
}

}  // namespace sem
