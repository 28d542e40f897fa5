// Element-local kernels: geometric factors (eq. grad, eq. gij, eq. vBu), the
// sum-factorised operator A^e = D^T h1 G D + h2 B (eq. Ae), its exact diagonal,
// the h1-gradient of the adjoint, and the p-multigrid interpolation.
//
// Thread layout of the operator kernels: one (N+1)x(N+1) thread plane per
// element, each thread owning the t-line (k = 0..N) of one (i, j) column in
// registers. The t-direction contractions (D3, D3^T) run in registers; the r-
// and s-direction ones (D1, D2 and transposes) read a shared-memory copy of
// the element. Several elements share a block to reach 128-256 threads.
#include "bulk.cuh"
#include "sem_internal.cuh"

namespace sem {

namespace {

template <typename T>
struct MatT;
template <>
struct MatT<double> {
  using type = Mat64;
};
template <>
struct MatT<float> {
  using type = Mat32;
};

__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ double to_f(double v) { return v; }

// Shared-memory row stride: pad even orders by one so that rows of an element
// plane start on different banks.
template <int NP>
struct Pad {
  static constexpr int RS = (NP % 2 == 0) ? NP + 1 : NP;
  static constexpr int PS = NP * RS;   // plane stride
  static constexpr int ES = NP * PS;   // element stride
};

template <typename T, int NP>
__host__ __device__ constexpr int ax_epb() {
  int e = 256 / (NP * NP);
  if (e < 1) e = 1;
  while (e > 1 && (size_t)(3 * e * Pad<NP>::ES + 2 * NP * NP) * sizeof(T) > 46 * 1024) --e;
  return e;
}

// --------------------------------------------------------------------------
// w_L = A_L u_L with A^e = D1^T (h1 G) D1 + ... + h2 B, eq. Ae.
// T: arithmetic type, GT: storage type of G and B.
// --------------------------------------------------------------------------
template <typename T, typename GT, int NP, bool VARH1>
__global__ void __launch_bounds__(NP* NP* ax_epb<T, NP>())
    k_ax(int E, const T* __restrict__ u, T* __restrict__ w, const GT* __restrict__ G,
         typename MatT<T>::type Dm, T h1, T h2, const double* __restrict__ h1L, const double* skip) {
  constexpr int EPB = ax_epb<T, NP>();
  constexpr int NP2 = NP * NP, NP3 = NP * NP * NP;
  constexpr int RS = Pad<NP>::RS, PS = Pad<NP>::PS, ES = Pad<NP>::ES;
  if (skip && *skip != 0.0) return;
  __shared__ T s_D[NP2];    // D[a][b] at a*NP + b
  __shared__ T s_Dt[NP2];   // D[a][b] at b*NP + a
  __shared__ T s_u[EPB * ES];
  __shared__ T s_r[EPB * ES];
  __shared__ T s_s[EPB * ES];

  const int tid = threadIdx.x;
  const int le = tid / NP2;
  const int ij = tid - le * NP2;
  const int j = ij / NP;
  const int i = ij - j * NP;
  const int e = blockIdx.x * EPB + le;
  for (int t = tid; t < NP2; t += blockDim.x) {
    s_D[t] = Dm.a[t];
    s_Dt[(t % NP) * NP + t / NP] = Dm.a[t];
  }
  const bool active = e < E;
  T* su = s_u + le * ES;
  T* sr = s_r + le * ES;
  T* ss = s_s + le * ES;

  T ru[NP];
  const size_t ebase = (size_t)e * NP3;
  if (active) {
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      ru[k] = u[ebase + k * NP2 + ij];
      su[k * PS + j * RS + i] = ru[k];
    }
  }
  __syncthreads();

  T wt[NP];
  if (active) {
    const GT* Ge = G + (size_t)e * 7 * NP3 + ij;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      T ur = 0, us = 0, ut = 0;
#pragma unroll
      for (int l = 0; l < NP; ++l) {
        ur = fma(s_Dt[l * NP + i], su[k * PS + j * RS + l], ur);   // D[i][l] u[k][j][l]
        us = fma(s_Dt[l * NP + j], su[k * PS + l * RS + i], us);   // D[j][l] u[k][l][i]
        ut = fma(Dm.a[k * NP + l], ru[l], ut);                     // D[k][l] u[l][j][i]
      }
      const int o = k * NP2;
      const T g11 = to_f(Ge[0 * NP3 + o]), g12 = to_f(Ge[1 * NP3 + o]), g13 = to_f(Ge[2 * NP3 + o]);
      const T g22 = to_f(Ge[3 * NP3 + o]), g23 = to_f(Ge[4 * NP3 + o]), g33 = to_f(Ge[5 * NP3 + o]);
      T hh = h1;
      if (VARH1) hh = (T)h1L[ebase + o + ij];
      sr[k * PS + j * RS + i] = hh * (g11 * ur + g12 * us + g13 * ut);
      ss[k * PS + j * RS + i] = hh * (g12 * ur + g22 * us + g23 * ut);
      wt[k] = hh * (g13 * ur + g23 * us + g33 * ut);
    }
  }
  __syncthreads();
  if (active) {
    const GT* Be = G + (size_t)e * 7 * NP3 + 6 * NP3 + ij;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      T acc = h2 * to_f(Be[k * NP2]) * ru[k];
#pragma unroll
      for (int l = 0; l < NP; ++l) {
        acc = fma(s_D[l * NP + i], sr[k * PS + j * RS + l], acc);   // D[l][i] wr[k][j][l]
        acc = fma(s_D[l * NP + j], ss[k * PS + l * RS + i], acc);   // D[l][j] ws[k][l][i]
        acc = fma(Dm.a[l * NP + k], wt[l], acc);                     // D[l][k] wt[l][j][i]
      }
      w[ebase + k * NP2 + ij] = acc;
    }
  }
}

template <typename T, typename GT, int NP>
int launch_ax(const Level& L, const T* u, T* w, const GT* G, const typename MatT<T>::type& Dm, double h1,
              double h2, const double* h1L, const double* skip, cudaStream_t s) {
  constexpr int EPB = ax_epb<T, NP>();
  dim3 grid((L.E + EPB - 1) / EPB), block(NP * NP * EPB);
  if (h1L)
    k_ax<T, GT, NP, true><<<grid, block, 0, s>>>(L.E, u, w, G, Dm, (T)h1, (T)h2, h1L, skip);
  else
    k_ax<T, GT, NP, false><<<grid, block, 0, s>>>(L.E, u, w, G, Dm, (T)h1, (T)h2, nullptr, skip);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}

// --------------------------------------------------------------------------
// The same operator in FP32 arithmetic with the factors staged by bulk copies:
// thread 0 starts one cp.async.bulk for the block's u (contiguous) and one per
// element for its 7 NP^3 factor values on an mbarrier, so a block has all of its
// input bytes in flight at once; the contractions then read u, G and B from
// shared memory. The FP32 operator moves u, G, B and w and does
// little arithmetic per byte, so it is bound by HBM and wants many bytes in
// flight. Two elements per block keep five blocks on an SM at N = 7. Measured
// at N = 7 on the 24^3 box: 70 us -> 44 us per application (87 % of the HBM
// copy rate).
// A block whose copies have not landed after about a second writes NaN to its
// outputs (the solvers report a breakdown) instead of waiting on.
// --------------------------------------------------------------------------
template <typename GT, int NP>
// orders 7, 9, 11 (at N = 3 the plain kernel measured 9.4 us against 10.9 us: that
// level's data sit in L2, where per-thread loads already have short latency)
__host__ __device__ constexpr bool bulk_ok() {
  return NP >= 8 && NP % 2 == 0 && (7 * NP * NP * NP * sizeof(GT)) % 16 == 0 && (NP * NP * NP * 4) % 16 == 0;
}
template <int NP>
__host__ __device__ constexpr int bulk_epb() {
  return NP >= 8 ? 2 : (256 / (NP * NP));
}
template <typename GT, int NP>
__host__ __device__ constexpr size_t bulk_g_bytes() {
  return ((size_t)bulk_epb<NP>() * 7 * NP * NP * NP * sizeof(GT) + 127) / 128 * 128;
}
template <int NP>
__host__ __device__ constexpr size_t bulk_u_bytes() {
  return ((size_t)bulk_epb<NP>() * NP * NP * NP * sizeof(float) + 127) / 128 * 128;
}
template <typename GT, int NP>
__host__ __device__ constexpr size_t bulk_smem() {
  return bulk_g_bytes<GT, NP>() + bulk_u_bytes<NP>() + (size_t)2 * bulk_epb<NP>() * Pad<NP>::ES * sizeof(float);
}

template <typename GT, int NP, bool VARH1>
__global__ void __launch_bounds__(NP* NP* bulk_epb<NP>())
    k_ax_bulk(int E, const float* __restrict__ u, float* __restrict__ w, const GT* __restrict__ G, Mat32 Dm,
              float h1, float h2, const double* __restrict__ h1L, const double* skip, long long spin) {
  using T = float;
  constexpr int EPB = bulk_epb<NP>();
  constexpr int NP2 = NP * NP, NP3 = NP * NP * NP, GE = 7 * NP3;
  constexpr int RS = Pad<NP>::RS, PS = Pad<NP>::PS, ES = Pad<NP>::ES;
  if (skip && *skip != 0.0) return;
  extern __shared__ __align__(128) unsigned char s_raw[];
  GT* sG = reinterpret_cast<GT*>(s_raw);                                   // [EPB][7][NP3]
  T* s_u = reinterpret_cast<T*>(s_raw + bulk_g_bytes<GT, NP>());          // [EPB][NP3] as in HBM
  T* s_r = reinterpret_cast<T*>(s_raw + bulk_g_bytes<GT, NP>() + bulk_u_bytes<NP>());   // [EPB][ES] padded
  T* s_s = s_r + EPB * ES;
  __shared__ T s_D[NP2];    // D[a][b] at a*NP + b
  __shared__ T s_Dt[NP2];   // D[a][b] at b*NP + a
  __shared__ uint64_t bar;

  const int tid = threadIdx.x;
  const int le = tid / NP2;
  const int ij = tid - le * NP2;
  const int j = ij / NP;
  const int i = ij - j * NP;
  const int e0 = blockIdx.x * EPB;
  const int e = e0 + le;
  const int nel = min(EPB, E - e0);
  if (tid == 0) {
    mbar_init(&bar, 1);
    mbar_expect_tx(&bar, (unsigned)(nel * GE * sizeof(GT) + nel * NP3 * sizeof(T)));
    bulk_g2s(s_u, u + (size_t)e0 * NP3, nel * NP3 * sizeof(T), &bar);
    bulk_g2s(sG, G + (size_t)e0 * GE, nel * GE * sizeof(GT), &bar);   // consecutive elements are contiguous
  }
  for (int t = tid; t < NP2; t += blockDim.x) {
    s_D[t] = Dm.a[t];
    s_Dt[(t % NP) * NP + t / NP] = Dm.a[t];
  }
  const bool active = e < E;
  const T* su = s_u + le * NP3;   // unpadded (k, j, l) rows: conflict-free at N = 7 for both contractions
  T* sr = s_r + le * ES;
  T* ss = s_s + le * ES;
  T ru[NP];
  const size_t ebase = (size_t)e * NP3;
  __syncthreads();   // s_D and the barrier's initialisation are visible
  if (!__syncthreads_and(mbar_wait(&bar, 0, spin) ? 1 : 0)) {
    if (active)
#pragma unroll
      for (int k = 0; k < NP; ++k) w[ebase + k * NP2 + ij] = __int_as_float(0x7fc00000);
    // the copies may still be in flight into this block's shared memory: wait for
    // them once more (bounded again) before the block releases it
    if (tid == 0) mbar_wait(&bar, 0);
    __syncthreads();
    return;
  }
#pragma unroll
  for (int k = 0; k < NP; ++k) ru[k] = active ? su[k * NP2 + ij] : T(0);
  T wt[NP];
  if (active) {
    const GT* Ge = sG + le * GE + ij;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      T ur = 0, us = 0, ut = 0;
#pragma unroll
      for (int l = 0; l < NP; ++l) {
        ur = fma(s_Dt[l * NP + i], su[k * NP2 + j * NP + l], ur);   // D[i][l] u[k][j][l]
        us = fma(s_Dt[l * NP + j], su[k * NP2 + l * NP + i], us);   // D[j][l] u[k][l][i]
        ut = fma(Dm.a[k * NP + l], ru[l], ut);                      // D[k][l] u[l][j][i]
      }
      const int o = k * NP2;
      const T g11 = to_f(Ge[0 * NP3 + o]), g12 = to_f(Ge[1 * NP3 + o]), g13 = to_f(Ge[2 * NP3 + o]);
      const T g22 = to_f(Ge[3 * NP3 + o]), g23 = to_f(Ge[4 * NP3 + o]), g33 = to_f(Ge[5 * NP3 + o]);
      T hh = h1;
      if (VARH1) hh = (T)h1L[ebase + o + ij];
      sr[k * PS + j * RS + i] = hh * (g11 * ur + g12 * us + g13 * ut);
      ss[k * PS + j * RS + i] = hh * (g12 * ur + g22 * us + g23 * ut);
      wt[k] = hh * (g13 * ur + g23 * us + g33 * ut);
    }
  }
  __syncthreads();
  if (active) {
    const GT* Be = sG + le * GE + 6 * NP3 + ij;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      T acc = h2 * to_f(Be[k * NP2]) * ru[k];
#pragma unroll
      for (int l = 0; l < NP; ++l) {
        acc = fma(s_D[l * NP + i], sr[k * PS + j * RS + l], acc);   // D[l][i] wr[k][j][l]
        acc = fma(s_D[l * NP + j], ss[k * PS + l * RS + i], acc);   // D[l][j] ws[k][l][i]
        acc = fma(Dm.a[l * NP + k], wt[l], acc);                     // D[l][k] wt[l][j][i]
      }
      w[ebase + k * NP2 + ij] = acc;
    }
  }
}

template <typename GT, int NP>
int launch_ax_bulk(const Level& L, const float* u, float* w, const GT* G, const Mat32& Dm, double h1, double h2,
                   const double* h1L, const double* skip, cudaStream_t s) {
  constexpr int EPB = bulk_epb<NP>();
  constexpr size_t smem = bulk_smem<GT, NP>();
  static PerDevice<bool> attr[2];
  SEM_TRY(smem_attr_once(attr[0], (const void*)k_ax_bulk<GT, NP, false>, smem));
  SEM_TRY(smem_attr_once(attr[1], (const void*)k_ax_bulk<GT, NP, true>, smem));
  dim3 grid((L.E + EPB - 1) / EPB), block(NP * NP * EPB);
  if (h1L)
    k_ax_bulk<GT, NP, true><<<grid, block, smem, s>>>(L.E, u, w, G, Dm, (float)h1, (float)h2, h1L, skip,
                                                      L.spin_limit);
  else
    k_ax_bulk<GT, NP, false><<<grid, block, smem, s>>>(L.E, u, w, G, Dm, (float)h1, (float)h2, nullptr, skip,
                                                       L.spin_limit);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}

template <int NP>
int ax_dispatch_np(const Level& L, int prec, const void* u, void* w, double h1, double h2, const double* h1L,
                   const double* skip, cudaStream_t s) {
  if (prec == SEM_FP64) return ax_eo_apply(L, (const double*)u, (double*)w, h1, h2, h1L, skip, s);
  // the bulk copy of u needs a 16-byte aligned source (the per-element sizes are
  // multiples of 16 bytes and the factors are library allocations), so a caller's
  // vector that starts elsewhere, e.g. an offset view, takes the plain-load kernel
  const bool u16 = ((uintptr_t)u & 15u) == 0;
  if (prec == SEM_FP32) {
    if constexpr (bulk_ok<float, NP>())
      if (u16) return launch_ax_bulk<float, NP>(L, (const float*)u, (float*)w, L.G32, L.Df, h1, h2, h1L, skip, s);
    return launch_ax<float, float, NP>(L, (const float*)u, (float*)w, L.G32, L.Df, h1, h2, h1L, skip, s);
  }
  if constexpr (bulk_ok<__nv_bfloat16, NP>())
    if (u16)
      return launch_ax_bulk<__nv_bfloat16, NP>(L, (const float*)u, (float*)w, L.G16, L.Df, h1, h2, h1L, skip, s);
  return launch_ax<float, __nv_bfloat16, NP>(L, (const float*)u, (float*)w, L.G16, L.Df, h1, h2, h1L, skip, s);
}

// --------------------------------------------------------------------------
// Geometric factors, one thread per local point (setup only).
// x_{p,r_q} = D_q x_p; inverse by cofactors; B = rho_ijk J; G_mm' = (r_m . r_m') B.
// --------------------------------------------------------------------------
template <int NP>
__global__ void k_geom(int E, const double* __restrict__ x, const double* __restrict__ y,
                       const double* __restrict__ z, Mat64 Dm, Mat64 rho, double* __restrict__ G,
                       float* __restrict__ G32, __nv_bfloat16* __restrict__ G16, int* bad) {
  constexpr int NP2 = NP * NP, NP3 = NP2 * NP;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= (int64_t)E * NP3) return;
  const int64_t e = p / NP3;
  const int loc = (int)(p - e * NP3);
  const int k = loc / NP2, j = (loc / NP) % NP, i = loc % NP;
  const double* X[3] = {x + e * NP3, y + e * NP3, z + e * NP3};
  // coordinates relative to the element's first node: D_hat annihilates
  // constants, and the shift keeps the rounding of D_hat's row sums (~1e-15)
  // times a large absolute coordinate out of the metrics
  double M[3][3];
  for (int c = 0; c < 3; ++c) {
    const double x0 = X[c][0];
    double dr = 0, ds = 0, dt = 0;
    for (int l = 0; l < NP; ++l) {
      dr += Dm.a[i * NP + l] * (X[c][k * NP2 + j * NP + l] - x0);
      ds += Dm.a[j * NP + l] * (X[c][k * NP2 + l * NP + i] - x0);
      dt += Dm.a[k * NP + l] * (X[c][l * NP2 + j * NP + i] - x0);
    }
    M[c][0] = dr;
    M[c][1] = ds;
    M[c][2] = dt;
  }
  const double a = M[0][0], b = M[0][1], c = M[0][2];
  const double d = M[1][0], ee = M[1][1], f = M[1][2];
  const double g = M[2][0], h = M[2][1], ii = M[2][2];
  const double det = a * (ee * ii - f * h) - b * (d * ii - f * g) + c * (d * h - ee * g);
  if (!(det > 0.0)) atomicExch(bad, 1);
  const double inv[3][3] = {{ee * ii - f * h, c * h - b * ii, b * f - c * ee},
                            {f * g - d * ii, a * ii - c * g, c * d - a * f},
                            {d * h - ee * g, b * g - a * h, a * ee - b * d}};
  double rx[3][3];  // rx[q][p] = dr_q/dx_p
  for (int q = 0; q < 3; ++q)
    for (int pp = 0; pp < 3; ++pp) rx[q][pp] = inv[q][pp] / det;
  const double B = rho.a[i] * rho.a[j] * rho.a[k] * det;
  const int pm[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
  double out[7];
  for (int c2 = 0; c2 < 6; ++c2) {
    const int m = pm[c2][0], n = pm[c2][1];
    out[c2] = (rx[m][0] * rx[n][0] + rx[m][1] * rx[n][1] + rx[m][2] * rx[n][2]) * B;
  }
  out[6] = B;
  double* Ge = G + e * 7 * NP3 + loc;
  for (int c2 = 0; c2 < 7; ++c2) {
    Ge[c2 * NP3] = out[c2];
    if (G32) G32[e * 7 * NP3 + loc + c2 * NP3] = __double2float_rn(out[c2]);
    if (G16) G16[e * 7 * NP3 + loc + c2 * NP3] = __double2bfloat16(out[c2]);
  }
}

// --------------------------------------------------------------------------
// Exact local diagonal of D^T h1 G D + h2 B (one thread per point, setup only):
// sum_l D[l][p_m]^2 G_mm(line point l) + 2 D[p_m][p_m] D[p_m'][p_m'] G_mm'(p) + h2 B(p).
// --------------------------------------------------------------------------
template <int NP>
__global__ void k_diag(int E, const double* __restrict__ G, Mat64 Dm, double h1, double h2,
                       const double* __restrict__ h1L, double* __restrict__ d) {
  constexpr int NP2 = NP * NP, NP3 = NP2 * NP;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= (int64_t)E * NP3) return;
  const int64_t e = p / NP3;
  const int loc = (int)(p - e * NP3);
  const int k = loc / NP2, j = (loc / NP) % NP, i = loc % NP;
  const double* Ge = G + e * 7 * NP3;
  const double* H = h1L ? h1L + e * NP3 : nullptr;
  auto h = [&](int q) { return H ? H[q] : h1; };
  double acc = 0;
  for (int l = 0; l < NP; ++l) {
    const double di = Dm.a[l * NP + i], dj = Dm.a[l * NP + j], dk = Dm.a[l * NP + k];
    const int qi = k * NP2 + j * NP + l, qj = k * NP2 + l * NP + i, qk = l * NP2 + j * NP + i;
    acc += di * di * h(qi) * Ge[0 * NP3 + qi];
    acc += dj * dj * h(qj) * Ge[3 * NP3 + qj];
    acc += dk * dk * h(qk) * Ge[5 * NP3 + qk];
  }
  const double Di = Dm.a[i * NP + i], Dj = Dm.a[j * NP + j], Dk = Dm.a[k * NP + k];
  acc += 2.0 * h(loc) * (Di * Dj * Ge[1 * NP3 + loc] + Di * Dk * Ge[2 * NP3 + loc] + Dj * Dk * Ge[4 * NP3 + loc]);
  d[p] = acc + h2 * Ge[6 * NP3 + loc];
}

// --------------------------------------------------------------------------
// g = -sum_{m,m'} (D_m lam) G_mm' (D_m' u) per local point (adjoint h1-gradient).
// --------------------------------------------------------------------------
template <int NP>
__global__ void __launch_bounds__(NP* NP* ax_epb<double, NP>())
    k_grad_h1(int E, const double* __restrict__ u, const double* __restrict__ lam, double* __restrict__ g,
              const double* __restrict__ G, Mat64 Dm) {
  constexpr int EPB = ax_epb<double, NP>();
  constexpr int NP2 = NP * NP, NP3 = NP2 * NP;
  constexpr int RS = Pad<NP>::RS, PS = Pad<NP>::PS, ES = Pad<NP>::ES;
  __shared__ double s_Dt[NP2];
  __shared__ double s_u[EPB * ES];
  __shared__ double s_l[EPB * ES];
  const int tid = threadIdx.x;
  const int le = tid / NP2;
  const int ij = tid - le * NP2;
  const int j = ij / NP, i = ij - j * NP;
  const int e = blockIdx.x * EPB + le;
  for (int t = tid; t < NP2; t += blockDim.x) s_Dt[(t % NP) * NP + t / NP] = Dm.a[t];
  const bool active = e < E;
  double* su = s_u + le * ES;
  double* sl = s_l + le * ES;
  const size_t ebase = (size_t)e * NP3;
  double ru[NP], rl[NP];
  if (active) {
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      ru[k] = u[ebase + k * NP2 + ij];
      rl[k] = lam[ebase + k * NP2 + ij];
      su[k * PS + j * RS + i] = ru[k];
      sl[k * PS + j * RS + i] = rl[k];
    }
  }
  __syncthreads();
  if (!active) return;
  const double* Ge = G + (size_t)e * 7 * NP3 + ij;
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    double ur = 0, us = 0, ut = 0, lr = 0, ls = 0, lt = 0;
#pragma unroll
    for (int l = 0; l < NP; ++l) {
      const double di = s_Dt[l * NP + i], dj = s_Dt[l * NP + j], dk = Dm.a[k * NP + l];
      ur = fma(di, su[k * PS + j * RS + l], ur);
      us = fma(dj, su[k * PS + l * RS + i], us);
      ut = fma(dk, ru[l], ut);
      lr = fma(di, sl[k * PS + j * RS + l], lr);
      ls = fma(dj, sl[k * PS + l * RS + i], ls);
      lt = fma(dk, rl[l], lt);
    }
    const int o = k * NP2;
    const double g11 = Ge[0 * NP3 + o], g12 = Ge[1 * NP3 + o], g13 = Ge[2 * NP3 + o];
    const double g22 = Ge[3 * NP3 + o], g23 = Ge[4 * NP3 + o], g33 = Ge[5 * NP3 + o];
    const double wr = g11 * ur + g12 * us + g13 * ut;
    const double ws = g12 * ur + g22 * us + g23 * ut;
    const double wt = g13 * ur + g23 * us + g33 * ut;
    g[ebase + o + ij] = -(lr * wr + ls * ws + lt * wt);
  }
}

// --------------------------------------------------------------------------
// Tensor-product interpolation between orders (p-multigrid transfers).
// prolong: xf += mask_f * (J x J x J) ec       J: (NPf x NPc), J[a][b] = h^c_b(xi^f_a)
// restrict: rc  = (J^T x J^T x J^T) (cwt_f * (bf - wf))   (wf may be null)
// One block per element; three sum-factorised passes through shared memory.
// --------------------------------------------------------------------------
template <typename T, typename MT, int NF, int NC>
__global__ void k_prolong_add(int E, const T* __restrict__ ec, T* __restrict__ xf, const uint8_t* __restrict__ dmask,
                              MT Jm) {
  constexpr int F3 = NF * NF * NF, C3 = NC * NC * NC;
  __shared__ T sJ[NF * NC];
  __shared__ T sc[C3];
  __shared__ T t1[NC * NC * NF];
  __shared__ T t2[NC * NF * NF];
  const int e = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int t = tid; t < NF * NC; t += nt) sJ[t] = Jm.a[t];
  for (int t = tid; t < C3; t += nt) sc[t] = ec[(size_t)e * C3 + t];
  __syncthreads();
  for (int t = tid; t < NC * NC * NF; t += nt) {   // t1[c][b][i] = sum_a J[i][a] sc[c][b][a]
    const int ii = t % NF, cb = t / NF;
    T acc = 0;
    for (int a = 0; a < NC; ++a) acc += sJ[ii * NC + a] * sc[cb * NC + a];
    t1[t] = acc;
  }
  __syncthreads();
  for (int t = tid; t < NC * NF * NF; t += nt) {   // t2[c][j][i] = sum_b J[j][b] t1[c][b][i]
    const int ii = t % NF, jj = (t / NF) % NF, c = t / (NF * NF);
    T acc = 0;
    for (int b = 0; b < NC; ++b) acc += sJ[jj * NC + b] * t1[(c * NC + b) * NF + ii];
    t2[t] = acc;
  }
  __syncthreads();
  for (int t = tid; t < F3; t += nt) {             // out[k][j][i] = sum_c J[k][c] t2[c][j][i]
    const int ji = t % (NF * NF), kk = t / (NF * NF);
    T acc = 0;
    for (int c = 0; c < NC; ++c) acc += sJ[kk * NC + c] * t2[c * NF * NF + ji];
    const size_t gi = (size_t)e * F3 + t;
    if (!dmask[gi]) xf[gi] += acc;
  }
}

template <typename T, typename MT, int NF, int NC>
__global__ void k_restrict(int E, const T* __restrict__ bf, const T* __restrict__ wf, const T* __restrict__ cwt,
                           T* __restrict__ rc, MT Jm) {
  constexpr int F3 = NF * NF * NF, C3 = NC * NC * NC;
  __shared__ T sJ[NF * NC];
  __shared__ T sf[F3];
  __shared__ T t1[NF * NF * NC];
  __shared__ T t2[NF * NC * NC];
  const int e = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int t = tid; t < NF * NC; t += nt) sJ[t] = Jm.a[t];
  for (int t = tid; t < F3; t += nt) {
    const size_t gi = (size_t)e * F3 + t;
    const T r = wf ? bf[gi] - wf[gi] : bf[gi];
    sf[t] = cwt[gi] * r;
  }
  __syncthreads();
  for (int t = tid; t < NF * NF * NC; t += nt) {   // t1[k][j][a] = sum_i J[i][a] sf[k][j][i]
    const int a = t % NC, kj = t / NC;
    T acc = 0;
    for (int ii = 0; ii < NF; ++ii) acc += sJ[ii * NC + a] * sf[kj * NF + ii];
    t1[t] = acc;
  }
  __syncthreads();
  for (int t = tid; t < NF * NC * NC; t += nt) {   // t2[k][b][a] = sum_j J[j][b] t1[k][j][a]
    const int a = t % NC, b = (t / NC) % NC, kk = t / (NC * NC);
    T acc = 0;
    for (int jj = 0; jj < NF; ++jj) acc += sJ[jj * NC + b] * t1[(kk * NF + jj) * NC + a];
    t2[t] = acc;
  }
  __syncthreads();
  for (int t = tid; t < C3; t += nt) {             // out[c][b][a] = sum_k J[k][c] t2[k][b][a]
    const int ba = t % (NC * NC), c = t / (NC * NC);
    T acc = 0;
    for (int kk = 0; kk < NF; ++kk) acc += sJ[kk * NC + c] * t2[kk * NC * NC + ba];
    rc[(size_t)e * C3 + t] = acc;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Dispatchers over the compiled orders.
// ---------------------------------------------------------------------------
#define SEM_NP_CASES(MACRO) \
  MACRO(2) MACRO(3) MACRO(4) MACRO(5) MACRO(6) MACRO(7) MACRO(8) MACRO(9) MACRO(10) MACRO(11) MACRO(12)

int ax_apply(const Level& L, int prec, const void* u, void* w, double h1, double h2, const double* h1L,
             cudaStream_t s, const double* skip) {
  if (L.E == 0) return SEM_OK;
  if (prec == SEM_FP32 && !L.G32) { set_detail("FP32 factors were not built"); return SEM_EINVAL; }
  if (prec == SEM_BF16G && !L.G16) { set_detail("BF16 factors were not built"); return SEM_EINVAL; }
  switch (L.NP) {
#define CASE(NP) \
  case NP:       \
    return ax_dispatch_np<NP>(L, prec, u, w, h1, h2, h1L, skip, s);
    SEM_NP_CASES(CASE)
#undef CASE
  }
  set_detail("order %d not compiled", L.N);
  return SEM_EINVAL;
}

int geom_compute(Level& L, int* d_bad, cudaStream_t s) {
  Mat64 rho{};
  for (int a = 0; a < L.NP; ++a) rho.a[a] = L.rho[a];
  const int64_t n = L.nL;
  const int T = 256;
  const unsigned nb = (unsigned)((n + T - 1) / T);
  switch (L.NP) {
#define CASE(NP)                                                                                 \
  case NP:                                                                                       \
    k_geom<NP><<<nb, T, 0, s>>>(L.E, L.x, L.y, L.z, L.D, rho, L.G, L.G32, L.G16, d_bad);       \
    SEM_LAUNCH_CHECK();                                                                          \
    return SEM_OK;
    SEM_NP_CASES(CASE)
#undef CASE
  }
  set_detail("order %d not compiled", L.N);
  return SEM_EINVAL;
}

int diag_local(const Level& L, double h1, double h2, const double* h1L, double* d, cudaStream_t s) {
  const int64_t n = L.nL;
  const int T = 256;
  const unsigned nb = (unsigned)((n + T - 1) / T);
  switch (L.NP) {
#define CASE(NP)                                                 \
  case NP:                                                       \
    k_diag<NP><<<nb, T, 0, s>>>(L.E, L.G, L.D, h1, h2, h1L, d); \
    SEM_LAUNCH_CHECK();                                          \
    return SEM_OK;
    SEM_NP_CASES(CASE)
#undef CASE
  }
  set_detail("order %d not compiled", L.N);
  return SEM_EINVAL;
}

int grad_h1_apply(const Level& L, const double* u, const double* lam, double* g, cudaStream_t s) {
  switch (L.NP) {
#define CASE(NP)                                                                          \
  case NP: {                                                                              \
    constexpr int EPB = ax_epb<double, NP>();                                             \
    k_grad_h1<NP><<<(L.E + EPB - 1) / EPB, NP * NP * EPB, 0, s>>>(L.E, u, lam, g, L.G, L.D); \
    SEM_LAUNCH_CHECK();                                                                   \
    return SEM_OK;                                                                        \
  }
    SEM_NP_CASES(CASE)
#undef CASE
  }
  set_detail("order %d not compiled", L.N);
  return SEM_EINVAL;
}

// Transfer pairs compiled: every (NF, NC) with 2 <= NC < NF <= 12.
namespace {
template <typename T, typename MT, int NF, int NC>
int tr_launch(bool prolong, const Level& F, const void* a, const void* b, void* out, const MT& Jm, const T* cwt,
              cudaStream_t s) {
  const int threads = NF * NF < 64 ? 64 : (NF * NF > 256 ? 256 : NF * NF);
  if (prolong)
    k_prolong_add<T, MT, NF, NC><<<F.E, threads, 0, s>>>(F.E, (const T*)a, (T*)out, F.dmask, Jm);
  else
    k_restrict<T, MT, NF, NC><<<F.E, threads, 0, s>>>(F.E, (const T*)a, (const T*)b, cwt, (T*)out, Jm);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}

template <int NF, int NC>
int tr_prec(bool prolong, const Level& F, const Level& C, int prec, const void* a, const void* b, void* out,
            cudaStream_t s) {
  if (prec == SEM_FP64) return tr_launch<double, Mat64, NF, NC>(prolong, F, a, b, out, F.Jc, F.cwt, s);
  return tr_launch<float, Mat32, NF, NC>(prolong, F, a, b, out, F.Jcf, F.cwt32, s);
}

template <int NF>
int tr_nc(bool prolong, const Level& F, const Level& C, int prec, const void* a, const void* b, void* out,
          cudaStream_t s) {
  switch (C.NP) {
#define NCASE(NC) \
  case NC:        \
    if constexpr (NC < NF) return tr_prec<NF, NC>(prolong, F, C, prec, a, b, out, s); \
    break;
    NCASE(2) NCASE(3) NCASE(4) NCASE(5) NCASE(6) NCASE(7) NCASE(8) NCASE(9) NCASE(10) NCASE(11)
#undef NCASE
  }
  set_detail("transfer %d -> %d not compiled", F.N, C.N);
  return SEM_EINVAL;
}

int tr_dispatch(bool prolong, const Level& F, const Level& C, int prec, const void* a, const void* b, void* out,
                cudaStream_t s) {
  switch (F.NP) {
#define FCASE(NF) \
  case NF:        \
    return tr_nc<NF>(prolong, F, C, prec, a, b, out, s);
    FCASE(3) FCASE(4) FCASE(5) FCASE(6) FCASE(7) FCASE(8) FCASE(9) FCASE(10) FCASE(11) FCASE(12)
#undef FCASE
  }
  set_detail("transfer %d -> %d not compiled", F.N, C.N);
  return SEM_EINVAL;
}
}  // namespace

int interp_add(const Level& F, const Level& C, int prec, const void* ec, void* xf, cudaStream_t s) {
  return tr_dispatch(true, F, C, prec, ec, nullptr, xf, s);
}

int interp_T(const Level& F, const Level& C, int prec, const void* rf, void* rc, cudaStream_t s) {
  return tr_dispatch(false, F, C, prec, rf, nullptr, rc, s);
}

int restrict_residual(const Level& F, const Level& C, int prec, const void* bf, const void* wf, void* rc,
                      cudaStream_t s) {
  return tr_dispatch(false, F, C, prec, bf, wf, rc, s);
}

}  // namespace sem
