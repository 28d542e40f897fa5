// Dealiased advection operator (Section 2.1, the nonlinear term of eq. stdadv
// and the hyperbolic substeps of eq. hyp; Section 3.3 "High-Order Kernels":
// the term is evaluated on N_q^3 quadrature points with a 2-D thread plane and
// one register line per thread).
//
// For an advecting field c (three components) and ncomp advected fields u:
//   (C u)_i = sum_q w_q J_q phi_i(x_q) (c . grad u)(x_q),
// q over nq^3 Gauss-Legendre points, nq = ceil(3 (N+1) / 2). Per element:
//   1. each c_m is interpolated to the Gauss points (three sum-factorised
//      passes, the last one into the thread's register line along t);
//   2. the contravariant wind chat_d = sum_m Gq[d][m] c_m with the cubature
//      factors Gq = w J dr_d/dx_m (stored per point, set up once) -- kept in
//      registers and reused for every advected component (Section 3.3);
//   3. for each u: interpolation as in 1, derivatives on the Gauss points
//      (t along the thread's register line; r and s on lines of the Gauss-point
//      array in shared memory, each thread differentiating one whole line; all
//      three in even-odd form with the coefficients as kernel parameters), the
//      pointwise product sum_d chat_d du/dr_d, and the transposed interpolation
//      back to the GLL points (three passes).
// Thread (a, b) of the nq x nq plane owns the Gauss points (a, b, *).
#include <algorithm>
#include <cmath>
#include <vector>

#include "pairs.cuh"
#include "sem_internal.cuh"

namespace sem {

namespace {

// Arithmetics of the advection kernel: V the working value, S the stored vectors (c, u, w), G
// the stored cubature factors and 1-D matrices. Plain FMA in FP64 or FP32; or FP32 pairs
// (pairs.cuh, about 48 significant bits) on FP64 vectors with pre-split factors. The pair
// form keeps its sums unnormalised (lo may exceed ulp(hi)/2): each value only enters the
// error-free additions and products of pairs.cuh and the FP64 join at the store. Where two
// computed values meet in a product the dropped lo * lo term then grows: errors rose from
// 1.5e-13 to 6.2e-13 against the oracle (N = 2..8), still far below the 3e-11 bar, for a
// 16 % faster kernel (normalising the derivatives alone cost more than it saved).
template <typename T>
struct AdvPlain {
  using V = T;
  using S = T;
  using G = T;
  __device__ static V ld(const S* p, size_t i) { return p[i]; }
  __device__ static void st(S* p, size_t i, V v) { p[i] = v; }
  __device__ static V lg(const G* p, size_t i) { return p[i]; }
  __device__ static V zero() { return T(0); }
  __device__ static V mac(V acc, V a, V b) { return fma(a, b, acc); }
  __device__ static V mul(V a, V b) { return a * b; }
  __device__ static V add(V a, V b) { return a + b; }
  __device__ static V sub(V a, V b) { return a - b; }
  __device__ static V norm(V a) { return a; }
  static V host(double x) { return (T)x; }
};

struct AdvPair {
  using V = ff;
  using S = double;
  using G = float2;
  __device__ static V ld(const S* p, size_t i) { return ff_split(p[i]); }
  __device__ static void st(S* p, size_t i, V v) { p[i] = ff_join(v); }
  __device__ static V lg(const G* p, size_t i) {
    const float2 g = p[i];
    return {g.x, g.y};
  }
  __device__ static V zero() { return {0.f, 0.f}; }
  __device__ static V mac(V acc, V a, V b) { return ff_mac(acc, a, b); }
  __device__ static V mul(V a, V b) { return ff_mul(a, b); }
  __device__ static V add(V a, V b) { return ff_add_u(a, b); }
  __device__ static V sub(V a, V b) { return ff_sub_u(a, b); }
  __device__ static V norm(V a) { return a; }
  static V host(double x) { return ff_host_split(x); }
};

// Gauss-Legendre nodes (ascending) and weights: roots of P_n by Newton's method
// from x = cos(pi (4i - 1) / (4n + 2)), weights 2 / ((1 - x^2) P_n'(x)^2).
void host_gauss(int n, double* z, double* w) {
  for (int i = 1; i <= n; ++i) {
    double x = std::cos(M_PI * (4.0 * i - 1.0) / (4.0 * n + 2.0));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 1; k < n; ++k) {
        const double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
        p0 = p1;
        p1 = p2;
      }
      const double pn = n == 0 ? 1.0 : p1, pm1 = n == 0 ? 0.0 : p0;
      dp = n * (x * pn - pm1) / (x * x - 1.0);
      const double step = pn / dp;
      x -= step;
      if (std::fabs(step) < 1e-16) break;
    }
    z[n - i] = x;
    w[n - i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
  for (int i = 0; i < n / 2; ++i) {   // exact symmetry
    const double a = 0.5 * (z[n - 1 - i] - z[i]), b = 0.5 * (w[i] + w[n - 1 - i]);
    z[n - 1 - i] = a;
    z[i] = -a;
    w[i] = w[n - 1 - i] = b;
  }
  if (n % 2 == 1) z[n / 2] = 0.0;
}

// Dq[a][b] = h_b'(z_a) for the cardinal polynomials on the nodes z (barycentric form).
void host_deriv(int n, const double* z, double* D) {
  std::vector<double> lam(n, 1.0);
  for (int b = 0; b < n; ++b)
    for (int c = 0; c < n; ++c)
      if (c != b) lam[b] /= (z[b] - z[c]);
  for (int a = 0; a < n; ++a) {
    double diag = 0.0;
    for (int b = 0; b < n; ++b) {
      if (a == b) continue;
      D[a * n + b] = lam[b] / lam[a] / (z[a] - z[b]);
      diag -= D[a * n + b];
    }
    D[a * n + a] = diag;
  }
}

__host__ __device__ constexpr int nq_of(int NP) { return (3 * NP + 1) / 2; }

template <int NP>
struct AdvShape {
  static constexpr int NQ = nq_of(NP);
  static constexpr int T = NQ * NQ;                      // threads per element
  static constexpr int RS = NQ % 2 == 0 ? NQ + 1 : NQ;   // padded row stride of the Gauss-point arrays
  static constexpr int PS = NQ * RS;                     // plane stride
};

// dynamic shared memory of k_advect<Ar, NP>
template <class Ar, int NP>
constexpr size_t advect_smem() {
  constexpr int NQ = AdvShape<NP>::NQ, PS = AdvShape<NP>::PS;
  return sizeof(typename Ar::V) * ((size_t)NQ * NP + NQ * NQ + NP * NP * NP + NP * NP * NQ + 2 * NQ * PS + 3 * NQ * NQ * NQ);
}

// 1-D operators in shared memory: Im [NQ][NP] (GLL -> Gauss), Dq [NQ][NQ]
template <class Ar, int NP, int NQ>
__device__ __forceinline__ void load_ops(const typename Ar::G* __restrict__ Im, const typename Ar::G* __restrict__ Dq,
                                         typename Ar::V* sI, typename Ar::V* sD) {
  for (int q = threadIdx.x; q < NQ * NP; q += blockDim.x) sI[q] = Ar::lg(Im, q);
  for (int q = threadIdx.x; q < NQ * NQ; q += blockDim.x) sD[q] = Ar::lg(Dq, q);
}

// Interpolate the element's nodal field src (in shared memory, [k][j][i]) to the
// Gauss points; thread (a, b) receives its t-line out[c] = f(z_a, z_b, z_c).
// Uses t1 [NP][NP][NQ] in shared memory.
template <class Ar, int NP, int NQ>
__device__ __forceinline__ void to_gauss(const typename Ar::V* src, typename Ar::V* t1, const typename Ar::V* sI,
                                         const typename Ar::V* cI, int a, int b, typename Ar::V (&out)[NQ]) {
  using T = typename Ar::V;
  // r-pass: t1[k][j][a] for j < NP (threads with b < NP); row a of I held in registers
  if (b < NP) {
    T ia[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) ia[i] = sI[a * NP + i];
#pragma unroll 2
    for (int k = 0; k < NP; ++k) {
      T acc = Ar::zero();
#pragma unroll
      for (int i = 0; i < NP; ++i) acc = Ar::mac(acc, ia[i], src[(k * NP + b) * NP + i]);
      t1[(k * NP + b) * NQ + a] = Ar::norm(acc);
    }
  }
  __syncthreads();
  // s-pass into registers: t2[k] = sum_j I[b][j] t1[k][j][a]; row b of I in registers
  T t2[NP];
  {
    T ib[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) ib[j] = sI[b * NP + j];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      T acc = Ar::zero();
#pragma unroll
      for (int j = 0; j < NP; ++j) acc = Ar::mac(acc, ib[j], t1[(k * NP + j) * NQ + a]);
      t2[k] = Ar::norm(acc);
    }
  }
  // t-pass in registers (cI: the interpolation matrix at compile-time indices)
#pragma unroll
  for (int c = 0; c < NQ; ++c) {
    T acc = Ar::zero();
#pragma unroll
    for (int k = 0; k < NP; ++k) acc = Ar::mac(acc, cI[c * NP + k], t2[k]);
    out[c] = Ar::norm(acc);
  }
}

// 1-D operators passed by value (kernel parameters: with fully unrolled loops the
// coefficients become constant-bank operands, no shared-memory loads): the
// interpolation Im [NQ][NP] and the even-odd pieces of the Gauss derivative Dq,
// which is centro-antisymmetric (Dq[NQ-1-a][NQ-1-b] = -Dq[a][b]): with
// H = NQ / 2, s_b = v_b + v_{NQ-1-b} and d_b = v_b - v_{NQ-1-b},
//   ev_a = sum_b ep[a][b] s_b (+ mc[a] v_H if NQ is odd), od_a = sum_b op[a][b] d_b,
//   (Dq v)_a = ev_a + od_a, (Dq v)_{NQ-1-a} = od_a - ev_a, (Dq v)_H = sum_b mr[b] d_b (NQ odd),
// ep = (Dq[a][b] + Dq[a][NQ-1-b]) / 2, op = (Dq[a][b] - Dq[a][NQ-1-b]) / 2.
template <typename T, int NP>
struct AdvOps {
  static constexpr int NQ = nq_of(NP), H = NQ / 2;
  T Im[NQ * NP];
  T ep[H * H], op[H * H], mc[H > 0 ? H : 1], mr[H > 0 ? H : 1];
};

template <class Ar, int NP>
__device__ __forceinline__ void eo_deriv(const AdvOps<typename Ar::V, NP>& P, const typename Ar::V (&v)[nq_of(NP)],
                                         typename Ar::V (&o)[nq_of(NP)]) {
  using T = typename Ar::V;
  constexpr int NQ = nq_of(NP), H = NQ / 2, N = NQ - 1;
  T sm[H], df[H];
#pragma unroll
  for (int b = 0; b < H; ++b) {
    sm[b] = Ar::add(v[b], v[N - b]);
    df[b] = Ar::sub(v[b], v[N - b]);
  }
#pragma unroll
  for (int a = 0; a < H; ++a) {
    T ev = Ar::zero(), od = Ar::zero();
#pragma unroll
    for (int b = 0; b < H; ++b) {
      ev = Ar::mac(ev, P.ep[a * H + b], sm[b]);
      od = Ar::mac(od, P.op[a * H + b], df[b]);
    }
    if (NQ % 2 == 1) ev = Ar::mac(ev, P.mc[a], v[H]);
    o[a] = Ar::add(ev, od);
    o[N - a] = Ar::sub(od, ev);
  }
  if (NQ % 2 == 1) {
    T m = Ar::zero();
#pragma unroll
    for (int b = 0; b < H; ++b) m = Ar::mac(m, P.mr[b], df[b]);
    o[H] = Ar::norm(m);
  }
}

// resident blocks requested from the register allocator: four in FP32 up to N = 7 (18
// warps per SM, 96 registers with a 128-byte spill: measured 1.63 ms against 1.74 ms at
// three blocks with no spill on the 32^3 box), two at N = 8; two in FP64 (a few hundred
// bytes of spills, measured 1.26x faster at N = 7 than one block with no spills)
template <class Ar, int NP>
__host__ __device__ constexpr int adv_min_blocks() {
  return sizeof(typename Ar::V) == 4 ? (NP <= 8 ? 4 : 2) : 2;
}

template <class Ar, int NP>
__global__ void __launch_bounds__(AdvShape<NP>::T, (adv_min_blocks<Ar, NP>()))
    k_advect(int E, int ncomp, int64_t nL, const typename Ar::S* __restrict__ cv, const typename Ar::S* __restrict__ uv,
             const typename Ar::G* __restrict__ Gq, const typename Ar::G* __restrict__ Im,
             const typename Ar::G* __restrict__ Dq, typename Ar::S* __restrict__ wv, AdvOps<typename Ar::V, NP> P) {
  using T = typename Ar::V;
  constexpr int NQ = AdvShape<NP>::NQ, NP3 = NP * NP * NP, NQ2 = NQ * NQ, NQ3 = NQ2 * NQ;
  constexpr int RS = AdvShape<NP>::RS, PS = AdvShape<NP>::PS;
  // dynamic shared memory (advect_smem<Ar, NP>() bytes):
  extern __shared__ __align__(16) unsigned char s_raw[];
  T* sI = reinterpret_cast<T*>(s_raw);   // [NQ * NP] interpolation, runtime-indexed rows and columns
  T* sD = sI + NQ * NP;                  // [NQ * NQ]
  T* s_src = sD + NQ * NQ;               // [NP3] nodal field
  T* s_t1 = s_src + NP3;                 // [NP * NP * NQ] first interpolation pass; last projection pass
  T* s_U = s_t1 + NP * NP * NQ;          // [NQ * PS] u on the Gauss points; later the t-projected planes
  T* s_R = s_U + NQ * PS;                // [NQ * PS] a derivative, one direction at a time
  T* s_ch = s_R + NQ * PS;               // [3 * NQ3] the contravariant wind
  const int e = blockIdx.x;
  const int a = threadIdx.x % NQ, b = threadIdx.x / NQ;
  load_ops<Ar, NP, NQ>(Im, Dq, sI, sD);
  const size_t eb = (size_t)e * NP3;
  const typename Ar::G* G = Gq + (size_t)e * 9 * NQ3 + b * NQ + a;
  // 1-2. contravariant wind at this thread's points, kept in shared memory
  const int pt0 = b * NQ + a;   // point (a, b, c) at pt0 + c * NQ2
#pragma unroll
  for (int c = 0; c < NQ; ++c)
    s_ch[pt0 + c * NQ2] = s_ch[NQ3 + pt0 + c * NQ2] = s_ch[2 * NQ3 + pt0 + c * NQ2] = Ar::zero();
  for (int m = 0; m < 3; ++m) {
    __syncthreads();
    for (int q = threadIdx.x; q < NP3; q += blockDim.x) s_src[q] = Ar::ld(cv, (size_t)m * nL + eb + q);
    __syncthreads();
    T cf[NQ];
    to_gauss<Ar, NP, NQ>(s_src, s_t1, sI, P.Im, a, b, cf);
#pragma unroll
    for (int c = 0; c < NQ; ++c) {
      const int pt = pt0 + c * NQ2;
#pragma unroll
      for (int d = 0; d < 3; ++d)
        s_ch[d * NQ3 + pt] = Ar::mac(s_ch[d * NQ3 + pt], Ar::lg(G, (d * 3 + m) * NQ3 + c * NQ2), cf[c]);
    }
  }
  // 3. every advected component
  for (int comp = 0; comp < ncomp; ++comp) {
    __syncthreads();
    for (int q = threadIdx.x; q < NP3; q += blockDim.x) s_src[q] = Ar::ld(uv, (size_t)comp * nL + eb + q);
    __syncthreads();
    T uf[NQ];
    to_gauss<Ar, NP, NQ>(s_src, s_t1, sI, P.Im, a, b, uf);
#pragma unroll
    for (int c = 0; c < NQ; ++c) s_U[c * PS + b * RS + a] = uf[c];
    T conv[NQ];
    {
      T ut[NQ];
      eo_deriv<Ar, NP>(P, uf, ut);   // t-derivative along this thread's line
#pragma unroll
      for (int c = 0; c < NQ; ++c) conv[c] = Ar::mul(s_ch[2 * NQ3 + pt0 + c * NQ2], ut[c]);
    }
    __syncthreads();
    // r-derivative on the line (plane c = b, row j = a) -> s_R
    {
      T v[NQ], o[NQ];
      const int rb = a, rc = b;
#pragma unroll
      for (int m = 0; m < NQ; ++m) v[m] = s_U[rc * PS + rb * RS + m];
      eo_deriv<Ar, NP>(P, v, o);
#pragma unroll
      for (int m = 0; m < NQ; ++m) s_R[rc * PS + rb * RS + m] = o[m];
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NQ; ++c) conv[c] = Ar::mac(conv[c], s_ch[pt0 + c * NQ2], s_R[c * PS + b * RS + a]);
    __syncthreads();
    // s-derivative on the column (plane c = b, column i = a) -> s_R
    {
      T v[NQ], o[NQ];
      const int sa = a, sc = b;
#pragma unroll
      for (int m = 0; m < NQ; ++m) v[m] = s_U[sc * PS + m * RS + sa];
      eo_deriv<Ar, NP>(P, v, o);
#pragma unroll
      for (int m = 0; m < NQ; ++m) s_R[sc * PS + m * RS + sa] = o[m];
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NQ; ++c)
      conv[c] = Ar::norm(Ar::mac(conv[c], s_ch[NQ3 + pt0 + c * NQ2], s_R[c * PS + b * RS + a]));
    // back to the GLL points: t-pass from registers into v2[k][b][a] (s_U reused)
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      T acc = Ar::zero();
#pragma unroll
      for (int c = 0; c < NQ; ++c) acc = Ar::mac(acc, P.Im[c * NP + k], conv[c]);
      s_U[k * PS + b * RS + a] = Ar::norm(acc);
    }
    __syncthreads();
    // s-pass: v1[k][j][a] = sum_b I[b][j] v2[k][b][a] (threads with b < NP own j = b)
    if (b < NP) {
      T cb[NQ];   // column b of I
#pragma unroll
      for (int q = 0; q < NQ; ++q) cb[q] = sI[q * NP + b];
#pragma unroll 2
      for (int k = 0; k < NP; ++k) {
        T acc = Ar::zero();
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc = Ar::mac(acc, cb[q], s_U[k * PS + q * RS + a]);
        s_t1[(k * NP + b) * NQ + a] = Ar::norm(acc);
      }
    }
    __syncthreads();
    // r-pass: w[k][j][i] = sum_a I[a][i] v1[k][j][a] (threads (i, j) = (a, b) with a, b < NP)
    if (a < NP && b < NP) {
      typename Ar::S* out = wv + (size_t)comp * nL + eb;
      T ca[NQ];   // column a of I
#pragma unroll
      for (int q = 0; q < NQ; ++q) ca[q] = sI[q * NP + a];
#pragma unroll 2
      for (int k = 0; k < NP; ++k) {
        T acc = Ar::zero();
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc = Ar::mac(acc, ca[q], s_t1[(k * NP + b) * NQ + q]);
        Ar::st(out, (size_t)(k * NP + b) * NP + a, acc);
      }
    }
  }
}

// Cubature factors Gq[e][d][m][point] = w_q J_q dr_d/dx_m at the Gauss points:
// the coordinates (relative to the element's first node) interpolated and
// differentiated on the Gauss points, the 3x3 metric inverted by cofactors.
template <int NP>
__global__ void __launch_bounds__(AdvShape<NP>::T)
    k_cub_geom(int E, const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ z,
               const double* __restrict__ Im, const double* __restrict__ Dq, const double* __restrict__ wq,
               double* __restrict__ Gq, float* __restrict__ Gq32, int* bad) {
  constexpr int NQ = AdvShape<NP>::NQ, NP3 = NP * NP * NP, NQ2 = NQ * NQ, NQ3 = NQ2 * NQ;
  __shared__ double sI[NQ * NP];
  __shared__ double sD[NQ * NQ];
  __shared__ double s_src[NP3];
  __shared__ double s_t1[NP * NP * NQ];
  __shared__ double s_X[NQ3];
  const int e = blockIdx.x;
  const int a = threadIdx.x % NQ, b = threadIdx.x / NQ;
  load_ops<AdvPlain<double>, NP, NQ>(Im, Dq, sI, sD);
  const size_t eb = (size_t)e * NP3;
  double Jl[3][3][NQ];   // Jl[m][d][c] = dx_m / dr_d at Gauss point (a, b, c)
  const double* X[3] = {x, y, z};
  for (int m = 0; m < 3; ++m) {
    __syncthreads();
    const double x0 = X[m][eb];
    for (int q = threadIdx.x; q < NP3; q += blockDim.x) s_src[q] = X[m][eb + q] - x0;
    __syncthreads();
    double line[NQ];
    to_gauss<AdvPlain<double>, NP, NQ>(s_src, s_t1, sI, sI, a, b, line);
#pragma unroll
    for (int c = 0; c < NQ; ++c) s_X[(c * NQ + b) * NQ + a] = line[c];
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NQ; ++c) {
      double dr = 0, ds = 0, dt = 0;
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        dr = fma(sD[a * NQ + q], s_X[(c * NQ + b) * NQ + q], dr);
        ds = fma(sD[b * NQ + q], s_X[(c * NQ + q) * NQ + a], ds);
        dt = fma(sD[c * NQ + q], line[q], dt);
      }
      Jl[m][0][c] = dr;
      Jl[m][1][c] = ds;
      Jl[m][2][c] = dt;
    }
  }
#pragma unroll
  for (int c = 0; c < NQ; ++c) {
    double J[3][3];   // J[m][d] = dx_m / dr_d
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
      for (int d = 0; d < 3; ++d) J[m][d] = Jl[m][d][c];
    const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    if (!(det > 0.0)) atomicExch(bad, 1);
    // R[d][m] = det * dr_d/dx_m (the adjugate); w J dr_d/dx_m = w R[d][m]
    double R[3][3];
    R[0][0] = c00;
    R[1][0] = c01;
    R[2][0] = c02;
    R[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
    R[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
    R[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
    R[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
    R[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
    R[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    const double wgt = wq[a] * wq[b] * wq[c];
    const size_t pt = (size_t)e * 9 * NQ3 + (c * NQ + b) * NQ + a;
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const double v = wgt * R[d][m];
        Gq[pt + (d * 3 + m) * NQ3] = v;
        if (Gq32) Gq32[pt + (d * 3 + m) * NQ3] = (float)v;
      }
  }
}

template <int NP>
int cub_geom_launch(const Level& L, const double* Im, const double* Dq, const double* wq, double* Gq, float* Gq32,
                    int* bad, cudaStream_t s) {
  k_cub_geom<NP><<<L.E, AdvShape<NP>::T, 0, s>>>(L.E, L.x, L.y, L.z, Im, Dq, wq, Gq, Gq32, bad);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}

template <class Ar, int NP>
int advect_launch(const Level& L, const AdvData& A, const typename Ar::S* c, const typename Ar::S* u,
                  typename Ar::S* w, int ncomp, const typename Ar::G* Gq, const typename Ar::G* Im,
                  const typename Ar::G* Dq, cudaStream_t s) {
  constexpr int NQ = nq_of(NP), H = NQ / 2, N = NQ - 1;
  AdvOps<typename Ar::V, NP> P{};
  for (int q = 0; q < NQ * NP; ++q) P.Im[q] = Ar::host(A.hIm[q]);
  auto d = [&](int r, int q) { return A.hDq[r * NQ + q]; };
  for (int r = 0; r < H; ++r)
    for (int q = 0; q < H; ++q) {
      P.ep[r * H + q] = Ar::host(0.5 * (d(r, q) + d(r, N - q)));
      P.op[r * H + q] = Ar::host(0.5 * (d(r, q) - d(r, N - q)));
    }
  if (NQ % 2 == 1)
    for (int r = 0; r < H; ++r) {
      P.mc[r] = Ar::host(d(r, H));
      P.mr[r] = Ar::host(d(H, r));
    }
  constexpr size_t smem = advect_smem<Ar, NP>();
  static PerDevice<bool> attr;
  SEM_TRY(smem_attr_once(attr, (const void*)k_advect<Ar, NP>, smem));
  k_advect<Ar, NP><<<L.E, AdvShape<NP>::T, smem, s>>>(L.E, ncomp, L.nL, c, u, Gq, Im, Dq, w, P);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}

#define ADV_DISPATCH(NPV, CALL) \
  case NPV: return CALL;

#define GRID_LOOP_ADV(l, n) \
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < (n); l += (int64_t)gridDim.x * blockDim.x)

inline unsigned vgrid_adv(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (unsigned)b;
}

// m = B_L, the local GLL mass (component 6 of the geometric factors)
__global__ void k_mass_local(int64_t n, int np3, const double* __restrict__ G, double* __restrict__ m) {
  GRID_LOOP_ADV(l, n) {
    const int64_t e = l / np3;
    m[l] = G[(e * 7 + 6) * np3 + (l - e * np3)];
  }
}

// minv = 1 / (QQ^T B) from the gathered mass in m (in place), FP64 and FP32 copies
__global__ void k_minv(int64_t n, double* __restrict__ m, float* __restrict__ m32) {
  GRID_LOOP_ADV(l, n) {
    const double v = 1.0 / m[l];
    m[l] = v;
    m32[l] = (float)v;
  }
}

// c(t) = c0 + th (c1 - c0) over the three wind components
template <typename T>
__global__ void k_wind(int64_t n, const T* __restrict__ c0, const T* __restrict__ c1, T th, T* __restrict__ c) {
  GRID_LOOP_ADV(l, n) c[l] = c0[l] + th * (c1[l] - c0[l]);
}

// (hi, lo) FP32 split of FP64 values
__global__ void k_split_adv(int64_t n, const double* __restrict__ a, float2* __restrict__ b) {
  GRID_LOOP_ADV(q, n) {
    const ff v = ff_split(a[q]);
    b[q] = make_float2(v.h, v.l);
  }
}

// One RK4 stage on ncomp components: k = -minv z (z = QQ^T C w_stage);
// mode 0: acc = k, ws = w + cw k; mode 1: acc += 2k, ws = w + cw k; mode 2: w += cw (acc + k).
template <typename T>
__global__ void k_rk_stage(int64_t n, int64_t nL, const T* __restrict__ z, const T* __restrict__ minv,
                           T* __restrict__ w, T* __restrict__ ws, T* __restrict__ acc, T cw, int mode) {
  GRID_LOOP_ADV(q, n) {
    const T k = -minv[q % nL] * z[q];
    if (mode == 0) {
      acc[q] = k;
      ws[q] = w[q] + cw * k;
    } else if (mode == 1) {
      acc[q] += T(2) * k;
      ws[q] = w[q] + cw * k;
    } else {
      w[q] += cw * (acc[q] + k);
    }
  }
}

}  // namespace

// Build the cubature data of level 0 (Gauss rule, interpolation and derivative
// matrices, Gq in FP64 and FP32). Synchronous.
int advect_build(Ctx& C, cudaStream_t s) {
  Level& L = C.lev[0];
  if (C.adv.ready) return SEM_OK;
  if (L.N < 2 || L.N > 8) {
    set_detail("the dealiased advection operator is compiled for 2 <= N <= 8 (order %d)", L.N);
    return SEM_EINVAL;
  }
  const int NP = L.NP, NQ = nq_of(NP);
  std::vector<double> z(NQ), w(NQ), Im(NQ * NP), Dq(NQ * NQ);
  host_gauss(NQ, z.data(), w.data());
  host_interp(NP, L.xi, NQ, z.data(), Im.data());
  host_deriv(NQ, z.data(), Dq.data());
  std::vector<float> Im32(Im.begin(), Im.end()), Dq32(Dq.begin(), Dq.end());
  AdvData& A = C.adv;
  A.nq = NQ;
  for (size_t q = 0; q < Im.size(); ++q) A.hIm[q] = Im[q];
  for (size_t q = 0; q < Dq.size(); ++q) A.hDq[q] = Dq[q];
  const size_t ng = (size_t)L.E * 9 * NQ * NQ * NQ;
  auto dm = [&](void** p, size_t bytes) -> int {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      *p = nullptr;
      cudaGetLastError();
      set_detail("cudaMalloc of %zu bytes failed (advection cubature data)", bytes);
      return SEM_ENOMEM;
    }
    return SEM_OK;
  };
  SEM_TRY(dm((void**)&A.Gq, ng * 8));
  SEM_TRY(dm((void**)&A.Gq32, ng * 4));
  SEM_TRY(dm((void**)&A.Im, Im.size() * 8));
  SEM_TRY(dm((void**)&A.Dq, Dq.size() * 8));
  SEM_TRY(dm((void**)&A.wq, NQ * 8));
  SEM_TRY(dm((void**)&A.Im32, Im.size() * 4));
  SEM_TRY(dm((void**)&A.Dq32, Dq.size() * 4));
  SEM_CUDA_TRY(cudaMemcpyAsync(A.Im, Im.data(), Im.size() * 8, cudaMemcpyHostToDevice, s));
  SEM_CUDA_TRY(cudaMemcpyAsync(A.Dq, Dq.data(), Dq.size() * 8, cudaMemcpyHostToDevice, s));
  SEM_CUDA_TRY(cudaMemcpyAsync(A.wq, w.data(), NQ * 8, cudaMemcpyHostToDevice, s));
  SEM_CUDA_TRY(cudaMemcpyAsync(A.Im32, Im32.data(), Im32.size() * 4, cudaMemcpyHostToDevice, s));
  SEM_CUDA_TRY(cudaMemcpyAsync(A.Dq32, Dq32.data(), Dq32.size() * 4, cudaMemcpyHostToDevice, s));
  int* bad = nullptr;
  SEM_TRY(dm((void**)&bad, sizeof(int)));
  SEM_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), s));
  int rc = SEM_OK;
  switch (NP) {
    case 3: rc = cub_geom_launch<3>(L, A.Im, A.Dq, A.wq, A.Gq, A.Gq32, bad, s); break;
    case 4: rc = cub_geom_launch<4>(L, A.Im, A.Dq, A.wq, A.Gq, A.Gq32, bad, s); break;
    case 5: rc = cub_geom_launch<5>(L, A.Im, A.Dq, A.wq, A.Gq, A.Gq32, bad, s); break;
    case 6: rc = cub_geom_launch<6>(L, A.Im, A.Dq, A.wq, A.Gq, A.Gq32, bad, s); break;
    case 7: rc = cub_geom_launch<7>(L, A.Im, A.Dq, A.wq, A.Gq, A.Gq32, bad, s); break;
    case 8: rc = cub_geom_launch<8>(L, A.Im, A.Dq, A.wq, A.Gq, A.Gq32, bad, s); break;
    default: rc = cub_geom_launch<9>(L, A.Im, A.Dq, A.wq, A.Gq, A.Gq32, bad, s); break;
  }
  int h_bad = 0;
  if (rc == SEM_OK) {
    if (cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      set_detail("advection cubature setup failed: %s", cudaGetErrorString(cudaGetLastError()));
      rc = SEM_ECUDA;
    }
  }
  cudaFree(bad);
  if (rc != SEM_OK) return rc;
  if (h_bad) {
    set_detail("non-positive Jacobian at a Gauss point");
    return SEM_EMESH;
  }
  A.ready = true;
  return SEM_OK;
}

// The FP32-pair copies of the cubature factors and the 1-D matrices (first pair evaluation).
int advect_pairs_build(AdvData& A, const Level& L, cudaStream_t s) {
  if (A.Gq2) return SEM_OK;
  const int NQ = A.nq, NP = L.NP;
  const size_t ng = (size_t)L.E * 9 * NQ * NQ * NQ;
  float2 *g2 = nullptr, *i2 = nullptr, *d2 = nullptr;
  if (cudaMalloc((void**)&g2, ng * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&i2, (size_t)NQ * NP * sizeof(float2)) != cudaSuccess ||
      cudaMalloc((void**)&d2, (size_t)NQ * NQ * sizeof(float2)) != cudaSuccess) {
    cudaGetLastError();
    if (g2) cudaFree(g2);
    if (i2) cudaFree(i2);
    set_detail("cudaMalloc of %zu bytes failed (FP32-pair cubature factors)", ng * sizeof(float2));
    return SEM_ENOMEM;
  }
  k_split_adv<<<vgrid_adv((int64_t)ng), 256, 0, s>>>((int64_t)ng, A.Gq, g2);
  k_split_adv<<<1, 256, 0, s>>>((int64_t)NQ * NP, A.Im, i2);
  k_split_adv<<<1, 256, 0, s>>>((int64_t)NQ * NQ, A.Dq, d2);
  SEM_LAUNCH_CHECK();
  A.Gq2 = g2;
  A.Im2 = i2;
  A.Dq2 = d2;
  return SEM_OK;
}

void advect_free(AdvData& A) {
  void* ptrs[] = {A.Gq, A.Gq32, A.Gq2, A.Im, A.Dq, A.wq, A.Im32, A.Dq32, A.Im2, A.Dq2, A.minv, A.minv32, A.ws};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  A = AdvData();
}

int advect_apply(Ctx& C, int prec, const void* c, const void* u, void* w, int ncomp, cudaStream_t s) {
  const Level& L = C.lev[0];
  AdvData& A = C.adv;
  if (prec == SEM_FP64P) {
    SEM_TRY(advect_pairs_build(A, L, s));
    const double *cc = (const double*)c, *uu = (const double*)u;
    double* ww = (double*)w;
    switch (L.NP) {
      ADV_DISPATCH(3, (advect_launch<AdvPair, 3>(L, A, cc, uu, ww, ncomp, A.Gq2, A.Im2, A.Dq2, s)))
      ADV_DISPATCH(4, (advect_launch<AdvPair, 4>(L, A, cc, uu, ww, ncomp, A.Gq2, A.Im2, A.Dq2, s)))
      ADV_DISPATCH(5, (advect_launch<AdvPair, 5>(L, A, cc, uu, ww, ncomp, A.Gq2, A.Im2, A.Dq2, s)))
      ADV_DISPATCH(6, (advect_launch<AdvPair, 6>(L, A, cc, uu, ww, ncomp, A.Gq2, A.Im2, A.Dq2, s)))
      ADV_DISPATCH(7, (advect_launch<AdvPair, 7>(L, A, cc, uu, ww, ncomp, A.Gq2, A.Im2, A.Dq2, s)))
      ADV_DISPATCH(8, (advect_launch<AdvPair, 8>(L, A, cc, uu, ww, ncomp, A.Gq2, A.Im2, A.Dq2, s)))
      ADV_DISPATCH(9, (advect_launch<AdvPair, 9>(L, A, cc, uu, ww, ncomp, A.Gq2, A.Im2, A.Dq2, s)))
      default: break;
    }
  } else if (prec == SEM_FP64) {
    const double *cc = (const double*)c, *uu = (const double*)u;
    double* ww = (double*)w;
    switch (L.NP) {
      ADV_DISPATCH(3, (advect_launch<AdvPlain<double>, 3>(L, A, cc, uu, ww, ncomp, A.Gq, A.Im, A.Dq, s)))
      ADV_DISPATCH(4, (advect_launch<AdvPlain<double>, 4>(L, A, cc, uu, ww, ncomp, A.Gq, A.Im, A.Dq, s)))
      ADV_DISPATCH(5, (advect_launch<AdvPlain<double>, 5>(L, A, cc, uu, ww, ncomp, A.Gq, A.Im, A.Dq, s)))
      ADV_DISPATCH(6, (advect_launch<AdvPlain<double>, 6>(L, A, cc, uu, ww, ncomp, A.Gq, A.Im, A.Dq, s)))
      ADV_DISPATCH(7, (advect_launch<AdvPlain<double>, 7>(L, A, cc, uu, ww, ncomp, A.Gq, A.Im, A.Dq, s)))
      ADV_DISPATCH(8, (advect_launch<AdvPlain<double>, 8>(L, A, cc, uu, ww, ncomp, A.Gq, A.Im, A.Dq, s)))
      ADV_DISPATCH(9, (advect_launch<AdvPlain<double>, 9>(L, A, cc, uu, ww, ncomp, A.Gq, A.Im, A.Dq, s)))
      default: break;
    }
  } else {
    const float *cc = (const float*)c, *uu = (const float*)u;
    float* ww = (float*)w;
    switch (L.NP) {
      ADV_DISPATCH(3, (advect_launch<AdvPlain<float>, 3>(L, A, cc, uu, ww, ncomp, A.Gq32, A.Im32, A.Dq32, s)))
      ADV_DISPATCH(4, (advect_launch<AdvPlain<float>, 4>(L, A, cc, uu, ww, ncomp, A.Gq32, A.Im32, A.Dq32, s)))
      ADV_DISPATCH(5, (advect_launch<AdvPlain<float>, 5>(L, A, cc, uu, ww, ncomp, A.Gq32, A.Im32, A.Dq32, s)))
      ADV_DISPATCH(6, (advect_launch<AdvPlain<float>, 6>(L, A, cc, uu, ww, ncomp, A.Gq32, A.Im32, A.Dq32, s)))
      ADV_DISPATCH(7, (advect_launch<AdvPlain<float>, 7>(L, A, cc, uu, ww, ncomp, A.Gq32, A.Im32, A.Dq32, s)))
      ADV_DISPATCH(8, (advect_launch<AdvPlain<float>, 8>(L, A, cc, uu, ww, ncomp, A.Gq32, A.Im32, A.Dq32, s)))
      ADV_DISPATCH(9, (advect_launch<AdvPlain<float>, 9>(L, A, cc, uu, ww, ncomp, A.Gq32, A.Im32, A.Dq32, s)))
      default: break;
    }
  }
  set_detail("the dealiased advection operator is compiled for 2 <= N <= 8");
  return SEM_EINVAL;
}

// RK4 substeps of dw/dt = -M^-1 QQ^T C(c(t)) w (the hyperbolic subproblem of the
// characteristics scheme, Section 2.1 eq. hyp): c(t) linear between c0 at t0 and
// c1 at t1 (c1 null: frozen), nsub classical Runge-Kutta steps, w in place.
int char_advance(Ctx& C, int prec, const void* c0, const void* c1, void* w, int ncomp, double t0, double t1,
                 int nsub, cudaStream_t s) {
  const Level& L = C.lev[0];
  AdvData& A = C.adv;
  const int64_t nL = L.nL, n = (int64_t)ncomp * nL;
  const int vp = prec == SEM_FP32 ? SEM_FP32 : SEM_FP64;   // the vectors' type (FP64 with the pair operator)
  const size_t esz = vp == SEM_FP64 ? 8 : 4;
  if (!A.minv) {
    if (cudaMalloc(&A.minv, nL * 8) != cudaSuccess || cudaMalloc(&A.minv32, nL * 4) != cudaSuccess) {
      cudaGetLastError();
      set_detail("cudaMalloc of the inverse mass failed");
      return SEM_ENOMEM;
    }
    k_mass_local<<<vgrid_adv(nL), 256, 0, s>>>(nL, L.NP * L.NP * L.NP, L.G, A.minv);
    SEM_LAUNCH_CHECK();
    SEM_TRY(gs_apply(L, SEM_FP64, A.minv, false, s));
    k_minv<<<vgrid_adv(nL), 256, 0, s>>>(nL, A.minv, A.minv32);
    SEM_LAUNCH_CHECK();
  }
  const size_t need = (3 * (size_t)n + 3 * (size_t)nL) * esz;
  if (A.ws_bytes < need) {
    if (A.ws) cudaFree(A.ws);
    A.ws = nullptr;
    A.ws_bytes = 0;
    if (cudaMalloc(&A.ws, need) != cudaSuccess) {
      cudaGetLastError();
      set_detail("cudaMalloc of %zu bytes failed (characteristics workspace)", need);
      return SEM_ENOMEM;
    }
    A.ws_bytes = need;
  }
  char* base = static_cast<char*>(A.ws);
  void* zb = base;                       // QQ^T C w_stage
  void* wsb = base + n * esz;            // w_stage
  void* accb = base + 2 * n * esz;       // sum of the weighted stages
  void* cb = base + 3 * n * esz;         // c(t)
  const double h = (t1 - t0) / nsub;
  auto wind = [&](double t) -> const void* {
    if (!c1) return c0;
    const double th = (t - t0) / (t1 - t0);
    if (vp == SEM_FP64)
      k_wind<double><<<vgrid_adv(3 * nL), 256, 0, s>>>(3 * nL, (const double*)c0, (const double*)c1, th, (double*)cb);
    else
      k_wind<float><<<vgrid_adv(3 * nL), 256, 0, s>>>(3 * nL, (const float*)c0, (const float*)c1, (float)th,
                                                     (float*)cb);
    return cb;
  };
  auto eval = [&](double t, const void* win) -> int {   // z = QQ^T C(c(t)) win
    const void* c = wind(t);
    SEM_LAUNCH_CHECK();
    SEM_TRY(advect_apply(C, prec, c, win, zb, ncomp, s));
    for (int q = 0; q < ncomp; ++q) SEM_TRY(gs_apply(L, vp, static_cast<char*>(zb) + q * nL * esz, false, s));
    return SEM_OK;
  };
  auto stage = [&](double cw, int mode) -> int {
    if (vp == SEM_FP64)
      k_rk_stage<double><<<vgrid_adv(n), 256, 0, s>>>(n, nL, (const double*)zb, A.minv, (double*)w, (double*)wsb,
                                                      (double*)accb, cw, mode);
    else
      k_rk_stage<float><<<vgrid_adv(n), 256, 0, s>>>(n, nL, (const float*)zb, A.minv32, (float*)w, (float*)wsb,
                                                     (float*)accb, (float)cw, mode);
    SEM_LAUNCH_CHECK();
    return SEM_OK;
  };
  for (int q = 0; q < nsub; ++q) {
    const double t = t0 + q * h;
    SEM_TRY(eval(t, w));
    SEM_TRY(stage(0.5 * h, 0));
    SEM_TRY(eval(t + 0.5 * h, wsb));
    SEM_TRY(stage(0.5 * h, 1));
    SEM_TRY(eval(t + 0.5 * h, wsb));
    SEM_TRY(stage(h, 1));
    SEM_TRY(eval(t + h, wsb));
    SEM_TRY(stage(h / 6.0, 2));
  }
  return SEM_OK;
}

}  // namespace sem
