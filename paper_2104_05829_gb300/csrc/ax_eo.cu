// FP64 local operator A^e = D^T h1 G D + h2 B (eq. Ae) with even-odd
// (centro-antisymmetric) 1-D contractions.
//
// On GB300 this kernel is bound by the FP64 pipe, so its speed is set by the
// number of FP64 instructions. D_hat on symmetric GLL nodes satisfies
// D[N-a][N-b] = -D[a][b] exactly (also in floating point: the nodes are
// exactly antisymmetric and P_N(-x) = (-1)^N P_N(x)). Writing a line v as
// s_b = v_b + v_{N-b}, d_b = v_b - v_{N-b} (b < H = (N+1)/2),
//   out_a = ev_a + od_a,  out_{N-a} = od_a - ev_a,
//   ev_a = sum_b E[a][b] s_b (+ D[a][m] v_m for the middle point m when N is even),
//   od_a = sum_b O[a][b] d_b,  E = (D[a][b] + D[a][N-b]) / 2, O = (D[a][b] - D[a][N-b]) / 2,
// and, when N is even, out_m = sum_b D[m][b] d_b. A line of N+1 outputs costs
// (N+1)^2/2 + 2(N+1) FP64 instructions instead of (N+1)^2 (48 instead of 64 at
// N = 7). The same holds for D^T.
//
// Every thread of the (N+1)^2 plane of an element transforms whole lines: its
// own t-line in registers, and one r-row and one s-column of shared memory.
// h1 multiplies the stiffness sum once per point instead of each factor.
#include "sem_internal.cuh"

namespace sem {

namespace {

struct EOMat {
  double ep[36];   // E[a][b], a, b < H
  double op[36];   // O[a][b]
  double mc[6];    // D[a][m]: the middle input's weight in ev_a (N even)
  double mr[6];    // D[m][b]: the middle output's weights on d_b (N even)
};

template <int NP>
struct Pad3 {
  // row stride NP+1 for even NP; plane stride chosen so that rows of
  // successive planes start on different banks
  static constexpr int RS = (NP % 2 == 0) ? NP + 1 : NP;
  static constexpr int PS = NP * RS + ((NP * RS) % 2 == 0 ? 2 : 1);
  static constexpr int ES = NP * PS;
};

template <int NP>
__host__ __device__ constexpr int eo_epb() {
  int e = 256 / (NP * NP);
  if (e < 1) e = 1;
  while (e > 1 && (size_t)(3 * e * Pad3<NP>::ES) * sizeof(double) > 46 * 1024) --e;
  return e;
}

template <int NP>
__device__ __forceinline__ void eo_apply(const EOMat& M, const double (&v)[NP], double (&out)[NP]) {
  constexpr int H = NP / 2, N = NP - 1;
  double s[H], d[H];
#pragma unroll
  for (int b = 0; b < H; ++b) {
    s[b] = v[b] + v[N - b];
    d[b] = v[b] - v[N - b];
  }
#pragma unroll
  for (int a = 0; a < H; ++a) {
    double ev = M.ep[a * H] * s[0];
    double od = M.op[a * H] * d[0];
#pragma unroll
    for (int b = 1; b < H; ++b) {
      ev = fma(M.ep[a * H + b], s[b], ev);
      od = fma(M.op[a * H + b], d[b], od);
    }
    if (NP % 2 == 1) ev = fma(M.mc[a], v[H], ev);
    out[a] = ev + od;
    out[N - a] = od - ev;
  }
  if (NP % 2 == 1) {
    double o = M.mr[0] * d[0];
#pragma unroll
    for (int b = 1; b < H; ++b) o = fma(M.mr[b], d[b], o);
    out[H] = o;
  }
}

template <int NP, bool VARH1>
__global__ void __launch_bounds__(NP* NP* eo_epb<NP>())
    k_ax_eo(int E, const double* __restrict__ u, double* __restrict__ w, const double* __restrict__ G, EOMat Df,
            EOMat Dt, double h1, double h2, const double* __restrict__ h1L, const double* skip) {
  constexpr int EPB = eo_epb<NP>();
  constexpr int NP2 = NP * NP, NP3 = NP2 * NP;
  constexpr int RS = Pad3<NP>::RS, PS = Pad3<NP>::PS, ES = Pad3<NP>::ES;
  if (skip && *skip != 0.0) return;
  __shared__ double s_a[EPB * ES];
  __shared__ double s_b[EPB * ES];
  __shared__ double s_c[EPB * ES];
  const int tid = threadIdx.x;
  const int le = tid / NP2;
  const int ij = tid - le * NP2;
  const int j = ij / NP, i = ij - j * NP;
  const int e = blockIdx.x * EPB + le;
  const bool active = e < E;
  double* A = s_a + le * ES;
  double* B = s_b + le * ES;
  double* Cc = s_c + le * ES;
  const size_t ebase = (size_t)e * NP3;

  // phase 0: the element into registers (own t-line) and shared memory
  double ru[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    ru[k] = active ? u[ebase + k * NP2 + ij] : 0.0;
    A[k * PS + j * RS + i] = ru[k];
  }
  __syncthreads();

  // phase 1: u_t (own line), u_r (row k = i, j), u_s (column k = i, i' = j)
  double ut[NP];
  eo_apply<NP>(Df, ru, ut);
  {
    double v[NP], o[NP];
#pragma unroll
    for (int l = 0; l < NP; ++l) v[l] = A[i * PS + j * RS + l];
    eo_apply<NP>(Df, v, o);
#pragma unroll
    for (int l = 0; l < NP; ++l) B[i * PS + j * RS + l] = o[l];
#pragma unroll
    for (int l = 0; l < NP; ++l) v[l] = A[i * PS + l * RS + j];
    eo_apply<NP>(Df, v, o);
#pragma unroll
    for (int l = 0; l < NP; ++l) Cc[i * PS + l * RS + j] = o[l];
  }
  __syncthreads();

  // phase 2: pointwise G-combine, in place
  if (active) {
    const double* Ge = G + (size_t)e * 7 * NP3 + ij;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int o = k * NP2;
      const double ur = B[k * PS + j * RS + i], us = Cc[k * PS + j * RS + i], uq = ut[k];
      const double g11 = Ge[0 * NP3 + o], g12 = Ge[1 * NP3 + o], g13 = Ge[2 * NP3 + o];
      const double g22 = Ge[3 * NP3 + o], g23 = Ge[4 * NP3 + o], g33 = Ge[5 * NP3 + o];
      double wr = fma(g13, uq, fma(g12, us, g11 * ur));
      double ws = fma(g23, uq, fma(g22, us, g12 * ur));
      double wt = fma(g33, uq, fma(g23, us, g13 * ur));
      if (VARH1) {
        const double hh = h1L[ebase + o + ij];
        wr *= hh;
        ws *= hh;
        wt *= hh;
      }
      B[k * PS + j * RS + i] = wr;
      Cc[k * PS + j * RS + i] = ws;
      ut[k] = wt;
    }
  }
  __syncthreads();

  // phase 3a: D_t^T on the own line, D_r^T on row (k = i, j) -> A
  double ot[NP];
  eo_apply<NP>(Dt, ut, ot);
  {
    double v[NP], o[NP];
#pragma unroll
    for (int l = 0; l < NP; ++l) v[l] = B[i * PS + j * RS + l];
    eo_apply<NP>(Dt, v, o);
#pragma unroll
    for (int l = 0; l < NP; ++l) A[i * PS + j * RS + l] = o[l];
  }
  __syncthreads();
  // phase 3b: D_s^T on column (k = i, i' = j) -> B
  {
    double v[NP], o[NP];
#pragma unroll
    for (int l = 0; l < NP; ++l) v[l] = Cc[i * PS + l * RS + j];
    eo_apply<NP>(Dt, v, o);
#pragma unroll
    for (int l = 0; l < NP; ++l) B[i * PS + l * RS + j] = o[l];
  }
  __syncthreads();

  // phase 4: w = h1 (D^T G D u) + h2 B u
  if (active) {
    const double* Be = G + (size_t)e * 7 * NP3 + 6 * NP3 + ij;
    const double hs = VARH1 ? 1.0 : h1;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const double st = A[k * PS + j * RS + i] + B[k * PS + j * RS + i] + ot[k];
      w[ebase + k * NP2 + ij] = fma(hs, st, h2 * Be[k * NP2] * ru[k]);
    }
  }
}

void make_eo(const double* D, int NP, bool transpose, EOMat& M) {
  const int H = NP / 2, N = NP - 1, m = NP / 2;
  auto at = [&](int a, int b) { return transpose ? D[b * NP + a] : D[a * NP + b]; };
  M = EOMat{};
  for (int a = 0; a < H; ++a)
    for (int b = 0; b < H; ++b) {
      M.ep[a * H + b] = 0.5 * (at(a, b) + at(a, N - b));
      M.op[a * H + b] = 0.5 * (at(a, b) - at(a, N - b));
    }
  if (NP % 2 == 1)
    for (int a = 0; a < H; ++a) {
      M.mc[a] = at(a, m);
      M.mr[a] = at(m, a);
    }
}

}  // namespace

// FP64 element operator with even-odd contractions (orders with N >= 1).
int ax_eo_apply(const Level& L, const double* u, double* w, double h1, double h2, const double* h1L,
                const double* skip, cudaStream_t s) {
  EOMat Df, Dt;
  make_eo(L.D.a, L.NP, false, Df);
  make_eo(L.D.a, L.NP, true, Dt);
  switch (L.NP) {
#define CASE(NP)                                                                                       \
  case NP: {                                                                                           \
    constexpr int EPB = eo_epb<NP>();                                                                  \
    const dim3 grid((L.E + EPB - 1) / EPB), block(NP * NP * EPB);                                      \
    if (h1L)                                                                                           \
      k_ax_eo<NP, true><<<grid, block, 0, s>>>(L.E, u, w, L.G, Df, Dt, h1, h2, h1L, skip);              \
    else                                                                                               \
      k_ax_eo<NP, false><<<grid, block, 0, s>>>(L.E, u, w, L.G, Df, Dt, h1, h2, nullptr, skip);         \
    SEM_LAUNCH_CHECK();                                                                                \
    return SEM_OK;                                                                                     \
  }
    CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10) CASE(11) CASE(12)
#undef CASE
  }
  set_detail("order %d not compiled", L.N);
  return SEM_EINVAL;
}

}  // namespace sem
