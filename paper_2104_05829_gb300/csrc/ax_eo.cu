// Local operator A^e = D^T h1 G D + h2 B (eq. Ae) with even-odd
// (centro-antisymmetric) 1-D contractions, in FP64 or in FP32-pair arithmetic.
//
// On GB300 both variants are bound by instruction throughput (the FP64 pipe,
// or the FP32 pipes for the pair arithmetic), so their speed is set by how
// many arithmetic instructions they issue. D_hat on symmetric GLL nodes
// satisfies D[N-a][N-b] = -D[a][b] exactly (also in floating point: the nodes
// are exactly antisymmetric and P_N(-x) = (-1)^N P_N(x)). Writing a line v as
// s_b = v_b + v_{N-b}, d_b = v_b - v_{N-b} (b < H = (N+1)/2),
//   out_a = ev_a + od_a,  out_{N-a} = od_a - ev_a,
//   ev_a = sum_b E[a][b] s_b (+ D[a][m] v_m for the middle point m when N is even),
//   od_a = sum_b O[a][b] d_b,  E = (D[a][b] + D[a][N-b]) / 2, O = (D[a][b] - D[a][N-b]) / 2,
// and, when N is even, out_m = sum_b D[m][b] d_b. A line of N+1 outputs costs
// (N+1)^2/2 multiply-adds and 2(N+1) additions instead of (N+1)^2 multiply-adds.
// The same holds for D^T.
//
// Every thread of the (N+1)^2 plane of an element transforms whole lines: its
// own t-line in registers, and one r-row and one s-column of shared memory.
// h1 multiplies the stiffness sum once per point instead of each factor.
//
// The pair variant keeps every value as an unevaluated sum of two floats
// (pairs.cuh); the factors are stored pre-split as float2 (hi, lo).
#include "pairs.cuh"
#include "sem_internal.cuh"

namespace sem {

namespace {

// ---- arithmetic back ends ------------------------------------------------------
struct ArF64 {
  static constexpr bool kPairs = false;
  using V = double;
  using GT = double;
  __device__ static V in(const double* u, size_t i) { return u[i]; }
  __device__ static void out(double* w, size_t i, V v) { w[i] = v; }
  __device__ static V gl(const GT* G, size_t i) { return G[i]; }
  __device__ static V zero() { return 0.0; }
  __device__ static V add(V a, V b) { return a + b; }
  __device__ static V sub(V a, V b) { return a - b; }
  __device__ static V add_u(V a, V b) { return a + b; }
  __device__ static V sub_u(V a, V b) { return a - b; }
  __device__ static V mul(V a, V b) { return a * b; }
  __device__ static V mac(V acc, V a, V b) { return fma(a, b, acc); }
  __device__ static V tidy(V a) { return a; }
  __device__ static V tidy_before_add(V a) { return a; }
  static V host(double x) { return x; }
};

struct ArPair {
  static constexpr bool kPairs = true;
  using V = ff;
  using GT = float2;
  __device__ static V in(const double* u, size_t i) { return ff_split(u[i]); }
  // the FP64 addition in ff_join rounds hi + lo correctly without renormalising first
  __device__ static void out(double* w, size_t i, V v) { w[i] = ff_join(v); }
  __device__ static V gl(const GT* G, size_t i) {
    const float2 g = G[i];
    return {g.x, g.y};
  }
  __device__ static V zero() { return {0.f, 0.f}; }
  __device__ static V add(V a, V b) { return ff_add(a, b); }
  __device__ static V sub(V a, V b) { return ff_sub(a, b); }
  // the additions inside the even-odd line transforms, whose results only enter further
  // error-free additions and products, skip the renormalisation
  __device__ static V add_u(V a, V b) { return ff_add_u(a, b); }
  __device__ static V sub_u(V a, V b) { return ff_sub_u(a, b); }
  __device__ static V mul(V a, V b) { return ff_mul(a, b); }
  __device__ static V mac(V acc, V a, V b) { return ff_mac(acc, a, b); }
  __device__ static V tidy(V a) { return ff_norm(a); }
  // values that next enter the error-free additions of eo_apply need no renormalising
  __device__ static V tidy_before_add(V a) { return a; }
  static V host(double x) { return ff_host_split(x); }
};

template <class Ar>
struct EOMat {
  typename Ar::V ep[36];   // E[a][b], a, b < H
  typename Ar::V op[36];   // O[a][b]
  typename Ar::V mc[6];    // D[a][m]: the middle input's weight in ev_a (N even)
  typename Ar::V mr[6];    // D[m][b]: the middle output's weights on d_b (N even)
};

template <int NP>
struct Pad3 {
  // row stride NP+1 for even NP; plane stride chosen so that rows of
  // successive planes start on different banks
  static constexpr int RS = (NP % 2 == 0) ? NP + 1 : NP;
  static constexpr int PS = NP * RS + ((NP * RS) % 2 == 0 ? 2 : 1);
  static constexpr int ES = NP * PS;
};

// Blocks per SM requested from the register allocator: at N = 7 four 192-thread blocks (at
// most 85 registers; five made the pair kernel spill and run slower). The pair kernel at other
// orders: three blocks, four at N = 9 (one 100-thread element per block there), against the
// register allocator's default of one or two blocks of up to 255 registers: at 16.8M points
// N = 3, 5, 11 took 0.390, 0.416, 1.347 ms with one block and 0.334, 0.371, 0.749 ms with three,
// and N = 8, 9, 10 took 0.518, 0.848, 0.625 ms with two blocks and 0.453, 0.634 (four),
// 0.492 ms; the FP64 kernel is bound by its pipe at any occupancy.
template <class Ar, int NP>
__host__ __device__ constexpr int eo_min_blocks() {
  return NP == 8 ? 4 : (Ar::kPairs ? (NP == 10 ? 4 : 3) : 1);
}

template <int NP>
__host__ __device__ constexpr int eo_epb() {
  int e = 256 / (NP * NP);
  if (e < 1) e = 1;
  while (e > 1 && (size_t)(3 * e * Pad3<NP>::ES) * 8 > 46 * 1024) --e;
  return e;
}

template <class Ar, int NP>
__device__ __forceinline__ void eo_apply(const EOMat<Ar>& M, const typename Ar::V (&v)[NP],
                                         typename Ar::V (&o)[NP]) {
  using V = typename Ar::V;
  constexpr int H = NP / 2, N = NP - 1;
  V s[H], d[H];
#pragma unroll
  for (int b = 0; b < H; ++b) {
    s[b] = Ar::add_u(v[b], v[N - b]);
    d[b] = Ar::sub_u(v[b], v[N - b]);
  }
#pragma unroll
  for (int a = 0; a < H; ++a) {
    V ev = Ar::mul(M.ep[a * H], s[0]);
    V od = Ar::mul(M.op[a * H], d[0]);
#pragma unroll
    for (int b = 1; b < H; ++b) {
      ev = Ar::mac(ev, M.ep[a * H + b], s[b]);
      od = Ar::mac(od, M.op[a * H + b], d[b]);
    }
    if (NP % 2 == 1) ev = Ar::mac(ev, M.mc[a], v[H]);
    o[a] = Ar::add_u(ev, od);
    o[N - a] = Ar::sub_u(od, ev);
  }
  if (NP % 2 == 1) {
    V m = Ar::mul(M.mr[0], d[0]);
#pragma unroll
    for (int b = 1; b < H; ++b) m = Ar::mac(m, M.mr[b], d[b]);
    o[H] = Ar::tidy(m);
  }
}

template <class Ar, int NP, bool VARH1>
__global__ void __launch_bounds__(NP* NP* eo_epb<NP>(), (eo_min_blocks<Ar, NP>()))
    k_ax_eo(int E, const double* __restrict__ u, double* __restrict__ w, const typename Ar::GT* __restrict__ G,
            EOMat<Ar> Df, EOMat<Ar> Dt, typename Ar::V h1, typename Ar::V h2, const double* __restrict__ h1L,
            const double* skip) {
  using V = typename Ar::V;
  constexpr int EPB = eo_epb<NP>();
  constexpr int NP2 = NP * NP, NP3 = NP2 * NP;
  constexpr int RS = Pad3<NP>::RS, PS = Pad3<NP>::PS, ES = Pad3<NP>::ES;
  if (skip && *skip != 0.0) return;
  __shared__ V s_a[EPB * ES];
  __shared__ V s_b[EPB * ES];
  __shared__ V s_c[EPB * ES];
  const int tid = threadIdx.x;
  const int le = tid / NP2;
  const int ij = tid - le * NP2;
  const int j = ij / NP, i = ij - j * NP;
  const int e = blockIdx.x * EPB + le;
  const bool active = e < E;
  V* A = s_a + le * ES;
  V* B = s_b + le * ES;
  V* Cc = s_c + le * ES;
  const size_t ebase = (size_t)e * NP3;

  // phase 0: the element into registers (own t-line) and shared memory
  V ru[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    ru[k] = active ? Ar::in(u, ebase + k * NP2 + ij) : Ar::zero();
    A[k * PS + j * RS + i] = ru[k];
  }
  __syncthreads();

  // phase 1: u_t (own line), u_r (row k = i, j), u_s (column k = i, i' = j)
  V ut[NP];
  eo_apply<Ar, NP>(Df, ru, ut);
  {
    V v[NP], o[NP];
#pragma unroll
    for (int l = 0; l < NP; ++l) v[l] = A[i * PS + j * RS + l];
    eo_apply<Ar, NP>(Df, v, o);
#pragma unroll
    for (int l = 0; l < NP; ++l) B[i * PS + j * RS + l] = o[l];
#pragma unroll
    for (int l = 0; l < NP; ++l) v[l] = A[i * PS + l * RS + j];
    eo_apply<Ar, NP>(Df, v, o);
#pragma unroll
    for (int l = 0; l < NP; ++l) Cc[i * PS + l * RS + j] = o[l];
  }
  __syncthreads();

  // phase 2: pointwise G-combine, in place
  if (active) {
    const typename Ar::GT* Ge = G + (size_t)e * 7 * NP3 + ij;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int o = k * NP2;
      const V ur = B[k * PS + j * RS + i], us = Cc[k * PS + j * RS + i], uq = ut[k];
      const V g11 = Ar::gl(Ge, 0 * NP3 + o), g12 = Ar::gl(Ge, 1 * NP3 + o), g13 = Ar::gl(Ge, 2 * NP3 + o);
      const V g22 = Ar::gl(Ge, 3 * NP3 + o), g23 = Ar::gl(Ge, 4 * NP3 + o), g33 = Ar::gl(Ge, 5 * NP3 + o);
      V wr = Ar::mac(Ar::mac(Ar::mul(g11, ur), g12, us), g13, uq);
      V ws = Ar::mac(Ar::mac(Ar::mul(g12, ur), g22, us), g23, uq);
      V wt = Ar::mac(Ar::mac(Ar::mul(g13, ur), g23, us), g33, uq);
      if (VARH1) {
        const V hh = Ar::in(h1L, ebase + o + ij);
        wr = Ar::mul(wr, hh);
        ws = Ar::mul(ws, hh);
        wt = Ar::mul(wt, hh);
      }
      B[k * PS + j * RS + i] = Ar::tidy_before_add(wr);
      Cc[k * PS + j * RS + i] = Ar::tidy_before_add(ws);
      ut[k] = Ar::tidy_before_add(wt);
    }
  }
  __syncthreads();

  // phase 3a: D_t^T on the own line, D_r^T on row (k = i, j) -> A
  V ot[NP];
  eo_apply<Ar, NP>(Dt, ut, ot);
  {
    V v[NP], o[NP];
#pragma unroll
    for (int l = 0; l < NP; ++l) v[l] = B[i * PS + j * RS + l];
    eo_apply<Ar, NP>(Dt, v, o);
#pragma unroll
    for (int l = 0; l < NP; ++l) A[i * PS + j * RS + l] = o[l];
  }
  __syncthreads();
  // phase 3b: D_s^T on column (k = i, i' = j) -> B
  {
    V v[NP], o[NP];
#pragma unroll
    for (int l = 0; l < NP; ++l) v[l] = Cc[i * PS + l * RS + j];
    eo_apply<Ar, NP>(Dt, v, o);
#pragma unroll
    for (int l = 0; l < NP; ++l) B[i * PS + l * RS + j] = o[l];
  }
  __syncthreads();

  // phase 4: w = h1 (D^T G D u) + h2 B u
  if (active) {
    const typename Ar::GT* Be = G + (size_t)e * 7 * NP3 + 6 * NP3 + ij;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const V st = Ar::add_u(Ar::add_u(A[k * PS + j * RS + i], B[k * PS + j * RS + i]), ot[k]);
      const V hb = Ar::mul(Ar::mul(h2, Ar::gl(Be, k * NP2)), ru[k]);
      Ar::out(w, ebase + k * NP2 + ij, VARH1 ? Ar::add(st, hb) : Ar::mac(hb, h1, st));
    }
  }
}

template <class Ar>
void make_eo(const double* D, int NP, bool transpose, EOMat<Ar>& M) {
  const int H = NP / 2, N = NP - 1, m = NP / 2;
  auto at = [&](int a, int b) { return transpose ? D[b * NP + a] : D[a * NP + b]; };
  for (int q = 0; q < 36; ++q) M.ep[q] = M.op[q] = Ar::host(0.0);
  for (int q = 0; q < 6; ++q) M.mc[q] = M.mr[q] = Ar::host(0.0);
  for (int a = 0; a < H; ++a)
    for (int b = 0; b < H; ++b) {
      M.ep[a * H + b] = Ar::host(0.5 * (at(a, b) + at(a, N - b)));
      M.op[a * H + b] = Ar::host(0.5 * (at(a, b) - at(a, N - b)));
    }
  if (NP % 2 == 1)
    for (int a = 0; a < H; ++a) {
      M.mc[a] = Ar::host(at(a, m));
      M.mr[a] = Ar::host(at(m, a));
    }
}

template <class Ar>
int eo_launch(const Level& L, const double* u, double* w, const typename Ar::GT* G, double h1, double h2,
              const double* h1L, const double* skip, cudaStream_t s) {
  EOMat<Ar> Df, Dt;
  make_eo<Ar>(L.D.a, L.NP, false, Df);
  make_eo<Ar>(L.D.a, L.NP, true, Dt);
  const typename Ar::V vh1 = Ar::host(h1), vh2 = Ar::host(h2);
  switch (L.NP) {
#define CASE(NP)                                                                                      \
  case NP: {                                                                                          \
    constexpr int EPB = eo_epb<NP>();                                                                 \
    const dim3 grid((L.E + EPB - 1) / EPB), block(NP * NP * EPB);                                     \
    if (h1L)                                                                                          \
      k_ax_eo<Ar, NP, true><<<grid, block, 0, s>>>(L.E, u, w, G, Df, Dt, vh1, vh2, h1L, skip);         \
    else                                                                                              \
      k_ax_eo<Ar, NP, false><<<grid, block, 0, s>>>(L.E, u, w, G, Df, Dt, vh1, vh2, nullptr, skip);    \
    SEM_LAUNCH_CHECK();                                                                               \
    return SEM_OK;                                                                                    \
  }
    CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10) CASE(11) CASE(12)
#undef CASE
  }
  set_detail("order %d not compiled", L.N);
  return SEM_EINVAL;
}

__global__ void k_split_pairs(int64_t n, const double* __restrict__ G, float2* __restrict__ G2) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const ff v = ff_split(G[q]);
    G2[q] = make_float2(v.h, v.l);
  }
}

}  // namespace

// FP64 element operator (even-odd contractions).
int ax_eo_apply(const Level& L, const double* u, double* w, double h1, double h2, const double* h1L,
                const double* skip, cudaStream_t s) {
  return eo_launch<ArF64>(L, u, w, L.G, h1, h2, h1L, skip, s);
}

// FP64-accurate element operator in FP32-pair arithmetic (scalar h1, or a nodal h1L, split
// into pairs as it is read).
int ax_pairs_apply(const Level& L, const double* u, double* w, double h1, double h2, const double* h1L,
                   cudaStream_t s) {
  if (!L.G2) {
    set_detail("FP32-pair factors were not built");
    return SEM_EINVAL;
  }
  return eo_launch<ArPair>(L, u, w, L.G2, h1, h2, h1L, nullptr, s);
}

// The element operator on elements [e0, e1) only (FP64 or FP32 pairs, scalar or nodal h1):
// the same kernels on a view of the level whose pointers start at element e0.
int ax_eo_apply_range(const Level& L, int e0, int e1, const double* u, double* w, double h1, double h2,
                      const double* h1L, bool pairs, cudaStream_t s) {
  if (e1 <= e0) return SEM_OK;
  const size_t off = (size_t)e0 * L.NP * L.NP * L.NP;
  Level V = L;
  V.E = e1 - e0;
  V.nL = (int64_t)V.E * L.NP * L.NP * L.NP;
  if (pairs) {
    if (!L.G2) {
      set_detail("FP32-pair factors not built");
      return SEM_EINVAL;
    }
    return eo_launch<ArPair>(V, u + off, w + off, L.G2 + 7 * off, h1, h2, h1L ? h1L + off : nullptr, nullptr, s);
  }
  return eo_launch<ArF64>(V, u + off, w + off, L.G + 7 * off, h1, h2, h1L ? h1L + off : nullptr, nullptr, s);
}

// (hi, lo) FP32 split of the FP64 factors for the pair kernel.
int pairs_build(Level& L, cudaStream_t s) {
  if (!L.G2) {
    cudaError_t e = cudaMalloc((void**)&L.G2, 7 * L.nL * sizeof(float2) + 16);
    if (e != cudaSuccess) {
      cudaGetLastError();
      L.G2 = nullptr;
      set_detail("cudaMalloc of the FP32-pair factors: %s", cudaGetErrorString(e));
      return SEM_ENOMEM;
    }
  }
  const int64_t n = 7 * L.nL;
  int64_t nb = (n + 255) / 256;
  if (nb > 152 * 32) nb = 152 * 32;
  k_split_pairs<<<(unsigned)nb, 256, 0, s>>>(n, L.G, L.G2);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}

}  // namespace sem
