// FP64-accurate local operator w_L = A_L u_L evaluated with FP32 pair arithmetic.
//
// GB300 runs FP32 FMA about 70x faster than FP64 FMA, so the FP64 operator of
// eq. Ae is bound by the FP64 pipe by an order of magnitude over HBM. This
// kernel keeps every intermediate as an unevaluated sum of two floats
// (hi + lo, about 48 significant bits) and uses only FP32 instructions in the
// contractions:
//   TwoProduct (Dekker / FMA form):  p = a*b, e = fma(a, b, -p)      a*b = p + e exactly
//   TwoSum (Knuth):                  s = a+b, t = s-a, e = (a-(s-t)) + (b-t)   a+b = s + e exactly
// A multiply-accumulate acc += x*y of pairs adds TwoProduct(x.h, y.h) to acc.h
// with TwoSum and gathers every lower-order term (the two rounding errors and
// x.h*y.l + x.l*y.h) in acc.l. Inputs and outputs stay FP64 in memory; the
// geometric factors are stored pre-split as (hi, lo) float pairs (8 bytes, as
// many as FP64). Intrinsics with explicit rounding (__fadd_rn, __fmul_rn,
// __fmaf_rn) keep the compiler from contracting the error-free transforms.
// Exponent range is that of FP32: values must stay within ~1e-30..1e30.
#include "sem_internal.cuh"

namespace sem {

namespace {

struct ff {
  float h, l;
};

__device__ __forceinline__ ff split(double x) {
  const float h = __double2float_rn(x);
  const float l = __double2float_rn(x - (double)h);
  return {h, l};
}

__device__ __forceinline__ double join(ff a) { return (double)a.h + (double)a.l; }

// acc += x * y   (pairs)
__device__ __forceinline__ void mac(ff& acc, const ff x, const ff y) {
  const float p = __fmul_rn(x.h, y.h);
  const float e = __fmaf_rn(x.h, y.h, -p);
  const float s = __fadd_rn(acc.h, p);
  const float t = __fsub_rn(s, acc.h);
  const float err = __fadd_rn(__fsub_rn(acc.h, __fsub_rn(s, t)), __fsub_rn(p, t));
  float l = __fadd_rn(acc.l, err);
  l = __fadd_rn(l, e);
  l = __fmaf_rn(x.h, y.l, l);
  l = __fmaf_rn(x.l, y.h, l);
  acc.h = s;
  acc.l = l;
}

// x * y as an unnormalised pair
__device__ __forceinline__ ff mul(const ff x, const ff y) {
  const float p = __fmul_rn(x.h, y.h);
  float e = __fmaf_rn(x.h, y.h, -p);
  e = __fmaf_rn(x.h, y.l, e);
  e = __fmaf_rn(x.l, y.h, e);
  return {p, e};
}

// renormalise so that |l| <= ulp(h)/2 (TwoSum: valid whatever the magnitudes)
__device__ __forceinline__ ff norm(const ff a) {
  const float s = __fadd_rn(a.h, a.l);
  const float t = __fsub_rn(s, a.h);
  const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, t)), __fsub_rn(a.l, t));
  return {s, e};
}

template <int NP>
struct Pad2 {
  static constexpr int RS = (NP % 2 == 0) ? NP + 1 : NP;
  static constexpr int PS = NP * RS;
  static constexpr int ES = NP * PS;
};

template <int NP>
__host__ __device__ constexpr int pairs_epb() {
  int e = 256 / (NP * NP);
  if (e < 1) e = 1;
  while (e > 1 && (size_t)(3 * e * Pad2<NP>::ES + 4 * NP * NP) * 8 > 46 * 1024) --e;
  return e;
}

struct DPair {
  float h[144];
  float l[144];
};

template <int NP>
__global__ void __launch_bounds__(NP* NP* pairs_epb<NP>())
    k_ax_pairs(int E, const double* __restrict__ u, double* __restrict__ w, const float2* __restrict__ G,
               DPair Dm, ff h1, ff h2) {
  constexpr int EPB = pairs_epb<NP>();
  constexpr int NP2 = NP * NP, NP3 = NP2 * NP;
  constexpr int RS = Pad2<NP>::RS, PS = Pad2<NP>::PS, ES = Pad2<NP>::ES;
  __shared__ ff s_D[NP2];    // D[a][b] at a*NP + b
  __shared__ ff s_Dt[NP2];   // D[a][b] at b*NP + a
  __shared__ ff s_u[EPB * ES];
  __shared__ ff s_r[EPB * ES];
  __shared__ ff s_s[EPB * ES];
  const int tid = threadIdx.x;
  const int le = tid / NP2;
  const int ij = tid - le * NP2;
  const int j = ij / NP, i = ij - j * NP;
  const int e = blockIdx.x * EPB + le;
  for (int t = tid; t < NP2; t += blockDim.x) {
    const ff d = {Dm.h[t], Dm.l[t]};
    s_D[t] = d;
    s_Dt[(t % NP) * NP + t / NP] = d;
  }
  const bool active = e < E;
  ff* su = s_u + le * ES;
  ff* sr = s_r + le * ES;
  ff* ss = s_s + le * ES;
  const size_t ebase = (size_t)e * NP3;
  ff ru[NP];
  if (active) {
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      ru[k] = split(u[ebase + k * NP2 + ij]);
      su[k * PS + j * RS + i] = ru[k];
    }
  }
  __syncthreads();
  ff wt[NP];
  if (active) {
    const float2* Ge = G + (size_t)e * 7 * NP3 + ij;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      ff ur = {0.f, 0.f}, us = {0.f, 0.f}, ut = {0.f, 0.f};
#pragma unroll
      for (int l = 0; l < NP; ++l) {
        mac(ur, s_Dt[l * NP + i], su[k * PS + j * RS + l]);
        mac(us, s_Dt[l * NP + j], su[k * PS + l * RS + i]);
        mac(ut, ff{Dm.h[k * NP + l], Dm.l[k * NP + l]}, ru[l]);
      }
      const int o = k * NP2;
      float2 g;
      g = Ge[0 * NP3 + o]; const ff g11 = {g.x, g.y};
      g = Ge[1 * NP3 + o]; const ff g12 = {g.x, g.y};
      g = Ge[2 * NP3 + o]; const ff g13 = {g.x, g.y};
      g = Ge[3 * NP3 + o]; const ff g22 = {g.x, g.y};
      g = Ge[4 * NP3 + o]; const ff g23 = {g.x, g.y};
      g = Ge[5 * NP3 + o]; const ff g33 = {g.x, g.y};
      ur = norm(ur);
      us = norm(us);
      ut = norm(ut);
      ff a = mul(g11, ur);
      mac(a, g12, us);
      mac(a, g13, ut);
      ff b = mul(g12, ur);
      mac(b, g22, us);
      mac(b, g23, ut);
      ff c = mul(g13, ur);
      mac(c, g23, us);
      mac(c, g33, ut);
      sr[k * PS + j * RS + i] = norm(a);
      ss[k * PS + j * RS + i] = norm(b);
      wt[k] = norm(c);
    }
  }
  __syncthreads();
  if (active) {
    const float2* Be = G + (size_t)e * 7 * NP3 + 6 * NP3 + ij;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      ff acc = {0.f, 0.f};
#pragma unroll
      for (int l = 0; l < NP; ++l) {
        mac(acc, s_D[l * NP + i], sr[k * PS + j * RS + l]);
        mac(acc, s_D[l * NP + j], ss[k * PS + l * RS + i]);
        mac(acc, ff{Dm.h[l * NP + k], Dm.l[l * NP + k]}, wt[l]);
      }
      // w = h1 * (D^T G D u) + h2 * (B u)
      ff out = mul(h1, norm(acc));
      const float2 bb = Be[k * NP2];
      const ff bu = norm(mul(ff{bb.x, bb.y}, ru[k]));
      mac(out, h2, bu);
      w[ebase + k * NP2 + ij] = join(out);
    }
  }
}

__global__ void k_split_pairs(int64_t n, const double* __restrict__ G, float2* __restrict__ G2) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const double v = G[q];
    const float h = __double2float_rn(v);
    G2[q] = make_float2(h, __double2float_rn(v - (double)h));
  }
}

inline ff host_split(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}

}  // namespace

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

int ax_pairs_apply(const Level& L, const double* u, double* w, double h1, double h2, cudaStream_t s) {
  if (!L.G2) {
    set_detail("FP32-pair factors were not built");
    return SEM_EINVAL;
  }
  DPair Dm{};
  for (int t = 0; t < L.NP * L.NP; ++t) {
    const ff d = host_split(L.D.a[t]);
    Dm.h[t] = d.h;
    Dm.l[t] = d.l;
  }
  const ff fh1 = host_split(h1), fh2 = host_split(h2);
  switch (L.NP) {
#define CASE(NP)                                                                                 \
  case NP: {                                                                                     \
    constexpr int EPB = pairs_epb<NP>();                                                         \
    k_ax_pairs<NP><<<(L.E + EPB - 1) / EPB, NP * NP * EPB, 0, s>>>(L.E, u, w, L.G2, Dm, fh1, fh2); \
    SEM_LAUNCH_CHECK();                                                                          \
    return SEM_OK;                                                                               \
  }
    CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8) CASE(9) CASE(10) CASE(11) CASE(12)
#undef CASE
  }
  set_detail("order %d not compiled", L.N);
  return SEM_EINVAL;
}

}  // namespace sem
