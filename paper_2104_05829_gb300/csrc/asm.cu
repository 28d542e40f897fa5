// Overlapping additive Schwarz smoother with fast-diagonalisation (FDM) local
// solves, and its Chebyshev acceleration (CHEBY-ASM) -- Section 3.4: ASM on
// extended elements of (N+3)^3 points, local solves by tensor-product fast
// diagonalisation in about 12 E (N+3)^4 operations (Lynch, Rice and Thomas
// 1964; Deville, Fischer and Mund 2002; Lottes and Fischer 2005).
//
// Subdomain of element e: its (N+1)^3 nodes plus, across every face with a
// neighbour, the neighbour's layer of nodes one step inside from the shared
// face ("face layer"); together they sit in an (N+3)^3 box whose edge and
// corner strips stay zero. The local operator is the separable one of a box
// with the element's mean lengths L_r, L_s, L_t (neighbours taken with the
// same length): on the extended 1-D segment, the GLL stiffness and mass of
// the element and its neighbours restricted to the segment's nodes (Dirichlet
// one node beyond the overlap; a Dirichlet boundary side drops its boundary
// node, a Neumann side keeps it). With the 1-D generalised eigenpairs
// A S = B S Lam (S^T B S = I) of the reference segment (element length 2),
//   F_e = c (S_t x S_s x S_r) diag(1 / (h1 (l_r + l_s + l_t) + h2)) (S_t x S_s x S_r)^T,
//   l_d = (2/L_d)^2 lam_d,  c = (2/L_r)(2/L_s)(2/L_t).
// The smoother is z = W sum_e P_e^T F_e P_e r (P_e: gather to the box,
// P_e^T: add the own and face-layer slots back), masked; W = 1 / (number of
// subdomain slots holding the node). Kernels: k_asm_fdm (gather, six 1-D
// contractions with the scaling fused between the t passes, store of the own
// part to z and the face layers to a staging array), k_asm_pull (adds the
// staged face-layer values to the nodes they belong to, in a fixed order),
// then gs and the weighted Chebyshev update.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "reduce.cuh"
#include "sem_internal.cuh"

namespace sem {

namespace {

constexpr int SCH_NB = 0, SCH_DIR = 1, SCH_NEU = 2;

// ---------------------------------------------------------------------------
// host: symmetric eigenproblem (cyclic Jacobi rotations), 1-D reference data
// ---------------------------------------------------------------------------

// Eigen-decomposition of the symmetric n x n matrix a (row-major, destroyed):
// a = V diag(w) V^T, V column-major in v[col * n + row].
void jacobi_eig(int n, double* a, double* w, double* v) {
  for (int i = 0; i < n * n; ++i) v[i] = 0.0;
  for (int i = 0; i < n; ++i) v[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = 0; q < n; ++q) {
        tot += a[p * n + q] * a[p * n + q];
        if (p != q) off += a[p * n + q] * a[p * n + q];
      }
    if (off <= 1e-32 * tot) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = a[p * n + q];
        if (apq == 0.0) continue;
        const double theta = (a[q * n + q] - a[p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {   // columns p, q
          const double akp = a[k * n + p], akq = a[k * n + q];
          a[k * n + p] = c * akp - s * akq;
          a[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {   // rows p, q
          const double apk = a[p * n + k], aqk = a[q * n + k];
          a[p * n + k] = c * apk - s * aqk;
          a[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = v[p * n + k], vkq = v[q * n + k];
          v[p * n + k] = c * vkp - s * vkq;
          v[q * n + k] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < n; ++i) w[i] = a[i * n + i];
}

// Reference 1-D data of the extended segment for side types (left, right):
// S[slot * M + col] (M = N+3 slots, slot = extended index + 1) and lam[col].
void fdm_1d_host(int N, int left, int right, double* S, double* lam) {
  const int NP = N + 1, M = N + 3;
  double xi[16], rho[16], D[256];
  host_gll(N, xi, rho);
  host_dhat(N, xi, D);
  std::vector<double> K(NP * NP, 0.0);   // D^T diag(rho) D
  for (int a = 0; a < NP; ++a)
    for (int b = 0; b < NP; ++b) {
      double t = 0;
      for (int q = 0; q < NP; ++q) t += D[q * NP + a] * rho[q] * D[q * NP + b];
      K[a * NP + b] = t;
    }
  const int n = 3 * N + 1;
  std::vector<double> A(n * n, 0.0), B(n, 0.0);
  const bool present[3] = {left == SCH_NB, true, right == SCH_NB};
  for (int el = 0; el < 3; ++el) {
    if (!present[el]) continue;
    for (int a = 0; a < NP; ++a) {
      B[el * N + a] += rho[a];
      for (int b = 0; b < NP; ++b) A[(el * N + a) * n + el * N + b] += K[a * NP + b];
    }
  }
  std::vector<int> slots;
  for (int ext = -1; ext <= N + 1; ++ext) {
    if (ext == -1 && left != SCH_NB) continue;
    if (ext == 0 && left == SCH_DIR) continue;
    if (ext == N && right == SCH_DIR) continue;
    if (ext == N + 1 && right != SCH_NB) continue;
    slots.push_back(ext);
  }
  const int m = (int)slots.size();
  std::vector<double> C(m * m), w(m), V(m * m), isq(m);
  for (int a = 0; a < m; ++a) isq[a] = 1.0 / std::sqrt(B[N + slots[a]]);
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b) C[a * m + b] = isq[a] * A[(N + slots[a]) * n + N + slots[b]] * isq[b];
  jacobi_eig(m, C.data(), w.data(), V.data());
  for (int t = 0; t < M * M; ++t) S[t] = 0.0;
  for (int c = 0; c < M; ++c) lam[c] = 1.0;
  for (int c = 0; c < m; ++c) {
    lam[c] = w[c];
    for (int a = 0; a < m; ++a) S[(slots[a] + 1) * M + c] = isq[a] * V[c * m + a];
  }
}

// ---------------------------------------------------------------------------
// device
// ---------------------------------------------------------------------------

template <int NP>
struct AsmShape {
  static constexpr int M = NP + 2;
  static constexpr int M2 = M * M;
  static constexpr int RS = (M % 2 == 0) ? M + 1 : M;                 // odd row stride
  static constexpr int PS = ((RS * M) % 2 == 0) ? RS * M + 1 : RS * M;   // odd plane stride
  static constexpr int BS = PS * M;                                    // box stride
  static constexpr int MR = (M + 3) / 4 * 4;                           // row stride of S (16-byte rows)
  static constexpr int REF = M * MR + MR;                              // S and lam of one side combination
  static constexpr int LPT = (M % 2 == 0) ? 2 : 1;                     // box lines per thread
  static constexpr int TPE = M2 / LPT;                                 // threads per element
  static constexpr int EPB = (320 / TPE) > 0 ? (320 / TPE) : 1;        // elements per block
  static constexpr int THREADS = EPB * TPE;
};

// Blocks per SM requested from the register allocator: about 64 registers per
// thread in FP32 and 96 in FP64 (the 1-D contractions otherwise keep whole
// matrices in registers).
template <typename T, int NP>
__host__ __device__ constexpr int asm_min_blocks() {
  constexpr int warps = (AsmShape<NP>::THREADS + 31) / 32;
  constexpr int target = sizeof(T) == 4 ? 64 : 96;
  constexpr int mb = 65536 / (warps * 32 * target);
  return mb > 0 ? mb : 1;
}

// Elements' mean lengths along r, s, t (mean over the grid lines of the end-to-end distance).
__global__ void k_elem_lengths(int E, int NP, const double* __restrict__ x, const double* __restrict__ y,
                               const double* __restrict__ z, double* __restrict__ len, float* __restrict__ len32) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= (int64_t)E * 3) return;
  const int64_t e = q / 3;
  const int d = (int)(q - e * 3);
  const int N = NP - 1, NP3 = NP * NP * NP;
  const int64_t eb = e * NP3;
  double acc = 0;
  for (int u = 0; u < NP; ++u)
    for (int v = 0; v < NP; ++v) {
      int i0, j0, k0, i1, j1, k1;
      if (d == 0) { i0 = 0; i1 = N; j0 = j1 = u; k0 = k1 = v; }
      else if (d == 1) { j0 = 0; j1 = N; i0 = i1 = u; k0 = k1 = v; }
      else { k0 = 0; k1 = N; i0 = i1 = u; j0 = j1 = v; }
      const int64_t p0 = eb + (k0 * NP + j0) * NP + i0, p1 = eb + (k1 * NP + j1) * NP + i1;
      const double dx = x[p1] - x[p0], dy = y[p1] - y[p0], dz = z[p1] - z[p0];
      acc += sqrt(dx * dx + dy * dy + dz * dz);
    }
  len[q] = acc / (NP * NP);
  if (len32) len32[q] = (float)len[q];
}

// box slot of face-layer position (a, b) of face f
template <int NP>
__device__ __forceinline__ int layer_slot(int f, int a, int b) {
  using Sh = AsmShape<NP>;
  const int d = f >> 1, c = (f & 1) ? NP + 1 : 0;
  int ib, jb, kb;
  if (d == 0) { ib = c; jb = a + 1; kb = b + 1; }
  else if (d == 1) { ib = a + 1; jb = c; kb = b + 1; }
  else { ib = a + 1; jb = b + 1; kb = c; }
  return kb * Sh::PS + jb * Sh::RS + ib;
}

// quotient for the eigenvalue scaling: IEEE division in FP64, the fast single-precision
// division (about 2 ulp) in FP32, where the local solves are a smoother anyway
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }

// Row q of a matrix with row stride MR (a multiple of 4), loaded four entries at a time.
template <typename T, int M, int MR>
__device__ __forceinline__ void load_row(const T* __restrict__ row, T (&r)[MR]) {
#pragma unroll
  for (int c = 0; c < MR; c += 4) {
    if (sizeof(T) == 4) {
      const float4 v = *reinterpret_cast<const float4*>(row + c);
      r[c] = v.x; r[c + 1] = v.y; r[c + 2] = v.z; r[c + 3] = v.w;
    } else {
      const double2 v0 = *reinterpret_cast<const double2*>(row + c);
      const double2 v1 = *reinterpret_cast<const double2*>(row + c + 2);
      r[c] = v0.x; r[c + 1] = v0.y; r[c + 2] = v1.x; r[c + 3] = v1.y;
    }
  }
}

// Forward pass on L box lines (bases line[c], common stride st): out[c][a] =
// sum_m S[m][a] line_c[m], streaming row m of S (stride MR) once for all L lines.
template <typename T, int M, int MR, int L>
__device__ __forceinline__ void lines_fwd(const T* __restrict__ S, T* const (&line)[L], int st, T (&out)[L][M]) {
#pragma unroll
  for (int c = 0; c < L; ++c)
#pragma unroll
    for (int a = 0; a < M; ++a) out[c][a] = T(0);
#pragma unroll 2
  for (int m = 0; m < M; ++m) {
    T v[L];
#pragma unroll
    for (int c = 0; c < L; ++c) v[c] = line[c][m * st];
    T r[MR];
    load_row<T, M, MR>(S + m * MR, r);
#pragma unroll
    for (int c = 0; c < L; ++c)
#pragma unroll
      for (int a = 0; a < M; ++a) out[c][a] = fma(r[a], v[c], out[c][a]);
  }
}

// Backward pass: line_c[a] = sum_m S[a][m] in[c][m], written straight to shared memory.
template <typename T, int M, int MR, int L>
__device__ __forceinline__ void lines_bwd(const T* __restrict__ S, const T (&in)[L][M], T* const (&line)[L], int st) {
#pragma unroll 2
  for (int a = 0; a < M; ++a) {
    T r[MR];
    load_row<T, M, MR>(S + a * MR, r);
#pragma unroll
    for (int c = 0; c < L; ++c) {
      T acc = T(0);
#pragma unroll
      for (int m = 0; m < M; ++m) acc = fma(r[m], in[c][m], acc);
      line[c][a * st] = acc;
    }
  }
}

template <typename T, int NP>
__global__ void __launch_bounds__(AsmShape<NP>::THREADS, (asm_min_blocks<T, NP>()))
    k_asm_fdm(int E, const T* __restrict__ bv, const T* __restrict__ wv, const int32_t* __restrict__ layer,
              const uint8_t* __restrict__ bt, const T* __restrict__ len, const T* __restrict__ ref, T h1, T h2,
              T* __restrict__ z, T* __restrict__ zf) {
  using Sh = AsmShape<NP>;
  constexpr int M = Sh::M, RS = Sh::RS, PS = Sh::PS, EPB = Sh::EPB, LPT = Sh::LPT, TPE = Sh::TPE;
  constexpr int NP2 = NP * NP, NP3 = NP2 * NP;
  __shared__ __align__(16) T s_ref[9 * Sh::REF];
  __shared__ T s_box[EPB * Sh::BS];
  for (int q = threadIdx.x; q < 9 * Sh::REF; q += blockDim.x) s_ref[q] = ref[q];
  const int le = threadIdx.x / TPE;
  const int tq = threadIdx.x - le * TPE;
  const int e = blockIdx.x * EPB + le;
  const bool active = e < E;
  T* box = s_box + le * Sh::BS;
  for (int q = tq; q < Sh::BS; q += TPE) box[q] = T(0);
  __syncthreads();
  if (active) {
    // every load of this thread's box values (own points, then face-layer indices and
    // values) goes out before the first is used
    constexpr int NO = (NP3 + TPE - 1) / TPE, NF = (6 * NP2 + TPE - 1) / TPE;
    const size_t eb = (size_t)e * NP3;
    T ob[NO], ow[NO];
#pragma unroll
    for (int c = 0; c < NO; ++c) {
      const int q = tq + c * TPE;
      ob[c] = q < NP3 ? bv[eb + q] : T(0);
      ow[c] = (wv && q < NP3) ? wv[eb + q] : T(0);
    }
    const int32_t* lay = layer + (size_t)e * 6 * NP2;
    int32_t src[NF];
#pragma unroll
    for (int c = 0; c < NF; ++c) {
      const int q = tq + c * TPE;
      src[c] = q < 6 * NP2 ? lay[q] : -1;
    }
    T fb[NF], fw[NF];
#pragma unroll
    for (int c = 0; c < NF; ++c) {
      fb[c] = src[c] >= 0 ? bv[src[c]] : T(0);
      fw[c] = (wv && src[c] >= 0) ? wv[src[c]] : T(0);
    }
#pragma unroll
    for (int c = 0; c < NO; ++c) {
      const int q = tq + c * TPE;
      if (q < NP3) {
        const int k = q / NP2, j = (q / NP) % NP, i = q % NP;
        box[(k + 1) * PS + (j + 1) * RS + i + 1] = ob[c] - ow[c];
      }
    }
#pragma unroll
    for (int c = 0; c < NF; ++c) {
      const int q = tq + c * TPE;
      if (src[c] >= 0) {
        const int f = q / NP2, ab = q - f * NP2;
        box[layer_slot<NP>(f, ab / NP, ab % NP)] = fb[c] - fw[c];
      }
    }
  }
  __syncthreads();
  // this thread's lines: (p, q0 + c M / LPT), c < LPT
  const int p = tq % M, q0 = tq / M;
  int cr = 0, cs = 0, ct = 0;
  T sr = T(1), ss = T(1), st = T(1);
  if (active) {
    const uint8_t* b6 = bt + (size_t)e * 6;
    cr = 3 * b6[0] + b6[1];
    cs = 3 * b6[2] + b6[3];
    ct = 3 * b6[4] + b6[5];
    sr = T(2) / len[(size_t)e * 3 + 0];
    ss = T(2) / len[(size_t)e * 3 + 1];
    st = T(2) / len[(size_t)e * 3 + 2];
  }
  const T* Sr = s_ref + cr * Sh::REF;
  const T* Ss = s_ref + cs * Sh::REF;
  const T* St = s_ref + ct * Sh::REF;
  T v[LPT][M];
  T* ln[LPT];
  // forward r: lines along i at (j, k) = (p, q)
#pragma unroll
  for (int c = 0; c < LPT; ++c) ln[c] = box + (q0 + c * (M / LPT)) * PS + p * RS;
  lines_fwd<T, M, Sh::MR, LPT>(Sr, ln, 1, v);
#pragma unroll
  for (int c = 0; c < LPT; ++c)
#pragma unroll
    for (int m = 0; m < M; ++m) ln[c][m] = v[c][m];
  __syncthreads();
  // forward s: lines along j at (i, k) = (p, q)
#pragma unroll
  for (int c = 0; c < LPT; ++c) ln[c] = box + (q0 + c * (M / LPT)) * PS + p;
  lines_fwd<T, M, Sh::MR, LPT>(Ss, ln, RS, v);
#pragma unroll
  for (int c = 0; c < LPT; ++c)
#pragma unroll
    for (int m = 0; m < M; ++m) ln[c][m * RS] = v[c][m];
  __syncthreads();
  // t: forward, eigenvalue scaling, backward, on the lines along k at (i, j) = (p, q)
#pragma unroll
  for (int c = 0; c < LPT; ++c) ln[c] = box + (q0 + c * (M / LPT)) * RS + p;
  lines_fwd<T, M, Sh::MR, LPT>(St, ln, PS, v);
  {
    const T lr = Sr[M * Sh::MR + p] * sr * sr;
    const T cc = sr * ss * st;
#pragma unroll
    for (int c = 0; c < LPT; ++c) {
      const T ls = Ss[M * Sh::MR + q0 + c * (M / LPT)] * ss * ss;
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const T den = h1 * (lr + ls + St[M * Sh::MR + m] * st * st) + h2;
        v[c][m] = den != T(0) ? fdiv(cc * v[c][m], den) : T(0);
      }
    }
  }
  lines_bwd<T, M, Sh::MR, LPT>(St, v, ln, PS);
  __syncthreads();
  // backward s
#pragma unroll
  for (int c = 0; c < LPT; ++c) {
    ln[c] = box + (q0 + c * (M / LPT)) * PS + p;
#pragma unroll
    for (int m = 0; m < M; ++m) v[c][m] = ln[c][m * RS];
  }
  lines_bwd<T, M, Sh::MR, LPT>(Ss, v, ln, RS);
  __syncthreads();
  // backward r
#pragma unroll
  for (int c = 0; c < LPT; ++c) {
    ln[c] = box + (q0 + c * (M / LPT)) * PS + p * RS;
#pragma unroll
    for (int m = 0; m < M; ++m) v[c][m] = ln[c][m];
  }
  lines_bwd<T, M, Sh::MR, LPT>(Sr, v, ln, 1);
  __syncthreads();
  if (!active) return;
  const size_t eb = (size_t)e * NP3;
  for (int t = tq; t < NP3; t += TPE) {
    const int k = t / NP2, j = (t / NP) % NP, i = t % NP;
    z[eb + t] = box[(k + 1) * PS + (j + 1) * RS + i + 1];
  }
  T* zfe = zf + (size_t)e * 6 * NP2;
  for (int t = tq; t < 6 * NP2; t += TPE) {
    const int f = t / NP2, ab = t - f * NP2;
    zfe[t] = box[layer_slot<NP>(f, ab / NP, ab % NP)];
  }
}

// z[pts[q]] += sum of the staged face-layer values that belong to that local point
template <typename T>
__global__ void k_asm_pull(int64_t npts, const int32_t* __restrict__ pts, const int32_t* __restrict__ off,
                           const int32_t* __restrict__ src, const T* __restrict__ zf, T* __restrict__ z) {
  GRID_LOOP(q, npts) {
    const int32_t pnt = pts[q];
    T acc = z[pnt];
    for (int32_t o = off[q]; o < off[q + 1]; ++o) acc += zf[src[o]];
    z[pnt] = acc;
  }
}

template <typename T>
__global__ void k_mul_w(int64_t n, const T* __restrict__ w, T* __restrict__ z) {
  GRID_LOOP(l, n) z[l] *= w[l];
}

// Chebyshev step with the weighted Schwarz output z: d = c1 d + c2 W z; x = (x_zero ? 0 : x) + d
template <typename T>
__global__ void k_cheb_w(int64_t n, const T* __restrict__ z, const T* __restrict__ W, T* __restrict__ x,
                         T* __restrict__ d, T c1, T c2, int first, int x_zero) {
  GRID_LOOP(l, n) {
    const T dl = first ? c2 * (W[l] * z[l]) : c1 * d[l] + c2 * (W[l] * z[l]);
    d[l] = dl;
    x[l] = x_zero ? dl : x[l] + dl;
  }
}

__global__ void k_cnt_to_w(int64_t n, const double* __restrict__ cnt, const uint8_t* __restrict__ dmask,
                           double* __restrict__ w, float* __restrict__ w32) {
  GRID_LOOP(l, n) {
    const double v = (dmask[l] || !(cnt[l] > 0.0)) ? 0.0 : 1.0 / cnt[l];
    w[l] = v;
    if (w32) w32[l] = (float)v;
  }
}

// w -= (*a) v
__global__ void k_axpy_ds(int64_t n, double* __restrict__ w, const double* __restrict__ v, const double* a) {
  const double c = *a;
  GRID_LOOP(l, n) w[l] -= c * v[l];
}

__global__ void k_scale_host(int64_t n, const double* __restrict__ v, double* __restrict__ out, double c) {
  GRID_LOOP(l, n) out[l] = c * v[l];
}

inline unsigned vgrid2(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (unsigned)b;
}

template <typename T, int NP>
int launch_fdm(const Level& L, const T* b, const T* w, T* z, T* zf, double h1, double h2, cudaStream_t s) {
  using Sh = AsmShape<NP>;
  const T* len = std::is_same<T, double>::value ? (const T*)L.sch_len : (const T*)L.sch_len32;
  const T* ref = std::is_same<T, double>::value ? (const T*)L.sch_ref : (const T*)L.sch_ref32;
  const unsigned grid = (unsigned)((L.E + Sh::EPB - 1) / Sh::EPB);
  k_asm_fdm<T, NP><<<grid, Sh::THREADS, 0, s>>>(L.E, b, w, L.sch_layer, L.sch_bt, len, ref, (T)h1, (T)h2, z, zf);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}

template <typename T>
int dispatch_fdm(const Level& L, const T* b, const T* w, T* z, T* zf, double h1, double h2, cudaStream_t s) {
  switch (L.NP) {
    case 3: return launch_fdm<T, 3>(L, b, w, z, zf, h1, h2, s);
    case 4: return launch_fdm<T, 4>(L, b, w, z, zf, h1, h2, s);
    case 5: return launch_fdm<T, 5>(L, b, w, z, zf, h1, h2, s);
    case 6: return launch_fdm<T, 6>(L, b, w, z, zf, h1, h2, s);
    case 7: return launch_fdm<T, 7>(L, b, w, z, zf, h1, h2, s);
    case 8: return launch_fdm<T, 8>(L, b, w, z, zf, h1, h2, s);
    case 9: return launch_fdm<T, 9>(L, b, w, z, zf, h1, h2, s);
    case 10: return launch_fdm<T, 10>(L, b, w, z, zf, h1, h2, s);
    case 11: return launch_fdm<T, 11>(L, b, w, z, zf, h1, h2, s);
    case 12: return launch_fdm<T, 12>(L, b, w, z, zf, h1, h2, s);
    default:
      set_detail("the Schwarz smoother needs 2 <= N <= 11 (level order %d)", L.N);
      return SEM_EINVAL;
  }
}

template <typename T>
int dmalloc_n(T** p, size_t count) {
  if (cudaMalloc((void**)p, count * sizeof(T) + 16) != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    set_detail("cudaMalloc of %zu bytes failed (Schwarz smoother)", count * sizeof(T));
    return SEM_ENOMEM;
  }
  return SEM_OK;
}

}  // namespace

// Build the Schwarz data of level L (face-layer maps, side types, lengths,
// reference 1-D data, weights, pull lists). Synchronous; host work O(nL).
int schwarz_build(Ctx& C, Level& L, cudaStream_t s) {
  if (L.sch_ready) return SEM_OK;
  if (L.N < 2 || L.N > 11) {
    set_detail("the Schwarz smoother needs 2 <= N <= 11 (level order %d)", L.N);
    return SEM_EINVAL;
  }
  const int N = L.N, NP = L.NP, NP2 = NP * NP, NP3 = NP2 * NP, M = N + 3;
  const int64_t E = L.E, nL = L.nL;
  std::vector<int32_t> node(nL);
  std::vector<uint8_t> dmask(nL);
  SEM_CUDA_TRY(cudaMemcpyAsync(node.data(), L.node, nL * 4, cudaMemcpyDeviceToHost, s));
  SEM_CUDA_TRY(cudaMemcpyAsync(dmask.data(), L.dmask, nL, cudaMemcpyDeviceToHost, s));
  SEM_CUDA_TRY(cudaStreamSynchronize(s));
  const int64_t nG = L.nG;
  // holders of every unique node (local indices, ascending)
  std::vector<int64_t> hoff(nG + 1, 0);
  for (int64_t l = 0; l < nL; ++l) ++hoff[node[l] + 1];
  for (int64_t g = 0; g < nG; ++g) hoff[g + 1] += hoff[g];
  std::vector<int64_t> hidx(nL), fill(hoff.begin(), hoff.end() - 1);
  for (int64_t l = 0; l < nL; ++l) hidx[fill[node[l]]++] = l;
  auto face_local = [&](int f, int a, int b) {   // local (i, j, k) offset in the element
    const int d = f >> 1, c = (f & 1) ? N : 0;
    int i, j, k;
    if (d == 0) { i = c; j = a; k = b; }
    else if (d == 1) { i = a; j = c; k = b; }
    else { i = a; j = b; k = c; }
    return (k * NP + j) * NP + i;
  };
  auto copy_in = [&](int64_t g, int64_t elem) -> int64_t {
    for (int64_t o = hoff[g]; o < hoff[g + 1]; ++o)
      if (hidx[o] / NP3 == elem) return hidx[o];
    return -1;
  };
  std::vector<int32_t> layer((size_t)E * 6 * NP2, -1);
  std::vector<uint8_t> bt((size_t)E * 6, SCH_NEU);
  std::vector<double> cnt(nL, 1.0);
  for (int64_t e = 0; e < E; ++e) {
    for (int f = 0; f < 6; ++f) {
      const int64_t centre = e * NP3 + face_local(f, 1, 1);
      const int64_t g = node[centre];
      int64_t e2 = -1;
      for (int64_t o = hoff[g]; o < hoff[g + 1]; ++o)
        if (hidx[o] / NP3 != e) {
          e2 = hidx[o] / NP3;
          break;
        }
      if (e2 < 0) {
        bt[e * 6 + f] = dmask[centre] ? SCH_DIR : SCH_NEU;
        continue;
      }
      bt[e * 6 + f] = SCH_NB;
      // the face of e2 on which the shared face lies: the index that is 0 or N at three of its corners
      int pos[3][3];
      const int corners[3][2] = {{0, 0}, {N, 0}, {0, N}};
      for (int c = 0; c < 3; ++c) {
        const int64_t lc = copy_in(node[e * NP3 + face_local(f, corners[c][0], corners[c][1])], e2);
        if (lc < 0) {
          set_detail("non-conforming face between elements %lld and %lld", (long long)e, (long long)e2);
          return SEM_EINVAL;
        }
        const int loc = (int)(lc - e2 * NP3);
        pos[c][0] = loc % NP;
        pos[c][1] = (loc / NP) % NP;
        pos[c][2] = loc / NP2;
      }
      int ax = -1;
      for (int d = 0; d < 3 && ax < 0; ++d)
        if (pos[0][d] == pos[1][d] && pos[0][d] == pos[2][d] && (pos[0][d] == 0 || pos[0][d] == N)) ax = d;
      if (ax < 0) {
        set_detail("non-conforming face between elements %lld and %lld", (long long)e, (long long)e2);
        return SEM_EINVAL;
      }
      const int inward = pos[0][ax] == 0 ? 1 : N - 1;
      for (int a = 0; a < NP; ++a)
        for (int b = 0; b < NP; ++b) {
          const int64_t lc = copy_in(node[e * NP3 + face_local(f, a, b)], e2);
          if (lc < 0) {
            set_detail("non-conforming face between elements %lld and %lld", (long long)e, (long long)e2);
            return SEM_EINVAL;
          }
          const int loc = (int)(lc - e2 * NP3);
          int ijk[3] = {loc % NP, (loc / NP) % NP, loc / NP2};
          ijk[ax] = inward;
          const int64_t src = e2 * NP3 + (ijk[2] * NP + ijk[1]) * NP + ijk[0];
          layer[((size_t)e * 6 + f) * NP2 + a * NP + b] = (int32_t)src;
          cnt[src] += 1.0;
        }
    }
  }
  // pull lists: for every local point, the staged slots that belong to it (slot order)
  std::vector<int32_t> nper(nL, 0);
  for (size_t t = 0; t < layer.size(); ++t)
    if (layer[t] >= 0) ++nper[layer[t]];
  std::vector<int32_t> pts, poff(1, 0), psrc;
  std::vector<int64_t> first(nL, -1);
  for (int64_t l = 0; l < nL; ++l)
    if (nper[l] > 0) {
      first[l] = (int64_t)pts.size();
      pts.push_back((int32_t)l);
      poff.push_back(poff.back() + nper[l]);
    }
  psrc.resize(poff.back());
  std::vector<int32_t> pfill(poff.begin(), poff.end() - 1);
  for (size_t t = 0; t < layer.size(); ++t)
    if (layer[t] >= 0) psrc[pfill[first[layer[t]]]++] = (int32_t)t;
  // reference 1-D data for the nine side combinations
  // packed per combination as S rows of stride MR (a multiple of 4), then lam
  const int MR = (M + 3) / 4 * 4, REF = M * MR + MR;
  std::vector<double> ref(9 * REF, 0.0);
  std::vector<float> ref32(ref.size());
  for (int lt = 0; lt < 3; ++lt)
    for (int rt = 0; rt < 3; ++rt) {
      std::vector<double> S(M * M), lam(M);
      fdm_1d_host(N, lt, rt, S.data(), lam.data());
      double* r0 = ref.data() + (3 * lt + rt) * REF;
      for (int a = 0; a < M; ++a)
        for (int c = 0; c < M; ++c) r0[a * MR + c] = S[a * M + c];
      for (int c = 0; c < M; ++c) r0[M * MR + c] = lam[c];
    }
  for (size_t t = 0; t < ref.size(); ++t) ref32[t] = (float)ref[t];
  // device copies
  const bool f32 = L.G32 != nullptr || L.G16 != nullptr;
  SEM_TRY(dmalloc_n(&L.sch_layer, layer.size()));
  SEM_TRY(dmalloc_n(&L.sch_bt, bt.size()));
  SEM_TRY(dmalloc_n(&L.sch_len, (size_t)E * 3));
  SEM_TRY(dmalloc_n(&L.sch_ref, ref.size()));
  SEM_TRY(dmalloc_n(&L.sch_w, (size_t)nL));
  SEM_TRY(dmalloc_n(&L.sch_zf, layer.size()));
  SEM_TRY(dmalloc_n(&L.sch_pts, pts.size()));
  SEM_TRY(dmalloc_n(&L.sch_poff, poff.size()));
  SEM_TRY(dmalloc_n(&L.sch_psrc, psrc.size()));
  if (f32) {
    SEM_TRY(dmalloc_n(&L.sch_len32, (size_t)E * 3));
    SEM_TRY(dmalloc_n(&L.sch_ref32, ref32.size()));
    SEM_TRY(dmalloc_n(&L.sch_w32, (size_t)nL));
    SEM_TRY(dmalloc_n(&L.sch_zf32, layer.size()));
  }
  L.sch_npts = (int64_t)pts.size();
  SEM_CUDA_TRY(cudaMemcpyAsync(L.sch_layer, layer.data(), layer.size() * 4, cudaMemcpyHostToDevice, s));
  SEM_CUDA_TRY(cudaMemcpyAsync(L.sch_bt, bt.data(), bt.size(), cudaMemcpyHostToDevice, s));
  SEM_CUDA_TRY(cudaMemcpyAsync(L.sch_ref, ref.data(), ref.size() * 8, cudaMemcpyHostToDevice, s));
  SEM_CUDA_TRY(cudaMemcpyAsync(L.sch_pts, pts.data(), pts.size() * 4, cudaMemcpyHostToDevice, s));
  SEM_CUDA_TRY(cudaMemcpyAsync(L.sch_poff, poff.data(), poff.size() * 4, cudaMemcpyHostToDevice, s));
  SEM_CUDA_TRY(cudaMemcpyAsync(L.sch_psrc, psrc.data(), psrc.size() * 4, cudaMemcpyHostToDevice, s));
  if (f32) SEM_CUDA_TRY(cudaMemcpyAsync(L.sch_ref32, ref32.data(), ref32.size() * 4, cudaMemcpyHostToDevice, s));
  k_elem_lengths<<<(unsigned)((E * 3 + 255) / 256), 256, 0, s>>>((int)E, NP, L.x, L.y, L.z, L.sch_len,
                                                                   f32 ? L.sch_len32 : nullptr);
  SEM_LAUNCH_CHECK();
  // weights: per-point counts summed over the copies of each node, inverted, 0 at Dirichlet nodes
  double* dcnt = nullptr;
  SEM_TRY(dmalloc_n(&dcnt, (size_t)nL));
  SEM_CUDA_TRY(cudaMemcpyAsync(dcnt, cnt.data(), nL * 8, cudaMemcpyHostToDevice, s));
  int rc = gs_apply(L, SEM_FP64, dcnt, false, s);
  if (rc == SEM_OK) {
    k_cnt_to_w<<<vgrid2(nL), 256, 0, s>>>(nL, dcnt, L.dmask, L.sch_w, f32 ? L.sch_w32 : nullptr);
    if (cudaGetLastError() != cudaSuccess) rc = SEM_ECUDA;
  }
  cudaError_t e1 = cudaStreamSynchronize(s);
  cudaFree(dcnt);
  if (rc != SEM_OK) return rc;
  if (e1 != cudaSuccess) {
    set_detail("schwarz_build: %s", cudaGetErrorString(e1));
    return SEM_ECUDA;
  }
  L.sch_ready = true;
  return SEM_OK;
}

// z = sum_e P_e^T F_e P_e (b - w) on level L, gathered over copies and masked
// (no weight). w may be null (r = b). prec: SEM_FP64 (double) or FP32 (float vectors).
int asm_sum(const Level& L, int prec, const void* b, const void* w, void* z, double h1, double h2, cudaStream_t s) {
  if (!L.sch_ready) {
    set_detail("Schwarz data of level order %d not built", L.N);
    return SEM_EINVAL;
  }
  if (prec == SEM_FP64) {
    SEM_TRY(dispatch_fdm<double>(L, (const double*)b, (const double*)w, (double*)z, L.sch_zf, h1, h2, s));
    k_asm_pull<double><<<vgrid2(L.sch_npts), 256, 0, s>>>(L.sch_npts, L.sch_pts, L.sch_poff, L.sch_psrc, L.sch_zf,
                                                          (double*)z);
  } else {
    if (!L.sch_ref32) {
      set_detail("FP32 Schwarz data not built (no FP32 factor copies)");
      return SEM_EINVAL;
    }
    SEM_TRY(dispatch_fdm<float>(L, (const float*)b, (const float*)w, (float*)z, L.sch_zf32, h1, h2, s));
    k_asm_pull<float><<<vgrid2(L.sch_npts), 256, 0, s>>>(L.sch_npts, L.sch_pts, L.sch_poff, L.sch_psrc, L.sch_zf32,
                                                         (float*)z);
  }
  SEM_LAUNCH_CHECK();
  return gs_apply(L, prec, z, true, s);
}

int asm_weight(const Level& L, int prec, void* z, cudaStream_t s) {
  if (prec == SEM_FP64) k_mul_w<double><<<vgrid2(L.nL), 256, 0, s>>>(L.nL, L.sch_w, (double*)z);
  else k_mul_w<float><<<vgrid2(L.nL), 256, 0, s>>>(L.nL, L.sch_w32, (float*)z);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}

int cheb_w_update(const Level& L, int prec, const void* z, void* x, void* d, double c1, double c2, bool first,
                  bool x_zero, cudaStream_t s) {
  if (prec == SEM_FP64)
    k_cheb_w<double><<<vgrid2(L.nL), 256, 0, s>>>(L.nL, (const double*)z, L.sch_w, (double*)x, (double*)d, c1, c2,
                                                  first ? 1 : 0, x_zero ? 1 : 0);
  else
    k_cheb_w<float><<<vgrid2(L.nL), 256, 0, s>>>(L.nL, (const float*)z, L.sch_w32, (float*)x, (float*)d, (float)c1,
                                                 (float)c2, first ? 1 : 0, x_zero ? 1 : 0);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}

// Upper estimate of lambda_max(M A) for the weighted Schwarz M on level l:
// `steps` Arnoldi steps (modified Gram-Schmidt, unique-node inner products) from
// the seeded start vector in v0, then the largest eigenvalue of the symmetric
// part of the Hessenberg matrix. FP64 throughout. Synchronous.
int arnoldi_lmax_asm(Ctx& C, int l, double h1, double h2, const double* v0, int steps, cudaStream_t s,
                     double* lam) {
  Level& L = C.lev[l];
  const int64_t n = L.nL;
  std::vector<double> H((size_t)(steps + 1) * steps, 0.0);
  double* V = nullptr;
  double* dh = nullptr;
  SEM_TRY(dmalloc_n(&V, (size_t)(steps + 1) * n));
  int rc = dmalloc_n(&dh, (size_t)(steps + 2));
  auto body = [&]() -> int {
    double* w = L.vw;
    double* t = L.vd;
    SEM_TRY(dot_owner(C, L, SEM_FP64, v0, v0, dh, s));
    double nn = 0;
    SEM_CUDA_TRY(cudaMemcpyAsync(&nn, dh, 8, cudaMemcpyDeviceToHost, s));
    SEM_CUDA_TRY(cudaStreamSynchronize(s));
    if (!(nn > 0.0)) {
      set_detail("Arnoldi start vector is zero on level %d", l);
      return SEM_EBREAKDOWN;
    }
    k_scale_host<<<vgrid2(n), 256, 0, s>>>(n, v0, V, 1.0 / std::sqrt(nn));
    SEM_LAUNCH_CHECK();
    int k = steps;
    for (int j = 0; j < steps; ++j) {
      const double* vj = V + (size_t)j * n;
      SEM_TRY(ax_apply(L, SEM_FP64, vj, t, h1, h2, nullptr, s));
      SEM_TRY(gs_apply(L, SEM_FP64, t, true, s));
      SEM_TRY(asm_sum(L, SEM_FP64, t, nullptr, w, h1, h2, s));
      SEM_TRY(asm_weight(L, SEM_FP64, w, s));
      for (int i = 0; i <= j; ++i) {
        SEM_TRY(dot_owner(C, L, SEM_FP64, V + (size_t)i * n, w, dh + i, s));
        k_axpy_ds<<<vgrid2(n), 256, 0, s>>>(n, w, V + (size_t)i * n, dh + i);
        SEM_LAUNCH_CHECK();
      }
      SEM_TRY(dot_owner(C, L, SEM_FP64, w, w, dh + j + 1, s));
      std::vector<double> col(j + 2);
      SEM_CUDA_TRY(cudaMemcpyAsync(col.data(), dh, (j + 2) * 8, cudaMemcpyDeviceToHost, s));
      SEM_CUDA_TRY(cudaStreamSynchronize(s));
      for (int i = 0; i <= j; ++i) H[(size_t)i * steps + j] = col[i];
      const double hn = std::sqrt(col[j + 1]);
      H[(size_t)(j + 1) * steps + j] = hn;
      if (!(hn > 0.0)) {
        k = j + 1;
        break;
      }
      k_scale_host<<<vgrid2(n), 256, 0, s>>>(n, w, V + (size_t)(j + 1) * n, 1.0 / hn);
      SEM_LAUNCH_CHECK();
    }
    std::vector<double> Hs((size_t)k * k), ev(k), evec((size_t)k * k);
    for (int a = 0; a < k; ++a)
      for (int b = 0; b < k; ++b) Hs[a * k + b] = 0.5 * (H[(size_t)a * steps + b] + H[(size_t)b * steps + a]);
    jacobi_eig(k, Hs.data(), ev.data(), evec.data());
    double mx = ev[0];
    for (int a = 1; a < k; ++a) mx = std::max(mx, ev[a]);
    *lam = mx;
    if (!(mx > 0.0) || !std::isfinite(mx)) {
      set_detail("Arnoldi eigenvalue estimate failed on level %d", l);
      return SEM_EBREAKDOWN;
    }
    return SEM_OK;
  };
  if (rc == SEM_OK) rc = body();
  cudaStreamSynchronize(s);
  cudaFree(V);
  if (dh) cudaFree(dh);
  return rc;
}

}  // namespace sem
