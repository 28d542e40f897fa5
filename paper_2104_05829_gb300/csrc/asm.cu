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
// subdomain slots holding the node). Kernels: k_asm_fdm or k_asm_fdm_tc (gather,
// six 1-D contractions with the scaling fused between the t passes, store of the
// own part to z and the face layers to a staging array), k_asm_sum (for every
// node that has several copies, receives staged face-layer values or is
// Dirichlet: the sum of its copies and of its staged values in a fixed order,
// written to every copy, zero at Dirichlet nodes; P^T and QQ^T in one pass),
// then the weighted Chebyshev update.
#include <algorithm>
#include <climits>
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

// ---------------------------------------------------------------------------
// Tensor-core form of the FDM local solves (FP32 data, TF32 mma.sync with FP32
// accumulation). One warp per element. Each of the six 1-D passes is the product
//   OUT[l][a] = sum_m IN[l][m] Q[m][a]     (Q = S forward, S^T inverse)
// over the M^2 lines l = (p, q) of the box (p the line's fast coordinate, q its
// slow one), issued as mma.m16n8k8 on OUT^T = Q^T IN^T: the A operand is Q^T
// (rows a and the contraction index m padded to 16 with zeros, loaded once per
// pass), the B operand is a tile of eight lines. Tiles (TcPlan): eight lines of
// one q (p = 8h .. 8h+7), and, when M = 8 P + R with R = 2 or 4, the R remaining
// lines of 8/R consecutive q; for other R the rows are padded to whole tiles.
// Every lane then reads and writes at a fixed offset from its own base in every
// tile, so the addresses of a fully unrolled pass are immediates.
// A pass reads a line-major buffer ((p + M q) LS + m) and writes each lane's two
// accumulator lines (p, p + 1 of one q) as one 64-bit word of the next pass's
// layout, whose contraction index is this pass's p. Lines (p, q) per pass: r
// (j, k), s (k, i), t and inverse t (j, i), inverse s (i, k), inverse r (j, k);
// the inverse t pass reads an index-major buffer (m LD + p + M q, LD = 8 mod 32)
// and the result lands index-major for the output loops. LS = 12 (or 20) puts
// the 32 lanes of a load on distinct banks (64-bit: each bank twice).
// SPLIT = 1: one TF32 product per term (operands rounded to 11 significant
// bits); SPLIT = 3: each operand as the sum of two TF32 numbers and three
// products (hi*hi + hi*lo + lo*hi), about FP32 accuracy.
// Warps per block (1..8) that put the most warps on an SM within 227 KB of shared memory
// (blocks of ref + w * per_warp bytes, plus 1 KB reserved per block).
constexpr int tc_warps_per_block(int ref, int per_warp) {
  int best = 1, most = 0;
  for (int w = 1; w <= 8; ++w) {
    const int bytes = ref + w * per_warp;
    if (bytes > 227 * 1024) break;
    const int warps = w * ((227 * 1024) / (bytes + 1024));
    if (warps > most) {
      most = warps;
      best = w;
    }
  }
  return best;
}

template <int NP>
struct TcShape {
  static constexpr int M = NP + 2;
  static constexpr int L = M * M;                        // lines of one pass
  static constexpr int KS = (M + 7) / 8;                 // k-steps of the contraction index
  static constexpr int LS = M <= 12 ? 12 : 20;           // line stride
  static constexpr int LD = L + ((8 - L % 32) + 32) % 32;   // index stride, = 8 mod 32
  static constexpr int BUF0 = L * LS > M * LD ? L * LS : M * LD;
  static constexpr int BUF = (BUF0 + 3) / 4 * 4;
  static constexpr int TAB = (L + 3) / 4 * 4;
  static constexpr int WARP_FLOATS = 2 * BUF + TAB;      // two buffers and the scaling table
  static constexpr int REFB = 9 * AsmShape<NP>::REF * 4;
  static constexpr int WPB = tc_warps_per_block(REFB, WARP_FLOATS * 4);   // elements (warps) per block
  static constexpr size_t SMEM = (size_t)REFB + (size_t)WPB * WARP_FLOATS * 4;
};

template <int NP>
struct TcPlan {
  static constexpr int M = NP + 2, PM = M / 8, R = M % 8;
  static constexpr bool LEFT = R == 2 || R == 4;             // remainder lines grouped over q
  static constexpr bool PAD = !(R == 0 || LEFT);             // rows padded to whole tiles
  static constexpr int PB = PAD ? PM + 1 : PM;               // tiles of one q
  static constexpr int RT = LEFT ? 8 / R : 1;                // q per remainder tile
  static constexpr int NMT = M * PB;
  static constexpr int NTT = NMT + (LEFT ? (M + RT - 1) / RT : 0);
};

// FP32 -> TF32 operand: round to 11 significant bits (half away from zero in magnitude) with
// two integer operations; the tensor cores read the top 19 bits of the word.
__device__ __forceinline__ uint32_t tf32_rn(float x) { return (__float_as_uint(x) + 0x1000u) & 0xffffe000u; }

__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int SPLIT>
__device__ __forceinline__ void tf32_split(float x, uint32_t& h, uint32_t& l) {
  h = tf32_rn(x);
  if (SPLIT == 3) l = tf32_rn(x - __uint_as_float(h));   // x - h is exact
}

// Q^T as the A operand of every k-step: a0 = Q[m(t)][g], a1 = Q[m(t)][g+8], a2 = Q[m'(t)][g],
// a3 = Q[m'(t)][g+8]; PERM pairs the contraction indices as m = 8ks + 2t, m' = m + 1 (so that
// the B operand's two words per lane are adjacent), otherwise m = 8ks + t, m' = m + 4.
template <int NP, bool TRANS, bool PERM, int SPLIT>
__device__ __forceinline__ void tc_qfrag(const float* __restrict__ S, int g, int t,
                                         uint32_t (&ah)[TcShape<NP>::KS][4], uint32_t (&al)[TcShape<NP>::KS][4]) {
  constexpr int M = TcShape<NP>::M, MR = AsmShape<NP>::MR;
  auto q = [&](int m, int a) -> float {
    if (m >= M || a >= M) return 0.f;
    return TRANS ? S[a * MR + m] : S[m * MR + a];
  };
#pragma unroll
  for (int ks = 0; ks < TcShape<NP>::KS; ++ks) {
    const int m0 = PERM ? 8 * ks + 2 * t : 8 * ks + t;
    const int m1 = PERM ? m0 + 1 : m0 + 4;
    tf32_split<SPLIT>(q(m0, g), ah[ks][0], al[ks][0]);
    tf32_split<SPLIT>(q(m0, g + 8), ah[ks][1], al[ks][1]);
    tf32_split<SPLIT>(q(m1, g), ah[ks][2], al[ks][2]);
    tf32_split<SPLIT>(q(m1, g + 8), ah[ks][3], al[ks][3]);
  }
}

template <int SPLIT>
__device__ __forceinline__ void tc_mma(float (&c)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4], float x0,
                                       float x1) {
  uint32_t bh0, bl0, bh1, bl1;
  tf32_split<SPLIT>(x0, bh0, bl0);
  tf32_split<SPLIT>(x1, bh1, bl1);
  if (SPLIT == 3) {
    mma_tf32(c, al, bh0, bh1);
    mma_tf32(c, ah, bl0, bl1);
  }
  mma_tf32(c, ah, bh0, bh1);
}

// Lines of tile tt for lane (g, t): the B operand's line (bp, bq), and the first of the two
// accumulator lines (sp, sq) (the second is sp + 1, same sq).
template <int NP>
__device__ __forceinline__ void tc_tile(int tt, int g, int t, int& bp, int& bq, int& sp, int& sq) {
  using P = TcPlan<NP>;
  if constexpr (P::LEFT) {
    if (tt >= P::NMT) {
      const int q0 = (tt - P::NMT) * P::RT;
      bq = q0 + g / P::R;
      bp = 8 * P::PM + g % P::R;
      sq = q0 + (2 * t) / P::R;
      sp = 8 * P::PM + (2 * t) % P::R;
      return;
    }
  }
  const int q = tt / P::PB, h = tt - q * P::PB;
  bq = sq = q;
  bp = 8 * h + g;
  sp = 8 * h + 2 * t;
}

// B operand loads from line-major buffers: the two words of a lane as one 64-bit load (m = 2t,
// 2t + 1; a half-warp then spans its banks twice at LS = 12) or as two 32-bit loads (m = t,
// t + 4; every lane on its own bank).
constexpr bool kTcPairLoads = false;

// the B operand of one tile (zero for lines or indices outside the box)
template <int NP, bool IN_LINE>
__device__ __forceinline__ void tc_load(const float* __restrict__ in, int bp, int bq, int t,
                                        float (&x)[TcShape<NP>::KS][2]) {
  using Sh = TcShape<NP>;
  constexpr int M = Sh::M, LS = Sh::LS, LD = Sh::LD;
  const bool ok = bp < M && bq < M;
  const int l = bp + M * bq;
#pragma unroll
  for (int ks = 0; ks < Sh::KS; ++ks) {
    x[ks][0] = 0.f;
    x[ks][1] = 0.f;
    if (IN_LINE && kTcPairLoads) {
      const int m0 = 8 * ks + 2 * t;
      if (ok && m0 + 1 < M) {
        const float2 v = *reinterpret_cast<const float2*>(in + l * LS + m0);
        x[ks][0] = v.x;
        x[ks][1] = v.y;
      } else if (ok && m0 < M) {
        x[ks][0] = in[l * LS + m0];
      }
    } else if (IN_LINE) {
      const int m0 = 8 * ks + t;
      if (ok && m0 < M) x[ks][0] = in[l * LS + m0];
      if (ok && m0 + 4 < M) x[ks][1] = in[l * LS + m0 + 4];
    } else {
      const int m0 = 8 * ks + t;
      if (ok && m0 < M) x[ks][0] = in[m0 * LD + l];
      if (ok && m0 + 4 < M) x[ks][1] = in[(m0 + 4) * LD + l];
    }
  }
}

// One pass over every tile, fully unrolled; the operands of the next tile are loaded before
// this tile's products and stores. post(sp, sq, c): c[0], c[1] = OUT[(sp, sq)][g],
// OUT[(sp + 1, sq)][g]; c[2], c[3] the same for output g + 8.
template <int NP, int SPLIT, bool IN_LINE, class Post>
__device__ __forceinline__ void tc_pass(const float* __restrict__ in, const uint32_t (&ah)[TcShape<NP>::KS][4],
                                        const uint32_t (&al)[TcShape<NP>::KS][4], int g, int t, Post post) {
  using Sh = TcShape<NP>;
  using P = TcPlan<NP>;
  float xn[Sh::KS][2];
  {
    int bp, bq, sp, sq;
    tc_tile<NP>(0, g, t, bp, bq, sp, sq);
    tc_load<NP, IN_LINE>(in, bp, bq, t, xn);
  }
#pragma unroll
  for (int tt = 0; tt < P::NTT; ++tt) {
    float x[Sh::KS][2];
#pragma unroll
    for (int ks = 0; ks < Sh::KS; ++ks) {
      x[ks][0] = xn[ks][0];
      x[ks][1] = xn[ks][1];
    }
    int bp, bq, sp, sq;
    if (tt + 1 < P::NTT) {
      tc_tile<NP>(tt + 1, g, t, bp, bq, sp, sq);
      tc_load<NP, IN_LINE>(in, bp, bq, t, xn);
    }
    tc_tile<NP>(tt, g, t, bp, bq, sp, sq);
    float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int ks = 0; ks < Sh::KS; ++ks) tc_mma<SPLIT>(c, ah[ks], al[ks], x[ks][0], x[ks][1]);
    post(sp, sq, c);
  }
}

// Store OUT[(p, q)][a] and OUT[(p + 1, q)][a] at addr(p, q, a), addr(p, q, a) + 1 (p is the
// next layout's fastest index): one 64-bit word when M is even, else two words.
template <int NP, class Addr>
__device__ __forceinline__ void tc_store_pair(float* __restrict__ out, int p, int q, int a, float v0, float v1,
                                              Addr addr) {
  constexpr int M = TcShape<NP>::M;
  if (a >= M || q >= M || p >= M) return;
  if (M % 2 == 0) {
    *reinterpret_cast<float2*>(out + addr(p, q, a)) = make_float2(v0, v1);
  } else {
    out[addr(p, q, a)] = v0;
    if (p + 1 < M) out[addr(p, q, a) + 1] = v1;
  }
}

template <int NP>
__device__ __forceinline__ void layer_coords(int f, int a, int b, int& ib, int& jb, int& kb) {
  const int d = f >> 1, c = (f & 1) ? NP + 1 : 0;
  if (d == 0) { ib = c; jb = a + 1; kb = b + 1; }
  else if (d == 1) { ib = a + 1; jb = c; kb = b + 1; }
  else { ib = a + 1; jb = b + 1; kb = c; }
}

template <int NP, int SPLIT>
__global__ void __launch_bounds__(32 * TcShape<NP>::WPB)
    k_asm_fdm_tc(int E, const float* __restrict__ bv, const float* __restrict__ wv,
                 const int32_t* __restrict__ layer, const uint8_t* __restrict__ bt, const float* __restrict__ len,
                 const float* __restrict__ ref, float h1, float h2, float* __restrict__ z, float* __restrict__ zf) {
  using Sh = TcShape<NP>;
  using As = AsmShape<NP>;
  constexpr int M = Sh::M, L = Sh::L, LS = Sh::LS, LD = Sh::LD, KS = Sh::KS, MR = As::MR;
  constexpr int NP2 = NP * NP, NP3 = NP2 * NP;
  extern __shared__ __align__(16) float s_tc[];
  float* s_ref = s_tc;                    // 9 side combinations (REF is a multiple of 4)
  float* s_warp = s_tc + 9 * As::REF;     // per warp: B0, B1, the scaling table
  for (int q = threadIdx.x; q < 9 * As::REF; q += blockDim.x) s_ref[q] = ref[q];
  __syncthreads();
  const int wq = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int e = blockIdx.x * Sh::WPB + wq;
  if (e >= E) return;   // no block-wide barrier follows
  float* B0 = s_warp + wq * Sh::WARP_FLOATS;
  float* B1 = B0 + Sh::BUF;
  float* base = B1 + Sh::BUF;   // h1 (l_r + l_s) + h2 per line (j, i) of the t pass
  for (int q = lane; q < Sh::BUF / 4; q += 32) reinterpret_cast<float4*>(B0)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  const uint8_t* b6 = bt + (size_t)e * 6;
  const float* Sr = s_ref + (3 * b6[0] + b6[1]) * As::REF;
  const float* Ss = s_ref + (3 * b6[2] + b6[3]) * As::REF;
  const float* St = s_ref + (3 * b6[4] + b6[5]) * As::REF;
  const float sr = 2.f / len[(size_t)e * 3 + 0], ss = 2.f / len[(size_t)e * 3 + 1], st = 2.f / len[(size_t)e * 3 + 2];
  for (int l = lane; l < L; l += 32) {
    const int i = l / M, j = l - i * M;
    base[l] = h1 * (Sr[M * MR + i] * sr * sr + Ss[M * MR + j] * ss * ss) + h2;
  }
  __syncwarp();
  // gather the box (r pass layout: (j + M k) LS + i), the loads of a chunk (all of them up to
  // N = 7) issued before the first store
  {
    constexpr int NO = (NP3 + 31) / 32, NF = (6 * NP2 + 31) / 32;
    constexpr int CO = NO < 16 ? NO : 16, CF = NF < 12 ? NF : 12;
    constexpr int IO = (NO + CO - 1) / CO, IF = (NF + CF - 1) / CF, NI = IO > IF ? IO : IF;
    const size_t eb = (size_t)e * NP3;
    const int32_t* lay = layer + (size_t)e * 6 * NP2;
#pragma unroll 1
    for (int it = 0; it < NI; ++it) {
      const int o0 = it * CO, f0 = it * CF;   // this chunk's own-point and face-layer slots
      float ob[CO], ow[CO];
#pragma unroll
      for (int c = 0; c < CO; ++c) {
        const int q = lane + 32 * (o0 + c);
        ob[c] = q < NP3 ? bv[eb + q] : 0.f;
        ow[c] = (wv && q < NP3) ? wv[eb + q] : 0.f;
      }
      int32_t src[CF];
#pragma unroll
      for (int c = 0; c < CF; ++c) {
        const int q = lane + 32 * (f0 + c);
        src[c] = q < 6 * NP2 ? lay[q] : -1;
      }
      float fb[CF], fw[CF];
#pragma unroll
      for (int c = 0; c < CF; ++c) {
        fb[c] = src[c] >= 0 ? bv[src[c]] : 0.f;
        fw[c] = (wv && src[c] >= 0) ? wv[src[c]] : 0.f;
      }
#pragma unroll
      for (int c = 0; c < CO; ++c) {
        const int q = lane + 32 * (o0 + c);
        if (q < NP3) {
          const int k = q / NP2, j = (q / NP) % NP, i = q % NP;
          B0[((j + 1) + M * (k + 1)) * LS + i + 1] = ob[c] - ow[c];
        }
      }
#pragma unroll
      for (int c = 0; c < CF; ++c) {
        const int q = lane + 32 * (f0 + c);
        if (src[c] >= 0) {
          const int f = q / NP2, ab = q - f * NP2;
          int ib, jb, kb;
          layer_coords<NP>(f, ab / NP, ab % NP, ib, jb, kb);
          B0[(jb + M * kb) * LS + ib] = fb[c] - fw[c];
        }
      }
    }
  }
  __syncwarp();
  uint32_t ah[KS][4], al[KS][4];
  // next layout (q + M a) LS + p: the s pass after r, the inverse s pass after inverse t
  auto ad_qa = [](int p, int q, int a) { return (q + M * a) * LS + p; };
  // next layout (a + M q) LS + p: the t pass after s, the inverse r pass after inverse s
  auto ad_aq = [](int p, int q, int a) { return (a + M * q) * LS + p; };
  // index-major a LD + p + M q: the inverse t pass after t, and the result
  auto ad_im = [](int p, int q, int a) { return a * LD + p + M * q; };
  // r: lines (j, k)
  tc_qfrag<NP, false, kTcPairLoads, SPLIT>(Sr, g, t, ah, al);
  tc_pass<NP, SPLIT, true>(B0, ah, al, g, t, [&](int p, int q, const float (&c)[4]) {
    tc_store_pair<NP>(B1, p, q, g, c[0], c[1], ad_qa);
    tc_store_pair<NP>(B1, p, q, g + 8, c[2], c[3], ad_qa);
  });
  __syncwarp();
  // s: lines (k, i)
  tc_qfrag<NP, false, kTcPairLoads, SPLIT>(Ss, g, t, ah, al);
  tc_pass<NP, SPLIT, true>(B1, ah, al, g, t, [&](int p, int q, const float (&c)[4]) {
    tc_store_pair<NP>(B0, p, q, g, c[0], c[1], ad_aq);
    tc_store_pair<NP>(B0, p, q, g + 8, c[2], c[3], ad_aq);
  });
  __syncwarp();
  // t: lines (j, i), scaled by c / (h1 (l_r + l_s + l_t) + h2)
  {
    const float cc = sr * ss * st;
    const float ht0 = g < M ? h1 * St[M * MR + g] * st * st : 0.f;
    const float ht1 = g + 8 < M ? h1 * St[M * MR + g + 8] * st * st : 0.f;
    tc_qfrag<NP, false, kTcPairLoads, SPLIT>(St, g, t, ah, al);
    tc_pass<NP, SPLIT, true>(B0, ah, al, g, t, [&](int p, int q, const float (&c)[4]) {
      if (p >= M || q >= M) return;
      const int l = p + M * q;
      const float b0 = base[l], b1 = p + 1 < M ? base[l + 1] : 1.f;
      const float dn[4] = {b0 + ht0, b1 + ht0, b0 + ht1, b1 + ht1};
      float v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = dn[k] != 0.f ? fdiv(cc * c[k], dn[k]) : 0.f;
      tc_store_pair<NP>(B1, p, q, g, v[0], v[1], ad_im);
      tc_store_pair<NP>(B1, p, q, g + 8, v[2], v[3], ad_im);
    });
  }
  __syncwarp();
  // inverse t: lines (j, i), index-major input
  tc_qfrag<NP, true, false, SPLIT>(St, g, t, ah, al);
  tc_pass<NP, SPLIT, false>(B1, ah, al, g, t, [&](int p, int q, const float (&c)[4]) {
    tc_store_pair<NP>(B0, p, q, g, c[0], c[1], ad_qa);
    tc_store_pair<NP>(B0, p, q, g + 8, c[2], c[3], ad_qa);
  });
  __syncwarp();
  // inverse s: lines (i, k)
  tc_qfrag<NP, true, kTcPairLoads, SPLIT>(Ss, g, t, ah, al);
  tc_pass<NP, SPLIT, true>(B0, ah, al, g, t, [&](int p, int q, const float (&c)[4]) {
    tc_store_pair<NP>(B1, p, q, g, c[0], c[1], ad_aq);
    tc_store_pair<NP>(B1, p, q, g + 8, c[2], c[3], ad_aq);
  });
  __syncwarp();
  // inverse r: lines (j, k) -> the result, index-major i LD + j + M k
  tc_qfrag<NP, true, kTcPairLoads, SPLIT>(Sr, g, t, ah, al);
  tc_pass<NP, SPLIT, true>(B1, ah, al, g, t, [&](int p, int q, const float (&c)[4]) {
    tc_store_pair<NP>(B0, p, q, g, c[0], c[1], ad_im);
    tc_store_pair<NP>(B0, p, q, g + 8, c[2], c[3], ad_im);
  });
  __syncwarp();
  // outputs, unrolled so that the slot arithmetic folds into per-lane constants
  const size_t eb = (size_t)e * NP3;
#pragma unroll
  for (int c = 0; c < (NP3 + 31) / 32; ++c) {
    const int q = lane + 32 * c;
    if (q < NP3) {
      const int k = q / NP2, j = (q / NP) % NP, i = q % NP;
      z[eb + q] = B0[(i + 1) * LD + (j + 1) + M * (k + 1)];
    }
  }
  float* zfe = zf + (size_t)e * 6 * NP2;
#pragma unroll
  for (int c = 0; c < (6 * NP2 + 31) / 32; ++c) {
    const int q = lane + 32 * c;
    if (q < 6 * NP2) {
      const int f = q / NP2, ab = q - f * NP2;
      int ib, jb, kb;
      layer_coords<NP>(f, ab / NP, ab % NP, ib, jb, kb);
      zfe[q] = B0[ib * LD + jb + M * kb];
    }
  }
}

// Threads [0, nw): for every work node w, s = sum of its items in list order (item >= 0: the
// local copy z[item]; item < 0: the staged face-layer value zf[-item - 1]), written to every
// copy; 0 at Dirichlet nodes. The copies of a node come first, ascending, then the staged slots
// of each copy. Threads [nw, nw + np): the nodes with one copy and one staged value, as
// (copy, slot) pairs: z[copy] += zf[slot].
template <typename T>
__global__ void k_asm_sum(int64_t nw, const int32_t* __restrict__ off, const int32_t* __restrict__ item,
                          const uint8_t* __restrict__ dir, int64_t np, const int2* __restrict__ pair,
                          const T* __restrict__ zf, T* __restrict__ z) {
  const int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (w >= nw) {
    if (w < nw + np) {
      const int2 cs = pair[w - nw];
      z[cs.x] = z[cs.x] + zf[cs.y];
    }
    return;
  }
  const int b = off[w], e = off[w + 1], m = e - b;
  if (dir[w]) {
    for (int p = b; p < e; ++p)
      if (item[p] >= 0) z[item[p]] = T(0);
    return;
  }
  if (m <= 8) {
    int id[8];
    T v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) id[q] = q < m ? item[b + q] : 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = q < m ? (id[q] >= 0 ? z[id[q]] : zf[-id[q] - 1]) : T(0);
    T s = v[0];
#pragma unroll
    for (int q = 1; q < 8; ++q)
      if (q < m) s += v[q];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (q < m && id[q] >= 0) z[id[q]] = s;
    return;
  }
  T s = T(0);
  for (int p = b; p < e; ++p) {
    const int it = item[p];
    s += it >= 0 ? z[it] : zf[-it - 1];
  }
  for (int p = b; p < e; ++p)
    if (item[p] >= 0) z[item[p]] = s;
}

template <typename T>
__global__ void k_mul_w(int64_t n, const T* __restrict__ w, T* __restrict__ z) {
  GRID_LOOP(l, n) z[l] *= w[l];
}

// the same in chunks of four (16-byte aligned FP32 vectors)
__global__ void k_cheb_w4(int64_t n, const float* __restrict__ z, const float* __restrict__ W, float* __restrict__ x,
                          float* __restrict__ d, float c1, float c2, int first, int x_zero) {
  auto one = [&](float zl, float Wl, float dl0, float xl) {
    const float dl = first ? c2 * (Wl * zl) : c1 * dl0 + c2 * (Wl * zl);
    return make_float2(dl, x_zero ? dl : xl + dl);
  };
  grid_loop_f4(
      n,
      [&](int64_t i) {
        const float4 zz = ld4(z, i), ww = ld4(W, i);
        const float4 dd = first ? make_float4(0.f, 0.f, 0.f, 0.f) : ld4(d, i);
        const float4 xx = x_zero ? make_float4(0.f, 0.f, 0.f, 0.f) : ld4(x, i);
        const float2 r0 = one(zz.x, ww.x, dd.x, xx.x), r1 = one(zz.y, ww.y, dd.y, xx.y);
        const float2 r2 = one(zz.z, ww.z, dd.z, xx.z), r3 = one(zz.w, ww.w, dd.w, xx.w);
        st4(d, i, make_float4(r0.x, r1.x, r2.x, r3.x));
        st4(x, i, make_float4(r0.y, r1.y, r2.y, r3.y));
      },
      [&](int64_t l) {
        const float2 r = one(z[l], W[l], first ? 0.f : d[l], x_zero ? 0.f : x[l]);
        d[l] = r.x;
        x[l] = r.y;
      });
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

// tc (FP32 data only): 0 the FP32 FMA kernel, 1 TF32 tensor cores, 3 three TF32 products.
template <typename T, int NP>
int launch_fdm(const Level& L, const T* b, const T* w, T* z, T* zf, double h1, double h2, int tc, cudaStream_t s) {
  using Sh = AsmShape<NP>;
  const T* len = std::is_same<T, double>::value ? (const T*)L.sch_len : (const T*)L.sch_len32;
  const T* ref = std::is_same<T, double>::value ? (const T*)L.sch_ref : (const T*)L.sch_ref32;
  if constexpr (std::is_same<T, float>::value) {
    if (tc) {
      using Tc = TcShape<NP>;
      const unsigned grid = (unsigned)((L.E + Tc::WPB - 1) / Tc::WPB);
      static PerDevice<bool> attr[2];
      if (tc == 3) {
        SEM_TRY(smem_attr_once(attr[1], (const void*)k_asm_fdm_tc<NP, 3>, Tc::SMEM));
        k_asm_fdm_tc<NP, 3><<<grid, 32 * Tc::WPB, Tc::SMEM, s>>>(L.E, b, w, L.sch_layer, L.sch_bt, len, ref,
                                                                 (float)h1, (float)h2, z, zf);
      } else {
        SEM_TRY(smem_attr_once(attr[0], (const void*)k_asm_fdm_tc<NP, 1>, Tc::SMEM));
        k_asm_fdm_tc<NP, 1><<<grid, 32 * Tc::WPB, Tc::SMEM, s>>>(L.E, b, w, L.sch_layer, L.sch_bt, len, ref,
                                                                 (float)h1, (float)h2, z, zf);
      }
      SEM_LAUNCH_CHECK();
      return SEM_OK;
    }
  }
  const unsigned grid = (unsigned)((L.E + Sh::EPB - 1) / Sh::EPB);
  k_asm_fdm<T, NP><<<grid, Sh::THREADS, 0, s>>>(L.E, b, w, L.sch_layer, L.sch_bt, len, ref, (T)h1, (T)h2, z, zf);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}

template <typename T>
int dispatch_fdm(const Level& L, const T* b, const T* w, T* z, T* zf, double h1, double h2, int tc,
                 cudaStream_t s) {
  switch (L.NP) {
    case 3: return launch_fdm<T, 3>(L, b, w, z, zf, h1, h2, tc, s);
    case 4: return launch_fdm<T, 4>(L, b, w, z, zf, h1, h2, tc, s);
    case 5: return launch_fdm<T, 5>(L, b, w, z, zf, h1, h2, tc, s);
    case 6: return launch_fdm<T, 6>(L, b, w, z, zf, h1, h2, tc, s);
    case 7: return launch_fdm<T, 7>(L, b, w, z, zf, h1, h2, tc, s);
    case 8: return launch_fdm<T, 8>(L, b, w, z, zf, h1, h2, tc, s);
    case 9: return launch_fdm<T, 9>(L, b, w, z, zf, h1, h2, tc, s);
    case 10: return launch_fdm<T, 10>(L, b, w, z, zf, h1, h2, tc, s);
    case 11: return launch_fdm<T, 11>(L, b, w, z, zf, h1, h2, tc, s);
    case 12: return launch_fdm<T, 12>(L, b, w, z, zf, h1, h2, tc, s);
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
  // work nodes of k_asm_sum: every node with several copies, staged values or a Dirichlet mask,
  // in the order of their first copies (neighbouring threads then touch neighbouring points);
  // items: its copies (ascending), then the staged slots of each copy (slot order)
  std::vector<int32_t> woff(1, 0), witem, wpair;
  std::vector<uint8_t> wdir;
  for (int64_t l = 0; l < nL; ++l) {
    const int64_t g = node[l];
    const int64_t c0 = hoff[g], c1 = hoff[g + 1];
    if (hidx[c0] != l) continue;
    bool pulled = false;
    for (int64_t o = c0; o < c1; ++o) pulled = pulled || first[hidx[o]] >= 0;
    const bool dirichlet = dmask[hidx[c0]] != 0;
    if (c1 - c0 < 2 && !pulled && !dirichlet) continue;
    if (c1 - c0 == 1 && !dirichlet) {
      const int64_t f = first[hidx[c0]];
      if (poff[f + 1] - poff[f] == 1) {   // one copy, one staged value: a (copy, slot) pair
        wpair.push_back((int32_t)hidx[c0]);
        wpair.push_back(psrc[poff[f]]);
        continue;
      }
    }
    for (int64_t o = c0; o < c1; ++o) witem.push_back((int32_t)hidx[o]);
    for (int64_t o = c0; o < c1; ++o) {
      const int64_t f = first[hidx[o]];
      if (f < 0) continue;
      for (int32_t q = poff[f]; q < poff[f + 1]; ++q) witem.push_back(-psrc[q] - 1);
    }
    if (witem.size() > (size_t)INT32_MAX) {
      set_detail("Schwarz work lists exceed 2^31 entries");
      return SEM_EINVAL;
    }
    woff.push_back((int32_t)witem.size());
    wdir.push_back(dirichlet ? 1 : 0);
  }
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
  SEM_TRY(dmalloc_n(&L.sch_woff, woff.size()));
  SEM_TRY(dmalloc_n(&L.sch_witem, witem.size()));
  SEM_TRY(dmalloc_n(&L.sch_wdir, wdir.size()));
  SEM_TRY(dmalloc_n(&L.sch_wpair, wpair.size() / 2));
  if (f32) {
    SEM_TRY(dmalloc_n(&L.sch_len32, (size_t)E * 3));
    SEM_TRY(dmalloc_n(&L.sch_ref32, ref32.size()));
    SEM_TRY(dmalloc_n(&L.sch_w32, (size_t)nL));
    SEM_TRY(dmalloc_n(&L.sch_zf32, layer.size()));
  }
  L.sch_nw = (int64_t)wdir.size();
  L.sch_np = (int64_t)wpair.size() / 2;
  SEM_CUDA_TRY(cudaMemcpyAsync(L.sch_layer, layer.data(), layer.size() * 4, cudaMemcpyHostToDevice, s));
  SEM_CUDA_TRY(cudaMemcpyAsync(L.sch_bt, bt.data(), bt.size(), cudaMemcpyHostToDevice, s));
  SEM_CUDA_TRY(cudaMemcpyAsync(L.sch_ref, ref.data(), ref.size() * 8, cudaMemcpyHostToDevice, s));
  SEM_CUDA_TRY(cudaMemcpyAsync(L.sch_woff, woff.data(), woff.size() * 4, cudaMemcpyHostToDevice, s));
  SEM_CUDA_TRY(cudaMemcpyAsync(L.sch_witem, witem.data(), witem.size() * 4, cudaMemcpyHostToDevice, s));
  SEM_CUDA_TRY(cudaMemcpyAsync(L.sch_wdir, wdir.data(), wdir.size(), cudaMemcpyHostToDevice, s));
  SEM_CUDA_TRY(cudaMemcpyAsync(L.sch_wpair, wpair.data(), wpair.size() * 4, cudaMemcpyHostToDevice, s));
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

// FP32 local solves: the FMA kernel (0), or TF32 tensor cores with one (1) or three (3) products.
constexpr int kFdmFp32Mode = 3;

// z = sum_e P_e^T F_e P_e (b - w) on level L, gathered over copies and masked
// (no weight). w may be null (r = b). prec: SEM_FP64 (double) or FP32 (float vectors).
int asm_sum(const Level& L, int prec, const void* b, const void* w, void* z, double h1, double h2, cudaStream_t s) {
  if (!L.sch_ready) {
    set_detail("Schwarz data of level order %d not built", L.N);
    return SEM_EINVAL;
  }
  const unsigned nb = (unsigned)((L.sch_nw + L.sch_np + 255) / 256);
  if (prec == SEM_FP64) {
    SEM_TRY(dispatch_fdm<double>(L, (const double*)b, (const double*)w, (double*)z, L.sch_zf, h1, h2, 0, s));
    if (nb)
      k_asm_sum<double><<<nb, 256, 0, s>>>(L.sch_nw, L.sch_woff, L.sch_witem, L.sch_wdir, L.sch_np, L.sch_wpair,
                                           L.sch_zf, (double*)z);
  } else {
    if (!L.sch_ref32) {
      set_detail("FP32 Schwarz data not built (no FP32 factor copies)");
      return SEM_EINVAL;
    }
    const int tc = prec == SEM_BF16G ? 1 : kFdmFp32Mode;
    SEM_TRY(dispatch_fdm<float>(L, (const float*)b, (const float*)w, (float*)z, L.sch_zf32, h1, h2, tc, s));
    if (nb)
      k_asm_sum<float><<<nb, 256, 0, s>>>(L.sch_nw, L.sch_woff, L.sch_witem, L.sch_wdir, L.sch_np, L.sch_wpair,
                                          L.sch_zf32, (float*)z);
  }
  SEM_LAUNCH_CHECK();
  return SEM_OK;
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
  else if (kVec4 && aligned16({z, L.sch_w32, x, d}))
    k_cheb_w4<<<vgrid2(L.nL / 4), 256, 0, s>>>(L.nL, (const float*)z, L.sch_w32, (float*)x, (float*)d, (float)c1,
                                               (float)c2, first ? 1 : 0, x_zero ? 1 : 0);
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
