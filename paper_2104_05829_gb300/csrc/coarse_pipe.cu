// Coarsest-level Jacobi-PCG (order 1) as pipelined PCG on sub-domains, in one
// cooperative launch with one exchange between blocks per iteration.
//
// The order-1 elements are split into one sub-domain per block by recursive
// coordinate bisection of their centroids (host, once per level). A block keeps
// the assembled Krylov vectors of every node its elements touch in registers
// (a node on a sub-domain interface is held by every block that touches it,
// with identical bits), and its elements' geometric factors, point-to-node map
// and node copy lists in shared memory. The direct-stiffness sum QQ^T of an
// operator output is a gather: every block sums, for each of its nodes, all
// copies of the node in canonical order (ascending local index), its own copies
// from shared memory and the other blocks' from an exchange buffer that those
// blocks publish. Nothing is scattered into another block, so one exchange per
// operator application suffices.
//
// The iteration is pipelined PCG (Ghysels and Vanroose, Parallel Computing
// 2014) with the Jacobi preconditioner: the dot products of an iteration need
// only vectors that exist before its operator application, so their block
// partials travel in the same exchange. In exact arithmetic the
// iterates are those of Jacobi-PCG.
//   r = b, u = D^-1 r, w = A u (one extra exchange); for i = 0, 1, ...
//     gamma = (r, u), delta = (w, u), rr = (r, r); m = D^-1 w; n = A m
//     stop if rr <= tol^2 (b, b) or i = maxit (x is the result)
//     beta = gamma / gamma_old (0 at i = 0), pi = delta - beta^2 pi_old (= (p, A p)),
//     alpha = gamma / pi
//     z = n + beta z, q = m + beta q, s = w + beta s, p = u + beta p
//     x += alpha p, r -= alpha s, u -= alpha q, w -= alpha z
// Dot products count each non-Dirichlet node once (in the block holding its
// owner copy); block partials (in the arithmetic type, published in FP64) are
// added by every block in one fixed order, so all blocks take the same
// decisions. The scalar step runs on one thread and keeps its FP64 work short
// (GB300's FP64 pipe is narrow): 1 / gamma_old is formed earlier by another
// thread, and the FP32 solve divides in FP32.
// Exchange: every block publishes each interface output and each block partial
// as tagged words (an FP32 value and its epoch in one 64-bit word; an FP64 value
// as two such words, one per half, in one 128-bit access; relaxed 64-bit accesses
// are single-copy atomic), and a block waits only on the words it reads, with no
// fence and no grid barrier. Exchange buffer and partials are double-buffered by
// epoch parity: the dot products couple every block once per iteration, so no
// block can overwrite a word another block has still to read. Waits are bounded (about a second of SM
// clock); after a timeout every wait ends at once and the solve reports a
// breakdown.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "sem_internal.cuh"
#include "spin.cuh"

namespace sem {

namespace {

constexpr int PT = 512;             // threads per block
constexpr int PIPE_MAX_BLOCKS = 256; // block partials are read eight per lane by one warp
constexpr int PW = PT / 32;
constexpr int NPC = 2;              // order 1
constexpr int NPC3 = 8;
constexpr int GF = 7 * NPC3;        // factor values per element
constexpr int32_t NODE_MASK = 0x7fffffff;

struct PipeArgs {
  const void* G;                    // [E][7][8]
  const void* b;
  void* x;
  const void* dinv;
  void* xbuf;                       // [2][nL] tagged values (8 bytes each in FP32, 16 in FP64)
  int64_t nL;
  const int32_t* el_off;
  const int32_t* el;
  const int32_t* p2n;
  const int32_t* nd_off;
  const int32_t* nd_src;
  const uint8_t* nd_fl;
  const int32_t* cp_off;
  const int32_t* cp;
  int max_el, max_nd, max_cp;
  double h1, h2, tol;
  int maxit;
  double* part;                     // [2][3][B] tagged partials
  int* err;
  double* sc;                       // outputs: S_ITER, S_TOTAL, S_RR, S_BB, S_DONE, S_BREAK
  double* outer_sc;                 // the calling solve's scalars: S_BREAK and S_DONE set when a wait gave up
  long long spin;                   // SM clocks a wait may spin
};

__host__ __device__ constexpr size_t al16(size_t v) { return (v + 15) / 16 * 16; }

// shared-memory layout of a block (the same offsets on host and device)
struct PipeSmem {
  size_t pt, m, el, p2n, cpo, cp, total;
  template <typename T, typename GT, bool SMEM_G>
  __host__ __device__ static PipeSmem make(int max_el, int max_nd, int max_cp) {
    PipeSmem o{};
    o.pt = SMEM_G ? al16((size_t)max_el * GF * sizeof(GT)) : 0;
    o.m = o.pt + al16((size_t)max_el * NPC3 * sizeof(T));
    o.el = o.m + al16((size_t)max_nd * sizeof(T));
    o.p2n = o.el + al16((size_t)max_el * 4);
    o.cpo = o.p2n + al16((size_t)max_el * NPC3 * 4);
    o.cp = o.cpo + al16((size_t)(max_nd + 1) * 4);
    o.total = o.cp + al16((size_t)max_cp * 4);
    return o;
  }
};

__device__ __forceinline__ double fval(double v) { return v; }
__device__ __forceinline__ float fval(float v) { return v; }
__device__ __forceinline__ float fval(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T>
__device__ __forceinline__ T quotient(double n, double d);
template <>
__device__ __forceinline__ double quotient<double>(double n, double d) { return n / d; }
template <>
__device__ __forceinline__ float quotient<float>(double n, double d) { return (float)n / (float)d; }

// Tagged words of the exchange. An FP32 value is one 64-bit word (value bits low,
// epoch high); an FP64 value is two such words, one per 32-bit half, written and
// read by one 128-bit access. Relaxed 64-bit accesses at GPU scope are single-copy
// atomic, so a reader that sees the awaited epoch in every word of a value holds
// that epoch's value; no fence and no flag are needed.
__device__ __forceinline__ bool tag_is(uint64_t w, unsigned tag) { return (unsigned)(w >> 32) == tag; }
__device__ __forceinline__ uint64_t tag_word(unsigned bits, unsigned tag) { return ((uint64_t)tag << 32) | bits; }

template <typename T>
struct Tagged;
template <>
struct Tagged<float> {
  using W = uint64_t;
  __device__ static void st(W* p, float v, unsigned tag) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(tag_word(__float_as_uint(v), tag)) : "memory");
  }
  __device__ static W ld(const W* p) {
    W w;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(w) : "l"(p) : "memory");
    return w;
  }
  __device__ static W zero() { return 0; }
  __device__ static bool ok(const W& w, unsigned tag) { return tag_is(w, tag); }
  __device__ static float val(const W& w) { return __uint_as_float((unsigned)w); }
};
template <>
struct Tagged<double> {
  struct __align__(16) W {
    uint64_t hi, lo;
  };
  __device__ static void st(W* p, double v, unsigned tag) {
    const uint64_t a = tag_word((unsigned)__double2hiint(v), tag), b = tag_word((unsigned)__double2loint(v), tag);
    asm volatile("st.relaxed.gpu.global.v2.b64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
  }
  __device__ static W ld(const W* p) {
    W w;
    asm volatile("ld.relaxed.gpu.global.v2.b64 {%0, %1}, [%2];" : "=l"(w.hi), "=l"(w.lo) : "l"(p) : "memory");
    return w;
  }
  __device__ static W zero() { return {0, 0}; }
  __device__ static bool ok(const W& w, unsigned tag) { return tag_is(w.hi, tag) && tag_is(w.lo, tag); }
  __device__ static double val(const W& w) { return __hiloint2double((int)(unsigned)w.hi, (int)(unsigned)w.lo); }
};

// Bound of a wait on tagged words: go() is false once the wait has run `limit` SM
// clock cycles (then the global and block error flags are set; the default is about
// a second) or, looked at every 16 polls, another block has given up.
struct SpinBound {
  long long t0, limit;
  unsigned polls;
  __device__ explicit SpinBound(long long lim) {
    t0 = clock64();
    limit = lim;
    polls = 0;
  }
  __device__ bool go(int* err, volatile int* s_err) {
    if (clock64() - t0 > limit) {
      atomicExch(err, 1);
      *s_err = 1;
      return false;
    }
    if ((++polls & 15u) != 0) return true;
    if (*s_err != 0 || *(volatile int*)err != 0) {
      *s_err = 1;
      return false;
    }
    return true;
  }
};

// Every block publishes tagged words and waits only on the words it reads.
template <typename T, typename GT, int NPT, bool SMEM_G>
__global__ void __launch_bounds__(PT, 1) k_coarse_pipe(PipeArgs a) {
  using TW = Tagged<T>;
  using W = typename TW::W;
  constexpr int GB = sizeof(T) == 8 ? 4 : 8;   // exchange words in flight per batch
  extern __shared__ __align__(16) unsigned char s_raw[];
  const PipeSmem lay = PipeSmem::make<T, GT, SMEM_G>(a.max_el, a.max_nd, a.max_cp);
  GT* sG = reinterpret_cast<GT*>(s_raw);
  T* s_pt = reinterpret_cast<T*>(s_raw + lay.pt);          // operator output per sub-domain point
  T* s_m = reinterpret_cast<T*>(s_raw + lay.m);            // operator input per sub-domain node
  int32_t* s_el = reinterpret_cast<int32_t*>(s_raw + lay.el);
  int32_t* s_p2n = reinterpret_cast<int32_t*>(s_raw + lay.p2n);
  int32_t* s_cpo = reinterpret_cast<int32_t*>(s_raw + lay.cpo);
  int32_t* s_cp = reinterpret_cast<int32_t*>(s_raw + lay.cp);
  __shared__ T s_red[PW][3];
  __shared__ double s_tot[3];
  __shared__ double s_gam, s_rgam;   // gamma of the last pass and its reciprocal
  __shared__ int s_flag;             // 0 go on, 1 converged, 2 breakdown, 3 iteration cap
  __shared__ int s_err;              // a grid-wide wait ran out
  __shared__ T s_al, s_be;
  const int B = gridDim.x, bk = blockIdx.x;
  const int el0 = a.el_off[bk], nel = a.el_off[bk + 1] - el0, npt = nel * NPC3;
  const int nd0 = a.nd_off[bk], nnd = a.nd_off[bk + 1] - nd0;
  const int cp0 = a.cp_off[nd0], ncp = a.cp_off[nd0 + nnd] - cp0;
  const GT* G = static_cast<const GT*>(a.G);
  const T* bv = static_cast<const T*>(a.b);
  const T* dv = static_cast<const T*>(a.dinv);
  W* xtag = static_cast<W*>(a.xbuf);                        // [2][nL] tagged values
  W* ptag = reinterpret_cast<W*>(a.part);                   // [2][3][B] tagged partials
  if (threadIdx.x == 0) {
    s_err = 0;
    s_gam = 1.0;
  }
  for (int q = threadIdx.x; q < nel; q += PT) s_el[q] = a.el[el0 + q];
  for (int q = threadIdx.x; q < npt; q += PT) s_p2n[q] = a.p2n[(int64_t)el0 * NPC3 + q];
  for (int q = threadIdx.x; q <= nnd; q += PT) s_cpo[q] = a.cp_off[nd0 + q] - cp0;
  for (int q = threadIdx.x; q < ncp; q += PT) s_cp[q] = a.cp[cp0 + q];
  __syncthreads();
  if (SMEM_G)
    for (int q = threadIdx.x; q < nel * GF; q += PT) {
      const int k = q / GF;
      sG[q] = G[(int64_t)s_el[k] * GF + (q - k * GF)];
    }
  // element operator constants of this thread's point within its element
  const int lq = threadIdx.x & 7;
  const int i = lq & 1, j = (lq >> 1) & 1, k = lq >> 2;
  // signs of the order-1 derivative at this point's position in its element
  const T sr_ = i ? T(1) : T(-1), ss_ = j ? T(1) : T(-1), st_ = k ? T(1) : T(-1);
  const T h1q = (T)(0.25 * a.h1), h2 = (T)a.h2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // node state (slot c: node threadIdx.x + c * PT of the sub-domain)
  T x[NPT], r[NPT], u[NPT], w[NPT], z[NPT], qv[NPT], sv[NPT], p[NPT], di[NPT], mv[NPT];
  unsigned own = 0, dir = 0, live = 0;
#pragma unroll
  for (int c = 0; c < NPT; ++c) {
    const int jn = threadIdx.x + c * PT;
    x[c] = r[c] = u[c] = w[c] = z[c] = qv[c] = sv[c] = p[c] = di[c] = mv[c] = T(0);
    if (jn < nnd) {
      live |= 1u << c;
      const uint8_t fl = a.nd_fl[nd0 + jn];
      const int32_t src = a.nd_src[nd0 + jn];
      if (fl & 1) own |= 1u << c;
      if (fl & 2) {
        dir |= 1u << c;
      } else {
        di[c] = dv[src];
        r[c] = bv[src];
      }
      u[c] = di[c] * r[c];
    }
  }
  __syncthreads();   // factors staged

  // factors of chunk ch for this thread's point (global-memory factors are read
  // one chunk ahead, so their L2 latency overlaps the previous chunk's work)
  auto fetch_g = [&](int ch, T (&g)[7]) {
    const int bp = threadIdx.x + ch * PT;
    if (bp < npt) {
      const GT* gp = SMEM_G ? sG + (bp >> 3) * GF + lq : G + (int64_t)s_el[bp >> 3] * GF + lq;
#pragma unroll
      for (int k = 0; k < 7; ++k) g[k] = (T)fval(gp[8 * k]);
    } else {
#pragma unroll
      for (int k = 0; k < 7; ++k) g[k] = T(0);
    }
  };
  // s_pt = A_L s_m on the sub-domain's points; interface points are also published
  // for epoch ep
  auto apply = [&](unsigned ep) {
    const int nch = (npt + PT - 1) / PT;
    T gc[7], gn[7];
    if (!SMEM_G) fetch_g(0, gc);
    for (int ch = 0; ch < nch; ++ch) {
      const int bp = threadIdx.x + ch * PT;
      const bool lv = bp < npt;
      if (SMEM_G) fetch_g(ch, gc);
      else if (ch + 1 < nch) fetch_g(ch + 1, gn);
      const int32_t pn = lv ? s_p2n[bp] : 0;
      const T uu = lv ? s_m[pn & NODE_MASK] : T(0);
      // order 1: D-hat = [-1/2 1/2; -1/2 1/2], so each derivative is the difference
      // u(1) - u(0) of the line (times 1/2) and each transposed term the signed sum of
      // the line's two values (times 1/2); both halves are in h1q = h1 / 4
      const T ur = sr_ * (uu - __shfl_xor_sync(0xffffffffu, uu, 1));
      const T us = ss_ * (uu - __shfl_xor_sync(0xffffffffu, uu, 2));
      const T ut = st_ * (uu - __shfl_xor_sync(0xffffffffu, uu, 4));
      // G11 G12 G13 G22 G23 G33 B (zero past the last point)
      const T wr = h1q * (gc[0] * ur + gc[1] * us + gc[2] * ut);
      const T ws = h1q * (gc[1] * ur + gc[3] * us + gc[4] * ut);
      const T wt = h1q * (gc[2] * ur + gc[4] * us + gc[5] * ut);
      T wv = h2 * gc[6] * uu;
      wv += sr_ * (wr + __shfl_xor_sync(0xffffffffu, wr, 1));
      wv += ss_ * (ws + __shfl_xor_sync(0xffffffffu, ws, 2));
      wv += st_ * (wt + __shfl_xor_sync(0xffffffffu, wt, 4));
      if (lv) {
        s_pt[bp] = wv;
        if (pn < 0) {
          const size_t o = (size_t)(ep & 1u) * a.nL + (size_t)s_el[bp >> 3] * NPC3 + lq;
          TW::st(xtag + o, wv, ep);
        }
      }
      if (!SMEM_G) {
#pragma unroll
        for (int k = 0; k < 7; ++k) gc[k] = gn[k];
      }
    }
  };
  // the block's own outputs of epoch ep are in shared memory; the other blocks'
  // are awaited word by word in the gathers
  auto exchange = [&](unsigned) { __syncthreads(); };
  // assembled value of node slot c at epoch ep: every copy, in canonical order
  auto gather = [&](int c, unsigned ep) -> T {
    const int jn = threadIdx.x + c * PT;
    if (!((live >> c) & 1u) || ((dir >> c) & 1u)) return T(0);
    const int q0 = s_cpo[jn], m = s_cpo[jn + 1] - q0;
    const size_t base = (size_t)(ep & 1u) * a.nL;
    T v[8];
    if (m <= 8) {
#pragma unroll
      for (int t = 0; t < 8; ++t) v[t] = T(0);
      // the copies' words in batches of GB (registers: an FP64 word pair is 16 bytes)
#pragma unroll
      for (int h = 0; h < 8; h += GB) {
        int32_t lr[GB];
        W wd[GB];
        unsigned need = 0;
#pragma unroll
        for (int t = 0; t < GB; ++t) {
          lr[t] = 0;
          wd[t] = TW::zero();
          if (h + t < m) {
            const int32_t e = s_cp[q0 + h + t];
            if (e >= 0) {
              v[h + t] = s_pt[e];
            } else {
              lr[t] = -e - 1;
              need |= 1u << t;
            }
          }
        }
#pragma unroll
        for (int t = 0; t < GB; ++t)
          if ((need >> t) & 1u) wd[t] = TW::ld(xtag + base + lr[t]);
        SpinBound sb(a.spin);
        while (true) {
#pragma unroll
          for (int t = 0; t < GB; ++t)
            if (((need >> t) & 1u) && TW::ok(wd[t], ep)) {
              v[h + t] = TW::val(wd[t]);
              need &= ~(1u << t);
            }
          if (need == 0 || !sb.go(a.err, &s_err)) break;
#pragma unroll
          for (int t = 0; t < GB; ++t)
            if ((need >> t) & 1u) wd[t] = TW::ld(xtag + base + lr[t]);
        }
      }
      T sum = v[0];
#pragma unroll
      for (int t = 1; t < 8; ++t)
        if (t < m) sum += v[t];
      return sum;
    }
    T sum = T(0);
    for (int t = 0; t < m; ++t) {
      const int32_t e = s_cp[q0 + t];
      T vt;
      if (e >= 0) {
        vt = s_pt[e];
      } else {
        const W* wp = xtag + base + (-(int64_t)e - 1);
        W wd = TW::ld(wp);
        SpinBound sb(a.spin);
        while (!TW::ok(wd, ep) && sb.go(a.err, &s_err)) wd = TW::ld(wp);
        vt = TW::val(wd);
      }
      sum = t == 0 ? vt : sum + vt;
    }
    return sum;
  };

  unsigned epoch = 0;
  // w = A u
#pragma unroll
  for (int c = 0; c < NPT; ++c)
    if ((live >> c) & 1u) s_m[threadIdx.x + c * PT] = u[c];
  __syncthreads();
  ++epoch;
  apply(epoch);
  exchange(epoch);
#pragma unroll
  for (int c = 0; c < NPT; ++c) w[c] = gather(c, epoch);

  // scalar state, held by the first lane of the first totals warp
  double bb = 0, tol2 = 0, den_old = 0, rr = 0;
  int flag = 0, it = 0;
  for (int pass = 0;; ++pass) {
    ++epoch;
    // gamma, delta, rr over owned nodes; m = D^-1 w
    T acc[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int c = 0; c < NPT; ++c) {
      mv[c] = di[c] * w[c];
      if ((live >> c) & 1u) s_m[threadIdx.x + c * PT] = mv[c];
      if ((own >> c) & 1u) {
        acc[0] = fma(r[c], u[c], acc[0]);
        acc[1] = fma(w[c], u[c], acc[1]);
        acc[2] = fma(r[c], r[c], acc[2]);
      }
    }
#pragma unroll
    for (int t = 0; t < 3; ++t) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
      if (lane == 0) s_red[warp][t] = acc[t];
    }
    __syncthreads();
    const size_t pbase = (size_t)(epoch & 1u) * 3 * B;
    if (warp == 0) {
      // block sums of the warp sums in a fixed tree
      T v[3];
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        v[t] = lane < PW ? s_red[lane][t] : T(0);
#pragma unroll
        for (int o = PW / 2; o > 0; o >>= 1) v[t] += __shfl_xor_sync(0xffffffffu, v[t], o);
      }
      const T mine = lane == 0 ? v[0] : (lane == 1 ? v[1] : v[2]);
      if (lane < 3) TW::st(ptag + pbase + (size_t)lane * B + bk, mine, epoch);
    }
    apply(epoch);
    exchange(epoch);
    // n = QQ^T of the published outputs; the last three warps add the block partials
    // (their loads go out before the gathers), a fourth lane forms 1 / gamma_old
    const int tw = warp - (PW - 3);
    double ld[8];
    W wd[GB];
    unsigned need = 0;
    if (tw >= 0) {
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) ld[kk] = 0.0;
#pragma unroll
      for (int kk = 0; kk < GB; ++kk) {
        const int q = lane + 32 * kk;
        wd[kk] = TW::zero();
        if (q < B) {
          wd[kk] = TW::ld(ptag + pbase + (size_t)tw * B + q);
          need |= 1u << kk;
        }
      }
    }
    if (warp == PW - 4) {
      if (lane == 0 && pass > 0) s_rgam = 1.0 / s_gam;
      asm volatile("bar.arrive 1, 128;" ::: "memory");   // s_rgam is visible to the scalar step
    }
    T nv[NPT];
#pragma unroll
    for (int c = 0; c < NPT; ++c) nv[c] = gather(c, epoch);
    if (tw >= 0) {
      // block partials lane + 32 k, k < 8 (B <= 256), GB words per round
#pragma unroll
      for (int h = 0; h < 8; h += GB) {
        if (h > 0) {
          need = 0;
#pragma unroll
          for (int kk = 0; kk < GB; ++kk) {
            const int q = lane + 32 * (h + kk);
            if (q < B) {
              wd[kk] = TW::ld(ptag + pbase + (size_t)tw * B + q);
              need |= 1u << kk;
            }
          }
        }
        SpinBound sb(a.spin);
        while (true) {
#pragma unroll
          for (int kk = 0; kk < GB; ++kk)
            if (((need >> kk) & 1u) && TW::ok(wd[kk], epoch)) {
              ld[h + kk] = (double)TW::val(wd[kk]);
              need &= ~(1u << kk);
            }
          if (need == 0 || !sb.go(a.err, &s_err)) break;
#pragma unroll
          for (int kk = 0; kk < GB; ++kk)
            if ((need >> kk) & 1u) wd[kk] = TW::ld(ptag + pbase + (size_t)tw * B + lane + 32 * (h + kk));
        }
      }
      double v = ((ld[0] + ld[1]) + (ld[2] + ld[3])) + ((ld[4] + ld[5]) + (ld[6] + ld[7]));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) s_tot[tw] = v;
      // the totals warps and the 1/gamma warp meet here; the scalar step then runs
      // while the other warps still wait on their gathers
      asm volatile("bar.sync 1, 128;" ::: "memory");
    }
    if (threadIdx.x == 32 * (PW - 3)) {
      const double gnew = s_tot[0], del = s_tot[1];
      rr = s_tot[2];
      if (pass == 0) {
        bb = rr;
        tol2 = a.tol * a.tol * bb;
      }
      it = pass;
      int f = 0;
      double beta = 0, den = 0;
      T alpha = T(0);
      if (s_err != 0 || !isfinite(rr)) f = 2;
      else if (rr <= tol2) f = 1;
      else if (pass >= a.maxit) f = 3;
      else {
        // (p, A p) = delta - beta^2 (p_old, A p_old), the pipelined form of
        // delta - beta gamma / alpha_old
        beta = pass == 0 ? 0.0 : gnew * s_rgam;
        den = pass == 0 ? del : fma(-beta * beta, den_old, del);
        alpha = quotient<T>(gnew, den);
        if (!(den > 0.0) || !(gnew > 0.0) || !isfinite(alpha)) f = 2;
      }
      den_old = den;
      s_gam = gnew;
      s_flag = f;
      s_al = alpha;
      s_be = (T)beta;
    }
    __syncthreads();   // the gathers are done and the scalars are visible
    flag = s_flag;
    if (flag != 0) break;
    const T al = s_al, be = s_be;
#pragma unroll
    for (int c = 0; c < NPT; ++c) {
      z[c] = fma(be, z[c], nv[c]);
      qv[c] = fma(be, qv[c], mv[c]);
      sv[c] = fma(be, sv[c], w[c]);
      p[c] = fma(be, p[c], u[c]);
      x[c] = fma(al, p[c], x[c]);
      r[c] = fma(-al, sv[c], r[c]);
      u[c] = fma(-al, qv[c], u[c]);
      w[c] = fma(-al, z[c], w[c]);
    }
  }
  // x at every point of the sub-domain
  __syncthreads();
#pragma unroll
  for (int c = 0; c < NPT; ++c)
    if ((live >> c) & 1u) s_m[threadIdx.x + c * PT] = x[c];
  __syncthreads();
  T* xg = static_cast<T*>(a.x);
  for (int bp = threadIdx.x; bp < npt; bp += PT)
    xg[(int64_t)s_el[bp >> 3] * NPC3 + (bp & 7)] = s_m[s_p2n[bp] & NODE_MASK];
  // a block whose wait gave up holds stale values: the calling solve must stop with a
  // breakdown, whichever block saw it (every such block writes the same flags)
  if (threadIdx.x == 0 && (s_err != 0 || *(volatile int*)a.err != 0) && a.outer_sc) {
    a.outer_sc[S_BREAK] = 1;
    a.outer_sc[S_DONE] = 1;
  }
  if (bk == 0 && threadIdx.x == 32 * (PW - 3)) {
    a.sc[S_ITER] = it;
    a.sc[S_TOTAL] += it;
    a.sc[S_RR] = rr;
    a.sc[S_BB] = bb;
    a.sc[S_BREAK] = flag == 2 ? 1 : 0;
    a.sc[S_DONE] = 1;
  }
}

template <typename V>
int upload(V** dst, const std::vector<V>& src, cudaStream_t s) {
  if (cudaMalloc((void**)dst, src.size() * sizeof(V) + 16) != cudaSuccess) {
    cudaGetLastError();
    *dst = nullptr;
    set_detail("cudaMalloc failed (sub-domain coarse solve)");
    return SEM_ENOMEM;
  }
  if (!src.empty()) SEM_CUDA_TRY(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(V), cudaMemcpyHostToDevice, s));
  return SEM_OK;
}

}  // namespace

// Recursive coordinate bisection: el[0..n) goes to parts part0 .. part0 + parts - 1,
// part sizes within one of each other; each part's elements end up ascending.
void rcb(int32_t* el, int n, int parts, int part0, int32_t base, const std::vector<double>* c,
         std::vector<int32_t>& el_off) {
  if (parts == 1) {
    el_off[part0] = base;
    std::sort(el, el + n);
    return;
  }
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int q = 0; q < n; ++q)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], c[d][el[q]]);
      hi[d] = std::max(hi[d], c[d][el[q]]);
    }
  int ax = 0;
  for (int d = 1; d < 3; ++d)
    if (hi[d] - lo[d] > hi[ax] - lo[ax]) ax = d;
  const std::vector<double>& cc = c[ax];
  const int p1 = parts / 2;
  const int n1 = (int)((int64_t)n * p1 / parts);
  std::nth_element(el, el + n1, el + n,
                   [&](int32_t x, int32_t y) { return cc[x] < cc[y] || (cc[x] == cc[y] && x < y); });
  rcb(el, n1, p1, part0, base, c, el_off);
  rcb(el + n1, n - n1, parts - p1, part0 + p1, base + n1, c, el_off);
}

namespace {

// Sub-domain structures of an order-1 level, built on the host.
struct PipeHost {
  std::vector<int32_t> el_off, el, p2n, nd_off, nd_src, cp_off, cp;
  std::vector<uint8_t> nd_fl;
  int max_el = 0, max_nd = 0, max_cp = 0;
};

// Partition E order-1 elements (points 8e .. 8e + 7, canonical node node[l] < nG)
// into B sub-domains and list, per sub-domain, its nodes (in order of first
// appearance), their copies in canonical order and the published points.
int pipe_partition(int E, int64_t nG, const int32_t* node, const uint8_t* dmask, const uint8_t* owner,
                   const double* x, const double* y, const double* z, int B, PipeHost* h) {
  const int64_t nL = (int64_t)E * NPC3;
  if (E < 1 || B < 1 || B > E || nL >= (int64_t)INT32_MAX / 2) {
    set_detail("sub-domain partition: E = %d, B = %d", E, B);
    return SEM_EINVAL;
  }
  for (int64_t l = 0; l < nL; ++l)
    if (node[l] < 0 || node[l] >= nG) {
      set_detail("sub-domain partition: node index out of range at point %lld", (long long)l);
      return SEM_EINVAL;
    }
  const double* xyz[3] = {x, y, z};
  std::vector<double> cen[3];
  for (int d = 0; d < 3; ++d) {
    cen[d].assign(E, 0.0);
    for (int e = 0; e < E; ++e) {
      double t = 0;
      for (int q = 0; q < NPC3; ++q) t += xyz[d][(int64_t)e * NPC3 + q];
      cen[d][e] = t / NPC3;
    }
  }
  h->el.resize(E);
  h->el_off.assign(B + 1, 0);
  std::iota(h->el.begin(), h->el.end(), 0);
  rcb(h->el.data(), E, B, 0, 0, cen, h->el_off);
  h->el_off[B] = E;
  const std::vector<int32_t>& el = h->el;
  const std::vector<int32_t>& el_off = h->el_off;
  std::vector<int32_t> blk(E), pos(E);
  for (int b = 0; b < B; ++b)
    for (int q = el_off[b]; q < el_off[b + 1]; ++q) {
      blk[el[q]] = b;
      pos[el[q]] = q - el_off[b];
    }
  // copies of every node, ascending local index
  std::vector<int64_t> hoff(nG + 1, 0);
  for (int64_t l = 0; l < nL; ++l) ++hoff[node[l] + 1];
  for (int64_t g = 0; g < nG; ++g) hoff[g + 1] += hoff[g];
  std::vector<int32_t> hidx(nL);
  {
    std::vector<int64_t> fill(hoff.begin(), hoff.end() - 1);
    for (int64_t l = 0; l < nL; ++l) hidx[fill[node[l]]++] = (int32_t)l;
  }
  h->p2n.assign(nL, 0);
  h->nd_off.assign(B + 1, 0);
  h->nd_src.clear();
  h->nd_fl.clear();
  h->cp.clear();
  h->cp_off.assign(1, 0);
  std::vector<int32_t> local(nG, -1), list;
  for (int b = 0; b < B; ++b) {
    h->nd_off[b] = (int32_t)h->nd_src.size();
    const int64_t pbase = (int64_t)el_off[b] * NPC3;
    list.clear();
    for (int q = el_off[b]; q < el_off[b + 1]; ++q)
      for (int t = 0; t < NPC3; ++t) {
        const int32_t g = node[(int64_t)el[q] * NPC3 + t];
        if (local[g] < 0) {
          local[g] = (int32_t)list.size();
          list.push_back(g);
        }
        h->p2n[pbase + (int64_t)(q - el_off[b]) * NPC3 + t] = local[g];
      }
    const size_t cp_b = h->cp.size();
    for (int32_t g : list) {
      int32_t src = -1;
      uint8_t fl = 0;
      bool remote = false;
      const size_t first = h->cp.size();
      for (int64_t o = hoff[g]; o < hoff[g + 1]; ++o) {
        const int32_t l = hidx[o];
        const int32_t e = l / NPC3;
        if (blk[e] == b) {
          h->cp.push_back(pos[e] * NPC3 + l % NPC3);
          if (src < 0) src = l;
          if (owner[l]) fl |= 1;
        } else {
          h->cp.push_back(-(l + 1));
          remote = true;
        }
      }
      if (dmask[src]) fl |= 2;
      if (remote)
        for (size_t o = first; o < h->cp.size(); ++o)
          if (h->cp[o] >= 0) h->p2n[pbase + h->cp[o]] |= (int32_t)0x80000000u;
      h->nd_src.push_back(src);
      h->nd_fl.push_back(fl);
      h->cp_off.push_back((int32_t)h->cp.size());
      if (h->cp.size() >= (size_t)INT32_MAX / 2) {
        set_detail("sub-domain partition: too many copy entries");
        return SEM_EINVAL;
      }
    }
    for (int32_t g : list) local[g] = -1;
    h->max_el = std::max(h->max_el, el_off[b + 1] - el_off[b]);
    h->max_nd = std::max(h->max_nd, (int)list.size());
    h->max_cp = std::max(h->max_cp, (int)(h->cp.size() - cp_b));
  }
  h->nd_off[B] = (int32_t)h->nd_src.size();
  return SEM_OK;
}

}  // namespace

// Sub-domains, node lists and copy lists of an order-1 level (synchronous, host
// work O(nL)); leaves L.pp_blocks = -1 where the solve does not apply.
int coarse_pipe_build(Level& L, cudaStream_t s) {
  if (L.pp_blocks != 0) return SEM_OK;
  L.pp_blocks = -1;
  if (L.NP != NPC || L.E < 1 || L.nL >= (int64_t)INT32_MAX / 2) return SEM_OK;
  int dev = 0, nsm = 0;
  SEM_CUDA_TRY(cudaGetDevice(&dev));
  SEM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int64_t nL = L.nL;
  std::vector<double> xyz[3];
  for (auto& v : xyz) v.resize(nL);
  std::vector<int32_t> node(nL);
  std::vector<uint8_t> dmask(nL), owner(nL);
  SEM_CUDA_TRY(cudaMemcpyAsync(xyz[0].data(), L.x, nL * 8, cudaMemcpyDeviceToHost, s));
  SEM_CUDA_TRY(cudaMemcpyAsync(xyz[1].data(), L.y, nL * 8, cudaMemcpyDeviceToHost, s));
  SEM_CUDA_TRY(cudaMemcpyAsync(xyz[2].data(), L.z, nL * 8, cudaMemcpyDeviceToHost, s));
  SEM_CUDA_TRY(cudaMemcpyAsync(node.data(), L.node, nL * 4, cudaMemcpyDeviceToHost, s));
  SEM_CUDA_TRY(cudaMemcpyAsync(dmask.data(), L.dmask, nL, cudaMemcpyDeviceToHost, s));
  SEM_CUDA_TRY(cudaMemcpyAsync(owner.data(), L.owner, nL, cudaMemcpyDeviceToHost, s));
  SEM_CUDA_TRY(cudaStreamSynchronize(s));
  // one sub-domain per SM, at least 8 elements each
  const int B = std::max(1, std::min({nsm, L.E / 8, PIPE_MAX_BLOCKS}));
  PipeHost h;
  SEM_TRY(pipe_partition(L.E, L.nG, node.data(), dmask.data(), owner.data(), xyz[0].data(), xyz[1].data(),
                         xyz[2].data(), B, &h));
  SEM_TRY(upload(&L.pp_el_off, h.el_off, s));
  SEM_TRY(upload(&L.pp_el, h.el, s));
  SEM_TRY(upload(&L.pp_p2n, h.p2n, s));
  SEM_TRY(upload(&L.pp_nd_off, h.nd_off, s));
  SEM_TRY(upload(&L.pp_nd_src, h.nd_src, s));
  SEM_TRY(upload(&L.pp_nd_fl, h.nd_fl, s));
  SEM_TRY(upload(&L.pp_cp_off, h.cp_off, s));
  SEM_TRY(upload(&L.pp_cp, h.cp, s));
  // room for FP64 values: two tagged 64-bit words each
  if (cudaMalloc((void**)&L.pp_xbuf, 4 * (size_t)nL * sizeof(double) + 16) != cudaSuccess ||
      cudaMalloc((void**)&L.pp_part, 12 * (size_t)B * sizeof(double) + 16) != cudaSuccess) {
    cudaGetLastError();
    set_detail("cudaMalloc failed (sub-domain coarse solve)");
    return SEM_ENOMEM;
  }
  SEM_CUDA_TRY(cudaStreamSynchronize(s));
  L.pp_max_el = h.max_el;
  L.pp_max_nd = h.max_nd;
  L.pp_max_cp = h.max_cp;
  L.pp_nsm = nsm;
  L.pp_blocks = B;
  return SEM_OK;
}

namespace {

template <typename T, typename GT, int NPT, bool SMEM_G>
int try_launch(Level& L, const GT* G, PipeArgs& a, int nsm, cudaStream_t s, bool* used) {
  const size_t smem = PipeSmem::make<T, GT, SMEM_G>(a.max_el, a.max_nd, a.max_cp).total;
  if (smem > 220 * 1024) return SEM_OK;
  const void* f = (const void*)k_coarse_pipe<T, GT, NPT, SMEM_G>;
  // the shared-memory attribute and the occupancy are asked once per size and device,
  // so that a launch captured into a CUDA graph issues no such calls
  struct Occ {
    size_t attr_smem, occ_smem;
    int per_sm;
  };
  static PerDevice<Occ> cache;
  int dev = 0;
  SEM_TRY(current_device(&dev));
  int occ_per_sm = 0;
  {
    std::lock_guard<std::mutex> lock(cache.m);
    Occ& o = cache.v[dev];
    if (o.attr_smem < 48 * 1024) o.attr_smem = 48 * 1024;
    if (smem > o.attr_smem) {
      if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return SEM_OK;
      }
      o.attr_smem = smem;
    }
    if (o.occ_smem != smem) {
      int per_sm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, PT, smem) != cudaSuccess) {
        cudaGetLastError();
        return SEM_OK;
      }
      o.occ_smem = smem;
      o.per_sm = per_sm;
    }
    occ_per_sm = o.per_sm;
  }
  if (occ_per_sm < 1 || L.pp_blocks > occ_per_sm * nsm) return SEM_OK;
  a.G = G;
  void* args[] = {&a};
  SEM_CUDA_TRY(cudaMemsetAsync(a.err, 0, sizeof(int), s));
  // epochs start at 1, so no stale word of an earlier launch can match
  using W = typename Tagged<T>::W;
  SEM_CUDA_TRY(cudaMemsetAsync(a.xbuf, 0, 2 * (size_t)L.nL * sizeof(W), s));
  SEM_CUDA_TRY(cudaMemsetAsync(a.part, 0, 6 * (size_t)L.pp_blocks * sizeof(W), s));
  SEM_CUDA_TRY(cudaLaunchCooperativeKernel(f, dim3(L.pp_blocks), dim3(PT), args, smem, s));
  *used = true;
  return SEM_OK;
}

template <typename T, typename GT, int NPT>
int launch_npt(Level& L, const GT* G, PipeArgs& a, int nsm, cudaStream_t s, bool* used) {
  SEM_TRY((try_launch<T, GT, NPT, true>(L, G, a, nsm, s, used)));
  if (*used) return SEM_OK;
  return try_launch<T, GT, NPT, false>(L, G, a, nsm, s, used);
}

template <typename T, typename GT>
int launch_pipe(Level& L, const GT* G, PipeArgs& a, int nsm, cudaStream_t s, bool* used) {
  const int npt = (L.pp_max_nd + PT - 1) / PT;
  if (npt <= 1) return launch_npt<T, GT, 1>(L, G, a, nsm, s, used);
  if (npt <= 2) return launch_npt<T, GT, 2>(L, G, a, nsm, s, used);
  if (npt <= 4) return launch_npt<T, GT, 4>(L, G, a, nsm, s, used);
  return SEM_OK;   // larger sub-domains: the caller falls back
}

}  // namespace

// Pipelined sub-domain coarse solve at order 1 (FP64, FP32 or BF16-factor V-cycles);
// *used = false when it does not apply. err: [1].
int coarse_pipe_solve(Level& L, int prec, const void* b, void* x, const void* dinv, double h1, double h2,
                      double tol, int maxit, double* sc, int* err, double* outer_sc, cudaStream_t s, bool* used) {
  *used = false;
  if (L.NP != NPC) return SEM_OK;
  SEM_TRY(coarse_pipe_build(L, s));
  if (L.pp_blocks < 1 || L.pp_blocks > PIPE_MAX_BLOCKS) return SEM_OK;
  const int nsm = L.pp_nsm;   // read at build time: no device query inside a graph capture
  PipeArgs a{};
  a.b = b;
  a.x = x;
  a.dinv = dinv;
  a.xbuf = L.pp_xbuf;
  a.nL = L.nL;
  a.el_off = L.pp_el_off;
  a.el = L.pp_el;
  a.p2n = L.pp_p2n;
  a.nd_off = L.pp_nd_off;
  a.nd_src = L.pp_nd_src;
  a.nd_fl = L.pp_nd_fl;
  a.cp_off = L.pp_cp_off;
  a.cp = L.pp_cp;
  a.max_el = L.pp_max_el;
  a.max_nd = L.pp_max_nd;
  a.max_cp = L.pp_max_cp;
  a.h1 = h1;
  a.h2 = h2;
  a.tol = tol;
  a.maxit = maxit;
  a.part = L.pp_part;
  a.err = err;
  a.sc = sc;
  a.outer_sc = outer_sc;
  a.spin = L.spin_limit;
  // with a nodal h1 the preconditioner's coarse factors are pre-scaled (h1 = 1 here)
  if (prec == SEM_FP64) return launch_pipe<double, double>(L, L.pc_scaled ? L.pcG : L.G, a, nsm, s, used);
  if (prec == SEM_FP32) return launch_pipe<float, float>(L, L.pc_scaled ? L.pcG32 : L.G32, a, nsm, s, used);
  return launch_pipe<float, __nv_bfloat16>(L, L.pc_scaled ? L.pcG16 : L.G16, a, nsm, s, used);
}

}  // namespace sem

using namespace sem;

extern "C" int sem_coarse_partition(int32_t E, int64_t nG, const int32_t* node, const uint8_t* dmask,
                                    const uint8_t* owner, const double* x, const double* y, const double* z,
                                    int32_t nblocks, int64_t cap_nodes, int64_t cap_copies, int32_t* el_off,
                                    int32_t* el, int32_t* p2n, int32_t* nd_off, int32_t* nd_src, uint8_t* nd_fl,
                                    int32_t* cp_off, int32_t* cp, int64_t* counts) {
  if (!node || !dmask || !owner || !x || !y || !z || !el_off || !el || !p2n || !nd_off || !nd_src || !nd_fl ||
      !cp_off || !cp || !counts) {
    set_detail("sem_coarse_partition: NULL argument");
    return SEM_EINVAL;
  }
  PipeHost h;
  const int rc = pipe_partition(E, nG, node, dmask, owner, x, y, z, nblocks, &h);
  if (rc != SEM_OK) return rc;
  counts[0] = (int64_t)h.nd_src.size();
  counts[1] = (int64_t)h.cp.size();
  counts[2] = h.max_el;
  counts[3] = h.max_nd;
  counts[4] = h.max_cp;
  if (counts[0] > cap_nodes || counts[1] > cap_copies) {
    set_detail("sem_coarse_partition: %lld nodes and %lld copies exceed the capacities given",
               (long long)counts[0], (long long)counts[1]);
    return SEM_EINVAL;
  }
  std::copy(h.el_off.begin(), h.el_off.end(), el_off);
  std::copy(h.el.begin(), h.el.end(), el);
  std::copy(h.p2n.begin(), h.p2n.end(), p2n);
  std::copy(h.nd_off.begin(), h.nd_off.end(), nd_off);
  std::copy(h.nd_src.begin(), h.nd_src.end(), nd_src);
  std::copy(h.nd_fl.begin(), h.nd_fl.end(), nd_fl);
  std::copy(h.cp_off.begin(), h.cp_off.end(), cp_off);
  std::copy(h.cp.begin(), h.cp.end(), cp);
  return SEM_OK;
}
