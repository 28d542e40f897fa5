// Vector kernels of the Krylov solvers and the Chebyshev smoother.
//
// Dot products are unique-node inner products of continuous L-vectors: the sum
// over one owner copy of every non-Dirichlet node (equal to the counting-
// weighted sum of the paper's w-weighted reductions, but with one product per
// node). Reductions are deterministic: a fixed grid of RED_BLOCKS blocks walks
// the vector with a fixed stride, each block reduces in a fixed shuffle tree,
// and the last block to finish (atomic ticket) adds the block partials in
// index order and finalises the Krylov scalars on the device. Nothing spins.
//
// Scalars (alpha, beta, residual norms) live in a device array `sc` so that a
// whole iteration runs without the host; sc[S_DONE] != 0 turns every kernel
// of that loop into a no-op (device-side convergence).
#include "reduce.cuh"
#include "sem_internal.cuh"

namespace sem {

namespace {

__device__ __forceinline__ bool skip(const double* sc) { return sc && sc[S_DONE] != 0.0; }

// ---- plain dot ---------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(RED_THREADS)
    k_dot(int64_t n, const T* __restrict__ a, const T* __restrict__ b, const uint8_t* __restrict__ own,
          double* part, unsigned* ticket, double* out) {
  struct V {
    T a, b;
    uint8_t o;
  };
  Sums<1> acc{{0}};
  grid_loop_u<4>(
      n, [&](int64_t l) { return V{a[l], b[l], own[l]}; },
      [&](int64_t, const V& v) {
        if (v.o) acc.v[0] = fma((double)v.a, (double)v.b, acc.v[0]);
      });
  reduce_finish<1>(acc, part, ticket, [=] __device__(const Sums<1>& t) { *out = t.v[0]; });
}

// ---- PCG start: r = b (- w), x = 0 unless given, p = dinv r; (b,b), (r, dinv r) ----
// bbref (device, may be null) replaces (b,b) as the reference norm^2 of the
// stopping test (a projected solve measures against the unprojected b).
template <typename T>
__global__ void __launch_bounds__(RED_THREADS)
    k_pcg_begin(int64_t n, const T* __restrict__ b, const T* __restrict__ w, T* __restrict__ x, T* __restrict__ r,
                const T* __restrict__ dinv, T* __restrict__ p, const uint8_t* __restrict__ own, double* part,
                unsigned* ticket, double* sc, double tol, const double* bbref) {
  Sums<3> acc{{0, 0, 0}};
  GRID_LOOP(l, n) {
    const T bl = b[l];
    T rl = bl;
    if (w) rl = bl - w[l];
    else x[l] = T(0);
    r[l] = rl;
    const T zl = dinv ? dinv[l] * rl : rl;
    if (p) p[l] = zl;
    if (own[l]) {
      acc.v[0] = fma((double)bl, (double)bl, acc.v[0]);
      acc.v[1] = fma((double)rl, (double)zl, acc.v[1]);
      acc.v[2] = fma((double)rl, (double)rl, acc.v[2]);
    }
  }
  reduce_finish<3>(acc, part, ticket, [=] __device__(const Sums<3>& t) {
    const double bb = bbref ? *bbref : t.v[0];
    sc[S_BB] = bb;
    sc[S_RZ] = t.v[1];
    sc[S_RR] = t.v[2];
    sc[S_TOL2] = tol * tol * bb;
    sc[S_ITER] = 0;
    sc[S_BREAK] = 0;
    sc[S_DONE] = (t.v[2] <= tol * tol * bb) ? 1.0 : 0.0;
  });
}

// ---- alpha = (r,z)/(p,w) ---------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(RED_THREADS)
    k_alpha(int64_t n, const T* __restrict__ p, const T* __restrict__ w, const uint8_t* __restrict__ own,
            double* part, unsigned* ticket, double* sc) {
  if (skip(sc)) return;
  struct V {
    T p, w;
    uint8_t o;
  };
  Sums<1> acc{{0}};
  grid_loop_u<4>(
      n, [&](int64_t l) { return V{p[l], w[l], own[l]}; },
      [&](int64_t, const V& v) {
        if (v.o) acc.v[0] = fma((double)v.p, (double)v.w, acc.v[0]);
      });
  reduce_finish<1>(acc, part, ticket, [=] __device__(const Sums<1>& t) {
    const double pw = t.v[0];
    sc[S_PW] = pw;
    if (!(pw > 0.0) || !isfinite(pw)) {
      sc[S_BREAK] = 1;
      sc[S_DONE] = 1;
      sc[S_ALPHA] = 0;
    } else {
      sc[S_ALPHA] = sc[S_RZ] / pw;
    }
  });
}

// ---- Jacobi-PCG update: x += a p, r -= a w; (r,r), (r, dinv r); beta ------------
template <typename T>
__global__ void __launch_bounds__(RED_THREADS)
    k_update_jacobi(int64_t n, T* __restrict__ x, const T* __restrict__ p, T* __restrict__ r,
                    const T* __restrict__ w, const T* __restrict__ dinv, const uint8_t* __restrict__ own,
                    double* part, unsigned* ticket, double* sc) {
  if (skip(sc)) return;
  const T a = (T)sc[S_ALPHA];
  struct V {
    T x, p, r, w, d;
    uint8_t o;
  };
  Sums<2> acc{{0, 0}};
  grid_loop_u<4>(
      n, [&](int64_t l) { return V{x[l], p[l], r[l], w[l], dinv[l], own[l]}; },
      [&](int64_t l, const V& v) {
        x[l] = fma(a, v.p, v.x);
        const T rl = fma(-a, v.w, v.r);
        r[l] = rl;
        if (v.o) {
          const double rd = (double)rl;
          acc.v[0] = fma(rd, rd, acc.v[0]);
          acc.v[1] = fma(rd, (double)(v.d * rl), acc.v[1]);
        }
      });
  reduce_finish<2>(acc, part, ticket, [=] __device__(const Sums<2>& t) {
    sc[S_RR] = t.v[0];
    sc[S_ITER] += 1;
    sc[S_TOTAL] += 1;
    sc[S_BETA] = t.v[1] / sc[S_RZ];
    sc[S_RZ] = t.v[1];
    if (!isfinite(t.v[0])) {
      sc[S_BREAK] = 1;
      sc[S_DONE] = 1;
    }
    if (t.v[0] <= sc[S_TOL2]) sc[S_DONE] = 1;
  });
}

template <typename T>
__global__ void k_direction_jacobi(int64_t n, T* __restrict__ p, const T* __restrict__ r,
                                   const T* __restrict__ dinv, const double* sc) {
  if (skip(sc)) return;
  const T beta = (T)sc[S_BETA];
  GRID_LOOP(l, n) p[l] = fma(beta, p[l], dinv[l] * r[l]);
}

// ---- flexible CG (FP64) ----------------------------------------------------------
// x += a p, r -= a w, (r, r); rb (may be null) receives r in the V-cycle's type, so
// the preconditioner reads its input without a conversion pass.
template <typename RB>
__global__ void __launch_bounds__(RED_THREADS)
    k_update_flex(int64_t n, double* __restrict__ x, const double* __restrict__ p, double* __restrict__ r,
                  const double* __restrict__ w, RB* __restrict__ rb, const uint8_t* __restrict__ own, double* part,
                  unsigned* ticket, double* sc) {
  if (skip(sc)) return;
  const double a = sc[S_ALPHA];
  struct V {
    double x, p, r, w;
    uint8_t o;
  };
  Sums<1> acc{{0}};
  grid_loop_u<4>(
      n, [&](int64_t l) { return V{x[l], p[l], r[l], w[l], own[l]}; },
      [&](int64_t l, const V& v) {
        x[l] = fma(a, v.p, v.x);
        const double rn = fma(-a, v.w, v.r);
        r[l] = rn;
        if (rb) rb[l] = (RB)rn;
        if (v.o) acc.v[0] = fma(rn, rn, acc.v[0]);
      });
  reduce_finish<1>(acc, part, ticket, [=] __device__(const Sums<1>& t) {
    sc[S_RR] = t.v[0];
    sc[S_ITER] += 1;
    if (!isfinite(t.v[0])) {
      sc[S_BREAK] = 1;
      sc[S_DONE] = 1;
    }
    if (t.v[0] <= sc[S_TOL2]) sc[S_DONE] = 1;
  });
}

// Flexible (Polak-Ribiere) beta = (z, r_new - r_old) / (z_old, r_old). With
// r_new = r_old - alpha w the numerator is -alpha (z, w), so the kernel reads w
// (still held from the operator) instead of a stored difference; w = null (the
// first direction) gives beta = 0. z is the V-cycle's output in its own type.
template <typename ZT>
__global__ void __launch_bounds__(RED_THREADS)
    k_beta_flex(int64_t n, const ZT* __restrict__ z, const double* __restrict__ r, const double* __restrict__ w,
                const uint8_t* __restrict__ own, double* part, unsigned* ticket, double* sc) {
  if (skip(sc)) return;
  struct V {
    double z, r, w;
    uint8_t o;
  };
  Sums<2> acc{{0, 0}};
  grid_loop_u<4>(
      n, [&](int64_t l) { return V{(double)z[l], r[l], w ? w[l] : 0.0, own[l]}; },
      [&](int64_t, const V& v) {
        if (v.o) {
          acc.v[0] = fma(v.z, v.r, acc.v[0]);
          acc.v[1] = fma(v.z, v.w, acc.v[1]);
        }
      });
  const bool first = w == nullptr;
  reduce_finish<2>(acc, part, ticket, [=] __device__(const Sums<2>& t) {
    const double zdr = first ? 0.0 : -sc[S_ALPHA] * t.v[1];
    sc[S_BETA] = zdr / sc[S_RZ];
    sc[S_RZ] = t.v[0];
    sc[S_ZDR] = zdr;
    if (!isfinite(t.v[0]) || !isfinite(zdr)) {
      sc[S_BREAK] = 1;
      sc[S_DONE] = 1;
    }
  });
}

template <typename ZT>
__global__ void k_direction(int64_t n, double* __restrict__ p, const ZT* __restrict__ z, const double* sc) {
  if (skip(sc)) return;
  const double beta = sc[S_BETA];
  GRID_LOOP(l, n) p[l] = fma(beta, p[l], (double)z[l]);
}

// ---- Chebyshev-Jacobi pieces (no reductions) -------------------------------------
// first step: d = inv_theta * dinv * (b - w) (w null: x was 0, r = b); x = x + d
template <typename T>
__global__ void k_cheb_first(int64_t n, const T* __restrict__ b, const T* __restrict__ w, T* __restrict__ x,
                             T* __restrict__ d, const T* __restrict__ dinv, T inv_theta, int x_zero) {
  GRID_LOOP(l, n) {
    const T r = w ? b[l] - w[l] : b[l];
    const T dl = inv_theta * (dinv[l] * r);
    d[l] = dl;
    x[l] = x_zero ? dl : x[l] + dl;
  }
}

// The FP32 forms in chunks of four (16-byte aligned vectors).
__global__ void k_cheb_first4(int64_t n, const float* __restrict__ b, const float* __restrict__ w,
                              float* __restrict__ x, float* __restrict__ d, const float* __restrict__ dinv,
                              float inv_theta, int x_zero) {
  auto one = [&](float bl, float wl, float dil, float xl) {
    const float dl = inv_theta * (dil * (w ? bl - wl : bl));
    return make_float2(dl, x_zero ? dl : xl + dl);
  };
  grid_loop_f4(
      n,
      [&](int64_t i) {
        const float4 bb = ld4(b, i), di = ld4(dinv, i);
        const float4 ww = w ? ld4(w, i) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 xx = x_zero ? make_float4(0.f, 0.f, 0.f, 0.f) : ld4(x, i);
        const float2 r0 = one(bb.x, ww.x, di.x, xx.x), r1 = one(bb.y, ww.y, di.y, xx.y);
        const float2 r2 = one(bb.z, ww.z, di.z, xx.z), r3 = one(bb.w, ww.w, di.w, xx.w);
        st4(d, i, make_float4(r0.x, r1.x, r2.x, r3.x));
        st4(x, i, make_float4(r0.y, r1.y, r2.y, r3.y));
      },
      [&](int64_t l) {
        const float2 r = one(b[l], w ? w[l] : 0.f, dinv[l], x_zero ? 0.f : x[l]);
        d[l] = r.x;
        x[l] = r.y;
      });
}

__global__ void k_cheb_step4(int64_t n, const float* __restrict__ b, const float* __restrict__ w,
                             float* __restrict__ x, float* __restrict__ d, const float* __restrict__ dinv, float c1,
                             float c2) {
  auto one = [&](float bl, float wl, float dl0, float dil, float xl) {
    const float dl = c1 * dl0 + c2 * (dil * (bl - wl));
    return make_float2(dl, xl + dl);
  };
  grid_loop_f4(
      n,
      [&](int64_t i) {
        const float4 bb = ld4(b, i), ww = ld4(w, i), dd = ld4(d, i), di = ld4(dinv, i), xx = ld4(x, i);
        const float2 r0 = one(bb.x, ww.x, dd.x, di.x, xx.x), r1 = one(bb.y, ww.y, dd.y, di.y, xx.y);
        const float2 r2 = one(bb.z, ww.z, dd.z, di.z, xx.z), r3 = one(bb.w, ww.w, dd.w, di.w, xx.w);
        st4(d, i, make_float4(r0.x, r1.x, r2.x, r3.x));
        st4(x, i, make_float4(r0.y, r1.y, r2.y, r3.y));
      },
      [&](int64_t l) {
        const float2 r = one(b[l], w[l], d[l], dinv[l], x[l]);
        d[l] = r.x;
        x[l] = r.y;
      });
}

// later steps: d = c1 d + c2 dinv (b - w); x += d
template <typename T>
__global__ void k_cheb_step(int64_t n, const T* __restrict__ b, const T* __restrict__ w, T* __restrict__ x,
                            T* __restrict__ d, const T* __restrict__ dinv, T c1, T c2) {
  GRID_LOOP(l, n) {
    const T r = b[l] - w[l];
    const T dl = c1 * d[l] + c2 * (dinv[l] * r);
    d[l] = dl;
    x[l] += dl;
  }
}

template <typename A, typename B>
__global__ void k_convert(int64_t n, const A* __restrict__ a, B* __restrict__ b) {
  GRID_LOOP(l, n) b[l] = (B)a[l];
}

template <typename T>
__global__ void k_fill(int64_t n, T* __restrict__ v, T val) {
  GRID_LOOP(l, n) v[l] = val;
}

__global__ void k_dinv(int64_t n, double* __restrict__ d, const uint8_t* __restrict__ dmask, float* __restrict__ d32) {
  GRID_LOOP(l, n) {
    const double v = dmask[l] ? 0.0 : 1.0 / d[l];
    d[l] = v;
    if (d32) d32[l] = (float)v;
  }
}

__global__ void k_rhs_mass(int64_t n, int np3, const double* __restrict__ f, const double* __restrict__ G,
                           double* __restrict__ b) {
  GRID_LOOP(l, n) {
    const int64_t e = l / np3;
    const int loc = (int)(l - e * np3);
    b[l] = G[(e * 7 + 6) * np3 + loc] * f[l];
  }
}

template <typename T>
__global__ void k_mul_cwt(int64_t n, const T* __restrict__ a, const T* __restrict__ c, T* __restrict__ o) {
  GRID_LOOP(l, n) o[l] = c[l] * a[l];
}

inline unsigned vgrid(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (unsigned)b;
}

}  // namespace

// ---------------------------------------------------------------------------------
int vec_fill(void* v, int prec, int64_t n, double val, cudaStream_t s) {
  if (prec == SEM_FP64) k_fill<double><<<vgrid(n), 256, 0, s>>>(n, (double*)v, val);
  else k_fill<float><<<vgrid(n), 256, 0, s>>>(n, (float*)v, (float)val);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}

int vec_copy_convert(const void* src, int sprec, void* dst, int dprec, int64_t n, cudaStream_t s) {
  const bool s64 = sprec == SEM_FP64, d64 = dprec == SEM_FP64;
  if (s64 && d64) SEM_CUDA_TRY(cudaMemcpyAsync(dst, src, n * 8, cudaMemcpyDeviceToDevice, s));
  else if (!s64 && !d64) SEM_CUDA_TRY(cudaMemcpyAsync(dst, src, n * 4, cudaMemcpyDeviceToDevice, s));
  else if (s64) k_convert<double, float><<<vgrid(n), 256, 0, s>>>(n, (const double*)src, (float*)dst);
  else k_convert<float, double><<<vgrid(n), 256, 0, s>>>(n, (const float*)src, (double*)dst);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}

int dot_owner(Ctx& C, const Level& L, int prec, const void* a, const void* b, double* d_out, cudaStream_t s) {
  if (prec == SEM_FP64)
    k_dot<double><<<RED_BLOCKS, RED_THREADS, 0, s>>>(L.nL, (const double*)a, (const double*)b, L.owner,
                                                     C.red_part, C.red_ticket, d_out);
  else
    k_dot<float><<<RED_BLOCKS, RED_THREADS, 0, s>>>(L.nL, (const float*)a, (const float*)b, L.owner, C.red_part,
                                                    C.red_ticket, d_out);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}

int dinv_finalize(const Level& L, double* d, float* d32, cudaStream_t s) {
  k_dinv<<<vgrid(L.nL), 256, 0, s>>>(L.nL, d, L.dmask, d32);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}

int dinv_finalize(const Level& L, double* d, cudaStream_t s) { return dinv_finalize(L, d, nullptr, s); }

int rhs_mass(const Level& L, const double* f, double* b, cudaStream_t s) {
  k_rhs_mass<<<vgrid(L.nL), 256, 0, s>>>(L.nL, L.NP * L.NP * L.NP, f, L.G, b);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}

int mul_counting_weight(const Level& L, int prec, const void* in, void* out, cudaStream_t s) {
  if (prec == SEM_FP64) k_mul_cwt<double><<<vgrid(L.nL), 256, 0, s>>>(L.nL, (const double*)in, L.cwt, (double*)out);
  else k_mul_cwt<float><<<vgrid(L.nL), 256, 0, s>>>(L.nL, (const float*)in, L.cwt32, (float*)out);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}

int pcg_begin_tol(Ctx& C, const Level& L, int prec, const void* b, const void* w, void* x, void* r,
                  const void* dinv, void* p, double* sc, double tol, cudaStream_t s, const double* bbref) {
  if (prec == SEM_FP64)
    k_pcg_begin<double><<<RED_BLOCKS, RED_THREADS, 0, s>>>(L.nL, (const double*)b, (const double*)w, (double*)x,
                                                           (double*)r, (const double*)dinv, (double*)p, L.owner,
                                                           C.red_part, C.red_ticket, sc, tol, bbref);
  else
    k_pcg_begin<float><<<RED_BLOCKS, RED_THREADS, 0, s>>>(L.nL, (const float*)b, (const float*)w, (float*)x,
                                                          (float*)r, (const float*)dinv, (float*)p, L.owner,
                                                          C.red_part, C.red_ticket, sc, tol, bbref);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}

int kr_alpha(Ctx& C, const Level& L, int prec, const void* p, const void* w, double* sc, cudaStream_t s) {
  if (prec == SEM_FP64)
    k_alpha<double><<<RED_BLOCKS, RED_THREADS, 0, s>>>(L.nL, (const double*)p, (const double*)w, L.owner,
                                                       C.red_part, C.red_ticket, sc);
  else
    k_alpha<float><<<RED_BLOCKS, RED_THREADS, 0, s>>>(L.nL, (const float*)p, (const float*)w, L.owner, C.red_part,
                                                      C.red_ticket, sc);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}

int kr_update_jacobi(Ctx& C, const Level& L, int prec, void* x, const void* p, void* r, const void* w,
                     const void* dinv, double* sc, cudaStream_t s) {
  if (prec == SEM_FP64)
    k_update_jacobi<double><<<RED_BLOCKS, RED_THREADS, 0, s>>>(L.nL, (double*)x, (const double*)p, (double*)r,
                                                               (const double*)w, (const double*)dinv, L.owner,
                                                               C.red_part, C.red_ticket, sc);
  else
    k_update_jacobi<float><<<RED_BLOCKS, RED_THREADS, 0, s>>>(L.nL, (float*)x, (const float*)p, (float*)r,
                                                              (const float*)w, (const float*)dinv, L.owner,
                                                              C.red_part, C.red_ticket, sc);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}

int kr_direction_jacobi(const Level& L, int prec, void* p, const void* r, const void* dinv, double* sc,
                        cudaStream_t s) {
  if (prec == SEM_FP64)
    k_direction_jacobi<double><<<vgrid(L.nL), 256, 0, s>>>(L.nL, (double*)p, (const double*)r,
                                                           (const double*)dinv, sc);
  else
    k_direction_jacobi<float><<<vgrid(L.nL), 256, 0, s>>>(L.nL, (float*)p, (const float*)r, (const float*)dinv,
                                                          sc);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}

int kr_update_flex(Ctx& C, const Level& L, double* x, const double* p, double* r, const double* w, void* rb,
                   int rb_prec, double* sc, cudaStream_t s) {
  if (rb_prec == SEM_FP64)
    k_update_flex<double><<<RED_BLOCKS, RED_THREADS, 0, s>>>(L.nL, x, p, r, w, (double*)rb, L.owner, C.red_part,
                                                             C.red_ticket, sc);
  else
    k_update_flex<float><<<RED_BLOCKS, RED_THREADS, 0, s>>>(L.nL, x, p, r, w, (float*)rb, L.owner, C.red_part,
                                                            C.red_ticket, sc);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}

int kr_beta_flex(Ctx& C, const Level& L, const void* z, int z_prec, const double* r, const double* w, double* sc,
                 cudaStream_t s) {
  if (z_prec == SEM_FP64)
    k_beta_flex<double><<<RED_BLOCKS, RED_THREADS, 0, s>>>(L.nL, (const double*)z, r, w, L.owner, C.red_part,
                                                           C.red_ticket, sc);
  else
    k_beta_flex<float><<<RED_BLOCKS, RED_THREADS, 0, s>>>(L.nL, (const float*)z, r, w, L.owner, C.red_part,
                                                          C.red_ticket, sc);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}

int kr_direction(const Level& L, double* p, const void* z, int z_prec, double* sc, cudaStream_t s) {
  if (z_prec == SEM_FP64) k_direction<double><<<vgrid(L.nL), 256, 0, s>>>(L.nL, p, (const double*)z, sc);
  else k_direction<float><<<vgrid(L.nL), 256, 0, s>>>(L.nL, p, (const float*)z, sc);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}

int cheb_first(const Level& L, int prec, const void* b, const void* w, void* x, void* d, bool x_zero,
               double inv_theta, cudaStream_t s) {
  if (prec == SEM_FP64)
    k_cheb_first<double><<<vgrid(L.nL), 256, 0, s>>>(L.nL, (const double*)b, (const double*)w, (double*)x,
                                                     (double*)d, L.dinv, inv_theta, x_zero ? 1 : 0);
  else if (kVec4 && aligned16({b, w, x, d, L.dinv32}))
    k_cheb_first4<<<vgrid(L.nL / 4), 256, 0, s>>>(L.nL, (const float*)b, (const float*)w, (float*)x, (float*)d,
                                                  L.dinv32, (float)inv_theta, x_zero ? 1 : 0);
  else
    k_cheb_first<float><<<vgrid(L.nL), 256, 0, s>>>(L.nL, (const float*)b, (const float*)w, (float*)x, (float*)d,
                                                    L.dinv32, (float)inv_theta, x_zero ? 1 : 0);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}

int cheb_step(const Level& L, int prec, const void* b, const void* w, void* x, void* d, double c1, double c2,
              cudaStream_t s) {
  if (prec == SEM_FP64)
    k_cheb_step<double><<<vgrid(L.nL), 256, 0, s>>>(L.nL, (const double*)b, (const double*)w, (double*)x,
                                                    (double*)d, L.dinv, c1, c2);
  else if (kVec4 && aligned16({b, w, x, d, L.dinv32}))
    k_cheb_step4<<<vgrid(L.nL / 4), 256, 0, s>>>(L.nL, (const float*)b, (const float*)w, (float*)x, (float*)d,
                                                 L.dinv32, (float)c1, (float)c2);
  else
    k_cheb_step<float><<<vgrid(L.nL), 256, 0, s>>>(L.nL, (const float*)b, (const float*)w, (float*)x, (float*)d,
                                                   L.dinv32, (float)c1, (float)c2);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}

}  // namespace sem
