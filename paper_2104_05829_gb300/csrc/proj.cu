// Projection of successive right-hand sides onto earlier solutions (Section
// 3.4, "projection-based initial guesses"; Fischer, CMAME 163, 1998).
//
// The space keeps an A-orthonormal basis x_1..x_l (x_i^T A x_j = delta_ij) of
// earlier solutions together with b_i = A x_i, as FP64 L-vectors (continuous,
// zero at Dirichlet nodes) in two slabs X[max][nL], AX[max][nL].
//
// * project(b): alpha_i = (x_i, b); xbar = sum_i alpha_i x_i, the A-norm-
//   closest element of the span to A^-1 b; r0 = b - sum_i alpha_i b_i, its
//   residual, with no operator application.
// * update(x, dx): the new direction v is dx (the correction the Krylov solve
//   found), or the whole solution x when the basis is full (restart). With
//   w = A v, classical Gram-Schmidt runs twice: beta_i = (x_i, w),
//   v -= sum beta_i x_i, w -= sum beta_i b_i; then v, w are scaled by
//   1/sqrt((v, w)) and appended unless (v, w) fell below PROJ_DROP times its
//   value before orthogonalisation.
//
// Every inner product is the unique-node dot (owner copies), reduced in a
// fixed order (reduce.cuh). Each pass over the basis is one multi-dot kernel
// (reads y once and NV basis vectors) and one combine kernel (reads NV
// vectors of each slab); bases of more than PROJ_CHUNK vectors take two passes.
#include <algorithm>
#include <cmath>

#include "reduce.cuh"
#include "sem_internal.cuh"

namespace sem {

namespace {

constexpr int PROJ_CHUNK = 8;
constexpr double PROJ_DROP = 1e-20;

// c[q] = (X_q, y) for q < NV; extra = (ea, eb) when ea is given.
template <int NV>
__global__ void __launch_bounds__(RED_THREADS)
    k_proj_dots(int64_t n, const double* __restrict__ X, int64_t ld, const double* __restrict__ y,
                const double* __restrict__ ea, const double* __restrict__ eb, const uint8_t* __restrict__ own,
                double* part, unsigned* ticket, double* c, double* extra) {
  Sums<NV + 1> acc;
#pragma unroll
  for (int q = 0; q <= NV; ++q) acc.v[q] = 0.0;
  GRID_LOOP(l, n) {
    if (own[l]) {
      const double yl = y[l];
#pragma unroll
      for (int q = 0; q < NV; ++q) acc.v[q] = fma(X[q * ld + l], yl, acc.v[q]);
      if (ea) acc.v[NV] = fma(ea[l], eb[l], acc.v[NV]);
    }
  }
  reduce_finish<NV + 1>(acc, part, ticket, [=] __device__(const Sums<NV + 1>& t) {
#pragma unroll
    for (int q = 0; q < NV; ++q) c[q] = t.v[q];
    if (extra) *extra = t.v[NV];
  });
}

// xo = (xb or 0) + sx * sum_q c[q] X_q ;  ro = rb - sum_q c[q] AX_q.
// DOT 1: *nrm = (xo, ro); DOT 2: *nrm = (ro, ro) (owner copies).
template <int NV, int DOT>
__global__ void __launch_bounds__(RED_THREADS)
    k_proj_combine(int64_t n, const double* __restrict__ X, const double* __restrict__ AX, int64_t ld,
                   const double* __restrict__ c, double sx, const double* xb, double* xo, const double* rb,
                   double* ro, const uint8_t* __restrict__ own, double* part, unsigned* ticket, double* nrm) {
  double cq[NV > 0 ? NV : 1];
#pragma unroll
  for (int q = 0; q < NV; ++q) cq[q] = c[q];
  Sums<1> acc{{0.0}};
  GRID_LOOP(l, n) {
    double sxv = 0.0, srv = 0.0;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      sxv = fma(cq[q], X[q * ld + l], sxv);
      srv = fma(cq[q], AX[q * ld + l], srv);
    }
    const double xv = (xb ? xb[l] : 0.0) + sx * sxv;
    const double rv = rb[l] - srv;
    xo[l] = xv;
    ro[l] = rv;
    if (DOT && own[l]) acc.v[0] = fma(DOT == 1 ? xv : rv, rv, acc.v[0]);
  }
  if (DOT) reduce_finish<1>(acc, part, ticket, [=] __device__(const Sums<1>& t) { *nrm = t.v[0]; });
}

// v *= 1/sqrt(*n2), w *= 1/sqrt(*n2)
__global__ void k_proj_scale(int64_t n, double* __restrict__ v, double* __restrict__ w, const double* n2) {
  const double s = 1.0 / sqrt(*n2);
  GRID_LOOP(l, n) {
    v[l] *= s;
    w[l] *= s;
  }
}

// u += xbar
__global__ void k_proj_add(int64_t n, double* __restrict__ u, const double* __restrict__ xbar) {
  GRID_LOOP(l, n) u[l] += xbar[l];
}

template <int NV>
void launch_dots(int64_t n, const double* X, int64_t ld, const double* y, const double* ea, const double* eb,
                 const uint8_t* own, double* part, unsigned* ticket, double* c, double* extra, cudaStream_t s) {
  k_proj_dots<NV><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, X, ld, y, ea, eb, own, part, ticket, c, extra);
}

template <int NV>
void launch_combine(int dot, int64_t n, const double* X, const double* AX, int64_t ld, const double* c, double sx,
                    const double* xb, double* xo, const double* rb, double* ro, const uint8_t* own, double* part,
                    unsigned* ticket, double* nrm, cudaStream_t s) {
  if (dot == 0)
    k_proj_combine<NV, 0><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, X, AX, ld, c, sx, xb, xo, rb, ro, own, part, ticket,
                                                            nrm);
  else if (dot == 1)
    k_proj_combine<NV, 1><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, X, AX, ld, c, sx, xb, xo, rb, ro, own, part, ticket,
                                                            nrm);
  else
    k_proj_combine<NV, 2><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, X, AX, ld, c, sx, xb, xo, rb, ro, own, part, ticket,
                                                            nrm);
}

using DotsFn = void (*)(int64_t, const double*, int64_t, const double*, const double*, const double*,
                        const uint8_t*, double*, unsigned*, double*, double*, cudaStream_t);
using CombFn = void (*)(int, int64_t, const double*, const double*, int64_t, const double*, double, const double*,
                        double*, const double*, double*, const uint8_t*, double*, unsigned*, double*, cudaStream_t);

const DotsFn kDots[PROJ_CHUNK + 1] = {launch_dots<0>, launch_dots<1>, launch_dots<2>, launch_dots<3>, launch_dots<4>,
                                      launch_dots<5>, launch_dots<6>, launch_dots<7>, launch_dots<8>};
const CombFn kComb[PROJ_CHUNK + 1] = {launch_combine<0>, launch_combine<1>, launch_combine<2>,
                                      launch_combine<3>, launch_combine<4>, launch_combine<5>,
                                      launch_combine<6>, launch_combine<7>, launch_combine<8>};

}  // namespace

struct Proj {
  Ctx* C = nullptr;
  int maxv = 0;
  int count = 0;
  int64_t nL = 0;
  double* X = nullptr;      // [maxv][nL]
  double* AX = nullptr;     // [maxv][nL]
  double* xbar = nullptr;   // [nL]
  double* c = nullptr;      // [SEM_PROJ_MAX] coefficients + 4 scalars
  double* part = nullptr;   // [RED_BLOCKS * (PROJ_CHUNK + 1)]
  unsigned* ticket = nullptr;
  double* h_sc = nullptr;   // pinned [4]
  // the operator the basis belongs to
  bool bound = false;
  double h1 = 0, h2 = 0;
  const double* h1L = nullptr;
  bool pairs = false;
};

enum ProjScal { P_BB = 0, P_RR0, P_N0, P_N2 };

inline double* pscal(Proj& P) { return P.c + SEM_PROJ_MAX; }

// c[0..count) = X^T y (chunked), with (ea, eb) in *extra when ea is given.
static int proj_dots(Proj& P, const double* y, const double* ea, const double* eb, double* extra, cudaStream_t s) {
  const Level& L = P.C->lev[0];
  int q0 = 0;
  do {
    const int nv = std::min(PROJ_CHUNK, P.count - q0);
    const bool last = q0 + nv >= P.count;
    kDots[nv](P.nL, P.X + q0 * P.nL, P.nL, y, last ? ea : nullptr, last ? eb : nullptr, L.owner, P.part, P.ticket,
              P.c + q0, last ? extra : nullptr, s);
    SEM_LAUNCH_CHECK();
    q0 += nv;
  } while (q0 < P.count);
  return SEM_OK;
}

// xo = (xb or 0) + sx X c ; ro = rb - AX c (chunked); the last chunk computes the dot `dot`.
static int proj_combine(Proj& P, double sx, const double* xb, double* xo, const double* rb, double* ro, int dot,
                        double* nrm, cudaStream_t s) {
  const Level& L = P.C->lev[0];
  int q0 = 0;
  do {
    const int nv = std::min(PROJ_CHUNK, P.count - q0);
    const bool last = q0 + nv >= P.count;
    kComb[nv](last ? dot : 0, P.nL, P.X + q0 * P.nL, P.AX + q0 * P.nL, P.nL, P.c + q0, sx, q0 == 0 ? xb : xo, xo,
              q0 == 0 ? rb : ro, ro, L.owner, P.part, P.ticket, nrm, s);
    SEM_LAUNCH_CHECK();
    q0 += nv;
  } while (q0 < P.count);
  return SEM_OK;
}

// Reset the basis if it was built for another operator; bind it to this one.
void proj_bind_coef(Proj& P, const sem_coef* c, bool pairs) {
  if (P.bound && (P.h1 != c->h1 || P.h2 != c->h2 || P.h1L != c->h1_L || P.pairs != pairs)) P.count = 0;
  P.bound = true;
  P.h1 = c->h1;
  P.h2 = c->h2;
  P.h1L = c->h1_L;
  P.pairs = pairs;
}

int proj_project(Proj& P, const double* b, double* xbar, double* r0, cudaStream_t s) {
  double* sc = pscal(P);
  SEM_TRY(proj_dots(P, b, b, b, sc + P_BB, s));
  SEM_TRY(proj_combine(P, 1.0, nullptr, xbar, b, r0, 2, sc + P_RR0, s));
  return SEM_OK;
}

// Append the direction v0 (A-orthogonalised, normalised). Synchronous.
int proj_update(Proj& P, const sem_coef* c, bool pairs, const double* x, const double* dx, int* added,
                cudaStream_t s) {
  Ctx& C = *P.C;
  Level& L = C.lev[0];
  proj_bind_coef(P, c, pairs);
  if (P.count == P.maxv) P.count = 0;
  const double* src = (P.count == 0 && x) ? x : dx;
  double* v = P.X + (int64_t)P.count * P.nL;
  double* w = P.AX + (int64_t)P.count * P.nL;
  SEM_CUDA_TRY(cudaMemcpyAsync(v, src, P.nL * 8, cudaMemcpyDeviceToDevice, s));
  if (pairs) SEM_TRY(ax_pairs_apply(L, v, w, c->h1, c->h2, c->h1_L, s));
  else SEM_TRY(ax_apply(L, SEM_FP64, v, w, c->h1, c->h2, c->h1_L, s));
  SEM_TRY(gs_apply(L, SEM_FP64, w, true, s));
  double* sc = pscal(P);
  if (P.count == 0) {
    SEM_TRY(dot_owner(C, L, SEM_FP64, v, w, sc + P_N0, s));
    SEM_CUDA_TRY(cudaMemcpyAsync(sc + P_N2, sc + P_N0, 8, cudaMemcpyDeviceToDevice, s));
  } else {
    for (int pass = 0; pass < 2; ++pass) {
      SEM_TRY(proj_dots(P, w, pass == 0 ? v : nullptr, w, sc + P_N0, s));
      SEM_TRY(proj_combine(P, -1.0, v, v, w, w, pass == 1 ? 1 : 0, sc + P_N2, s));
    }
  }
  SEM_CUDA_TRY(cudaMemcpyAsync(P.h_sc, sc, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  SEM_CUDA_TRY(cudaStreamSynchronize(s));
  const double n0 = P.h_sc[P_N0], n2 = P.h_sc[P_N2];
  const bool ok = std::isfinite(n2) && n2 > 0.0 && n2 > PROJ_DROP * n0;
  if (ok) {
    k_proj_scale<<<RED_BLOCKS * 2, 256, 0, s>>>(P.nL, v, w, sc + P_N2);
    SEM_LAUNCH_CHECK();
    ++P.count;
  }
  if (added) *added = ok ? 1 : 0;
  return SEM_OK;
}

int proj_add_xbar(Proj& P, double* u, cudaStream_t s) {
  k_proj_add<<<RED_BLOCKS * 2, 256, 0, s>>>(P.nL, u, P.xbar);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}

bool proj_belongs(const Proj& P, const Ctx* C) { return P.C == C; }

// Sizes and buffers for the projected solve; h_bb_rr0 (host, 2 values) receives
// (b, b) and (r0, r0) of the last projection (reads back; synchronous on the caller's stream).
int proj_state(const Proj& P, int* count, int* maxv, double** xbar, const double** bb_dev, double* h_bb_rr0,
               cudaStream_t s) {
  if (count) *count = P.count;
  if (maxv) *maxv = P.maxv;
  if (xbar) *xbar = P.xbar;
  if (bb_dev) *bb_dev = P.c + SEM_PROJ_MAX + P_BB;
  if (h_bb_rr0) {
    SEM_CUDA_TRY(cudaMemcpyAsync(P.h_sc, P.c + SEM_PROJ_MAX + P_BB, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    SEM_CUDA_TRY(cudaStreamSynchronize(s));
    h_bb_rr0[0] = P.h_sc[0];
    h_bb_rr0[1] = P.h_sc[1];
  }
  return SEM_OK;
}

}  // namespace sem

using namespace sem;

namespace {
Proj* proj_of(sem_proj* h) { return reinterpret_cast<Proj*>(h); }

void proj_release(Proj* P) {
  void* ptrs[] = {P->X, P->AX, P->xbar, P->c, P->part, P->ticket};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (P->h_sc) cudaFreeHost(P->h_sc);
  delete P;
}
}  // namespace

extern "C" {

int sem_proj_create(sem_ctx* h, int max_vectors, sem_proj** out) {
  if (out) *out = nullptr;
  Ctx* C = reinterpret_cast<Ctx*>(h);
  if (!C || !out || C->nlevels < 1 || max_vectors < 1 || max_vectors > SEM_PROJ_MAX) {
    set_detail("sem_proj_create: NULL context/output or max_vectors outside 1..%d", SEM_PROJ_MAX);
    return SEM_EINVAL;
  }
  Proj* P = new Proj();
  P->C = C;
  P->maxv = max_vectors;
  P->nL = C->lev[0].nL;
  const size_t slab = (size_t)max_vectors * P->nL * sizeof(double);
  bool ok = cudaMalloc(&P->X, slab) == cudaSuccess && cudaMalloc(&P->AX, slab) == cudaSuccess &&
            cudaMalloc(&P->xbar, P->nL * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&P->c, (SEM_PROJ_MAX + 4) * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&P->part, RED_BLOCKS * (PROJ_CHUNK + 1) * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&P->ticket, sizeof(unsigned)) == cudaSuccess &&
            cudaMallocHost(&P->h_sc, 4 * sizeof(double)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    proj_release(P);
    set_detail("sem_proj_create: device allocation of %zu bytes failed", 2 * slab);
    return SEM_ENOMEM;
  }
  if (cudaMemset(P->ticket, 0, sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(P->c, 0, (SEM_PROJ_MAX + 4) * sizeof(double)) != cudaSuccess) {
    proj_release(P);
    set_detail("sem_proj_create: cudaMemset failed");
    return SEM_ECUDA;
  }
  *out = reinterpret_cast<sem_proj*>(P);
  return SEM_OK;
}

void sem_proj_free(sem_proj* h) {
  if (h) proj_release(proj_of(h));
}

int sem_proj_reset(sem_proj* h) {
  Proj* P = proj_of(h);
  if (!P) {
    set_detail("sem_proj_reset: NULL space");
    return SEM_EINVAL;
  }
  P->count = 0;
  P->bound = false;
  return SEM_OK;
}

int sem_proj_count(const sem_proj* h) {
  const Proj* P = reinterpret_cast<const Proj*>(h);
  return P ? P->count : SEM_EINVAL;
}

int sem_proj_vectors(const sem_proj* h, int i, const double** x_L, const double** ax_L) {
  const Proj* P = reinterpret_cast<const Proj*>(h);
  if (!P || i < 0 || i >= P->count) {
    set_detail("sem_proj_vectors: NULL space or index outside 0..count-1");
    return SEM_EINVAL;
  }
  if (x_L) *x_L = P->X + (int64_t)i * P->nL;
  if (ax_L) *ax_L = P->AX + (int64_t)i * P->nL;
  return SEM_OK;
}

int sem_proj_project(sem_proj* h, const double* b, double* xbar, double* r0, void* stream) {
  Proj* P = proj_of(h);
  if (!P || !b || !xbar || !r0 || xbar == b || xbar == r0) {
    set_detail("sem_proj_project: NULL space or vector, or xbar aliases b/r0");
    return SEM_EINVAL;
  }
  return proj_project(*P, b, xbar, r0, (cudaStream_t)stream);
}

int sem_proj_update(sem_proj* h, const sem_coef* c, int flags, const double* x, const double* dx, int* added,
                    void* stream) {
  Proj* P = proj_of(h);
  if (!P || !c || !dx || (flags & ~SEM_OUTER_PAIRS)) {
    set_detail("sem_proj_update: NULL space, coefficients or dx, or unknown flag");
    return SEM_EINVAL;
  }
  const bool pairs = (flags & SEM_OUTER_PAIRS) != 0;
  if (pairs && !P->C->lev[0].G2) {
    set_detail("sem_proj_update: SEM_OUTER_PAIRS needs scalar h1 and the pair factors");
    return SEM_EINVAL;
  }
  return proj_update(*P, c, pairs, x, dx, added, (cudaStream_t)stream);
}

}  // extern "C"
