// Solvers and the remaining entry points.
//
// * Jacobi-PCG (the viscous-substep solver of Section 2.2) and flexible PCG
//   preconditioned by a p-multigrid V-cycle (Section 3.4, "Poisson Solve Preconditioning":
//   orders N, N/2, ..., 1, Chebyshev-accelerated Jacobi smoothing on every level
//   but the coarsest, a Jacobi-PCG coarse solve). FP64 outer iteration; the
//   V-cycle runs in FP64, FP32 or FP32 with BF16 geometric factors.
// * Chebyshev-Jacobi of degree k (Saad's three-term Chebyshev recurrence):
//   theta = (lmax+lmin)/2, delta = (lmax-lmin)/2, sigma = theta/delta;
//   d = D^-1 r / theta, x += d; then r = b - A x, rho' = 1/(2 sigma - rho),
//   d = rho' rho d + (2 rho'/delta) D^-1 r, x += d.
// * The interval is [lmin_factor, lmax_factor] * lambda_est, with lambda_est the
//   largest Ritz value of a few Lanczos steps on D^-1/2 A D^-1/2 from a seeded
//   SplitMix64 start vector.
#include <cmath>
#include <vector>

#include "sem_internal.cuh"

namespace sem {

namespace {

__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t c) {
  uint64_t z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

#define GRID_LOOP(l, n) \
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < (n); l += (int64_t)gridDim.x * blockDim.x)

inline unsigned vgrid(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (unsigned)b;
}

// v = U[-1,1) drawn at the node's smallest local index, 0 at Dirichlet nodes
__global__ void k_lanczos_start(int64_t n, const int32_t* __restrict__ label, const uint8_t* __restrict__ dmask,
                                uint64_t seed, double* __restrict__ v) {
  GRID_LOOP(l, n) {
    const uint64_t z = splitmix64(seed, (uint64_t)label[l]);
    const double u = (double)(z >> 11) * 0x1.0p-53;
    v[l] = dmask[l] ? 0.0 : 2.0 * u - 1.0;
  }
}

__global__ void k_scale(int64_t n, double* __restrict__ v, const double* __restrict__ nrm2) {
  const double c = 1.0 / sqrt(*nrm2);
  GRID_LOOP(l, n) v[l] *= c;
}

__global__ void k_sqrt_mul(int64_t n, const double* __restrict__ dinv, const double* __restrict__ v,
                           double* __restrict__ t) {
  GRID_LOOP(l, n) t[l] = sqrt(dinv[l]) * v[l];
}

// w = sqrt(dinv) * w - beta * vprev
__global__ void k_lanczos_w(int64_t n, const double* __restrict__ dinv, double* __restrict__ w,
                            const double* __restrict__ vprev, double beta) {
  GRID_LOOP(l, n) w[l] = sqrt(dinv[l]) * w[l] - beta * vprev[l];
}

// w -= alpha v
__global__ void k_axpy_dev(int64_t n, double* __restrict__ w, const double* __restrict__ v, double alpha) {
  GRID_LOOP(l, n) w[l] -= alpha * v[l];
}

// vprev = v; v = w / beta
__global__ void k_lanczos_shift(int64_t n, double* __restrict__ vprev, double* __restrict__ v,
                                const double* __restrict__ w, double inv_beta) {
  GRID_LOOP(l, n) {
    vprev[l] = v[l];
    v[l] = w[l] * inv_beta;
  }
}

// Factors of the coarsest level with the stiffness parts scaled by the nodal h1 (point by
// point: the GLL quadrature of h1 G), B copied, in FP64 and the low-precision copies that exist.
__global__ void k_scale_factors(int64_t n, int np3, const double* __restrict__ G, const double* __restrict__ h1,
                                double* __restrict__ out, float* __restrict__ out32,
                                __nv_bfloat16* __restrict__ out16) {
  GRID_LOOP(p, n) {
    const int64_t e = p / np3;
    const int loc = (int)(p - e * np3);
    const double hp = h1[p];
    for (int c = 0; c < 7; ++c) {
      const int64_t q = (e * 7 + c) * np3 + loc;
      const double v = c < 6 ? G[q] * hp : G[q];
      out[q] = v;
      if (out32) out32[q] = __double2float_rn(v);
      if (out16) out16[q] = __double2bfloat16(v);
    }
  }
}

template <typename T>
int alloc_once(T** p, size_t count) {
  if (*p) return SEM_OK;
  if (cudaMalloc((void**)p, count * sizeof(T) + 16) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    set_detail("cudaMalloc of %zu bytes failed (nodal preconditioner)", count * sizeof(T));
    return SEM_ENOMEM;
  }
  return SEM_OK;
}

// Largest eigenvalue of the symmetric tridiagonal (a, b) by Sturm-sequence bisection.
double tridiag_max_eig(const std::vector<double>& a, const std::vector<double>& b) {
  const int m = (int)a.size();
  double lo = a[0], hi = a[0];
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i < m - 1 ? std::fabs(b[i]) : 0.0);
    lo = std::fmin(lo, a[i] - r);
    hi = std::fmax(hi, a[i] + r);
  }
  auto count_below = [&](double x) {   // eigenvalues < x
    int cnt = 0;
    double q = a[0] - x;
    if (q < 0) ++cnt;
    for (int i = 1; i < m; ++i) {
      if (q == 0.0) q = 1e-300;
      q = a[i] - x - b[i - 1] * b[i - 1] / q;
      if (q < 0) ++cnt;
    }
    return cnt;
  };
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (count_below(mid) >= m) hi = mid;
    else lo = mid;
    if (hi - lo <= 1e-15 * std::fabs(hi)) break;
  }
  return 0.5 * (lo + hi);
}

// the preconditioner's operator on level l (a nodal h1 of the preconditioner replaces h1)
int level_op(Ctx& C, int l, int prec, const void* x, void* w, double h1, double h2, cudaStream_t s,
             const double* skip = nullptr) {
  const Level& L = C.lev[l];
  SEM_TRY(ax_apply(L, prec, x, w, h1, h2, C.pc_nodal ? L.h1n : nullptr, s, skip));
  return gs_apply_skip(L, prec, w, true, skip, s);
}

int read_scalars(Ctx& C, int slot, cudaStream_t s) {
  SEM_CUDA_TRY(cudaMemcpyAsync(C.h_scal + slot * S_NSLOTS, C.scal + slot * S_NSLOTS, S_NSLOTS * sizeof(double),
                               cudaMemcpyDeviceToHost, s));
  SEM_CUDA_TRY(cudaStreamSynchronize(s));
  return SEM_OK;
}

// dinv on level l for (h1, h2): exact local diagonal, gs-summed, inverted, 0 at Dirichlet nodes.
int level_dinv(Ctx& C, int l, double h1, double h2, const double* h1L, double* out, float* out32, cudaStream_t s) {
  const Level& L = C.lev[l];
  SEM_TRY(diag_local(L, h1, h2, h1L, out, s));
  SEM_TRY(gs_apply(L, SEM_FP64, out, false, s));
  return dinv_finalize(L, out, out32, s);
}

int lanczos(Ctx& C, int l, double h1, double h2, cudaStream_t s, double* lam) {
  Level& L = C.lev[l];
  const int64_t n = L.nL;
  double *v = L.vb, *vprev = L.vx, *w = L.vw, *t = L.vd;
  double* d_tmp = C.scal + 3 * S_NSLOTS;   // spare slot set
  k_lanczos_start<<<vgrid(n), 256, 0, s>>>(n, L.label, L.dmask, C.opts.lanczos_seed, v);
  SEM_LAUNCH_CHECK();
  SEM_CUDA_TRY(cudaMemsetAsync(vprev, 0, n * 8, s));
  SEM_TRY(dot_owner(C, L, SEM_FP64, v, v, d_tmp, s));
  k_scale<<<vgrid(n), 256, 0, s>>>(n, v, d_tmp);
  SEM_LAUNCH_CHECK();
  std::vector<double> al, be;
  double beta = 0.0;
  for (int j = 0; j < C.opts.lanczos_steps; ++j) {
    k_sqrt_mul<<<vgrid(n), 256, 0, s>>>(n, L.dinv, v, t);
    SEM_LAUNCH_CHECK();
    SEM_TRY(level_op(C, l, SEM_FP64, t, w, h1, h2, s));
    k_lanczos_w<<<vgrid(n), 256, 0, s>>>(n, L.dinv, w, vprev, beta);
    SEM_LAUNCH_CHECK();
    SEM_TRY(dot_owner(C, L, SEM_FP64, w, v, d_tmp, s));
    double alpha = 0;
    SEM_CUDA_TRY(cudaMemcpyAsync(&alpha, d_tmp, 8, cudaMemcpyDeviceToHost, s));
    SEM_CUDA_TRY(cudaStreamSynchronize(s));
    k_axpy_dev<<<vgrid(n), 256, 0, s>>>(n, w, v, alpha);
    SEM_LAUNCH_CHECK();
    al.push_back(alpha);
    SEM_TRY(dot_owner(C, L, SEM_FP64, w, w, d_tmp, s));
    double b2 = 0;
    SEM_CUDA_TRY(cudaMemcpyAsync(&b2, d_tmp, 8, cudaMemcpyDeviceToHost, s));
    SEM_CUDA_TRY(cudaStreamSynchronize(s));
    beta = std::sqrt(b2);
    if (j == C.opts.lanczos_steps - 1 || beta == 0.0) break;
    be.push_back(beta);
    k_lanczos_shift<<<vgrid(n), 256, 0, s>>>(n, vprev, v, w, 1.0 / beta);
    SEM_LAUNCH_CHECK();
  }
  *lam = tridiag_max_eig(al, be);
  if (!(*lam > 0.0) || !std::isfinite(*lam)) {
    set_detail("eigenvalue estimate failed on level %d", l);
    return SEM_EBREAKDOWN;
  }
  return SEM_OK;
}

struct VecSet {
  void *b, *x, *r, *d, *w, *p;
  const void* dinv;
};

VecSet vecs(Level& L, int prec) {
  if (prec == SEM_FP64) return {L.vb, L.vx, L.vr, L.vd, L.vw, L.cp, L.dinv};
  return {L.fb, L.fx, L.fr, L.fd, L.fw, L.cpf, L.dinv32};
}

// Chebyshev-accelerated weighted Schwarz (CHEBY-ASM): the Chebyshev-Jacobi
// recurrence with D^-1 r replaced by the Schwarz output W z, z = asm_sum(b - A x);
// the Schwarz output lives in the level's r vector (unused on smoothed levels).
int cheb_asm(Ctx& C, int l, int prec, const void* b, void* x, bool x_zero, cudaStream_t s) {
  Level& L = C.lev[l];
  VecSet v = vecs(L, prec);
  const double lmin = C.opts.cheb_lmin_factor * L.lmax, lmax = C.opts.cheb_lmax_factor * L.lmax;
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  if (!x_zero) SEM_TRY(level_op(C, l, prec, x, v.w, C.pc_h1, C.pc_h2, s));
  SEM_TRY(asm_sum(L, prec, b, x_zero ? nullptr : v.w, v.r, C.pc_h1, C.pc_h2, s));
  SEM_TRY(cheb_w_update(L, prec, v.r, x, v.d, 0.0, 1.0 / theta, true, x_zero, s));
  for (int j = 1; j < C.opts.cheb_degree; ++j) {
    SEM_TRY(level_op(C, l, prec, x, v.w, C.pc_h1, C.pc_h2, s));
    SEM_TRY(asm_sum(L, prec, b, v.w, v.r, C.pc_h1, C.pc_h2, s));
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    SEM_TRY(cheb_w_update(L, prec, v.r, x, v.d, rho_new * rho, 2.0 * rho_new / delta, false, false, s));
    rho = rho_new;
  }
  return SEM_OK;
}

int cheb(Ctx& C, int l, int prec, const void* b, void* x, bool x_zero, cudaStream_t s) {
  if (C.opts.smoother == SEM_SMOOTH_ASM) return cheb_asm(C, l, prec, b, x, x_zero, s);
  Level& L = C.lev[l];
  VecSet v = vecs(L, prec);
  const double lmin = C.opts.cheb_lmin_factor * L.lmax, lmax = C.opts.cheb_lmax_factor * L.lmax;
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  if (x_zero) {
    SEM_TRY(cheb_first(L, prec, b, nullptr, x, v.d, true, 1.0 / theta, s));
  } else {
    SEM_TRY(level_op(C, l, prec, x, v.w, C.pc_h1, C.pc_h2, s));
    SEM_TRY(cheb_first(L, prec, b, v.w, x, v.d, false, 1.0 / theta, s));
  }
  for (int j = 1; j < C.opts.cheb_degree; ++j) {
    SEM_TRY(level_op(C, l, prec, x, v.w, C.pc_h1, C.pc_h2, s));
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    SEM_TRY(cheb_step(L, prec, b, v.w, x, v.d, rho_new * rho, 2.0 * rho_new / delta, s));
    rho = rho_new;
  }
  return SEM_OK;
}

// Coarsest level: Jacobi-PCG from zero to coarse_tol or coarse_maxit, entirely
// on the device (every launch after convergence returns at once).
int coarse_solve(Ctx& C, int l, int prec, const void* b, void* x, cudaStream_t s) {
  Level& L = C.lev[l];
  VecSet v = vecs(L, prec);
  double* sc = C.scal + 1 * S_NSLOTS;
  // order 1: the whole solve in one cooperative launch, pipelined on one
  // sub-domain per SM, when the sub-domains fit; else the batched kernels below
  bool used = false;
  const int mode = C.opts.coarse_mode;
  if (mode == SEM_COARSE_AUTO || mode == SEM_COARSE_PIPE)
    SEM_TRY(coarse_pipe_solve(L, prec, b, x, v.dinv, C.pc_h1, C.pc_h2, C.opts.coarse_tol, C.opts.coarse_maxit, sc,
                              C.cg_err, C.scal, s, &used));
  if (used) return SEM_OK;
  SEM_TRY(pcg_begin_tol(C, L, prec, b, nullptr, x, v.r, v.dinv, v.p, sc, C.opts.coarse_tol, s));
  // Iterations go out in batches. After each batch the device's "done" flag is
  // copied to pinned host memory; the host looks at the previous batch's flag
  // while the current batch runs, and stops launching once it is set. Launches
  // that follow convergence return at once, so the result does not depend on
  // where the host stops.
  constexpr int BATCH = 6;
  int launched = 0, q = 0;
  bool pending = false;
  while (launched < C.opts.coarse_maxit) {
    const int nb = std::min(BATCH, C.opts.coarse_maxit - launched);
    for (int it = 0; it < nb; ++it) {
      SEM_TRY(level_op(C, l, prec, v.p, v.w, C.pc_h1, C.pc_h2, s, sc + S_DONE));
      SEM_TRY(kr_alpha(C, L, prec, v.p, v.w, sc, s));
      SEM_TRY(kr_update_jacobi(C, L, prec, x, v.p, v.r, v.w, v.dinv, sc, s));
      SEM_TRY(kr_direction_jacobi(L, prec, v.p, v.r, v.dinv, sc, s));
    }
    launched += nb;
    SEM_CUDA_TRY(cudaMemcpyAsync(C.h_done + q, sc + S_DONE, sizeof(double), cudaMemcpyDeviceToHost, s));
    SEM_CUDA_TRY(cudaEventRecord(C.cev[q], s));
    if (pending) {
      SEM_CUDA_TRY(cudaEventSynchronize(C.cev[1 - q]));
      if (C.h_done[1 - q] != 0.0) break;
    }
    pending = true;
    q = 1 - q;
  }
  return SEM_OK;
}

int vcycle_level(Ctx& C, int l, int prec, cudaStream_t s) {
  Level& L = C.lev[l];
  VecSet v = vecs(L, prec);
  if (l == C.nlevels - 1) return coarse_solve(C, l, prec, v.b, v.x, s);
  Level& Cl = C.lev[l + 1];
  VecSet vc = vecs(Cl, prec);
  SEM_TRY(cheb(C, l, prec, v.b, v.x, true, s));
  SEM_TRY(level_op(C, l, prec, v.x, v.w, C.pc_h1, C.pc_h2, s));
  SEM_TRY(restrict_residual(L, Cl, prec, v.b, v.w, vc.b, s));
  SEM_TRY(gs_apply(Cl, prec, vc.b, true, s));
  SEM_TRY(vcycle_level(C, l + 1, prec, s));
  SEM_TRY(interp_add(L, Cl, prec, vc.x, v.x, s));
  return cheb(C, l, prec, v.b, v.x, false, s);
}

}  // namespace

int precond_setup(Ctx& C, double h1, double h2, int prec, cudaStream_t s, const double* h1L) {
  if (h1L && C.opts.smoother != SEM_SMOOTH_JACOBI) {
    set_detail("a nodal h1 needs the Chebyshev-Jacobi smoother (the Schwarz local solves take a scalar h1)");
    return SEM_EINVAL;
  }
  if (prec != SEM_FP64 && !C.lev[0].dinv32) {
    set_detail("FP32 preconditioner copies were not built");
    return SEM_EINVAL;
  }
  if (prec == SEM_FP32 && !C.lev[0].G32) {
    set_detail("FP32 factors were not built");
    return SEM_EINVAL;
  }
  if (prec == SEM_BF16G && !C.lev[0].G16) {
    set_detail("BF16 factors were not built");
    return SEM_EINVAL;
  }
  C.pc_ready = false;
  ++C.pc_gen;
  // a nodal h1: the fine values, then each coarser level's from the level above; the
  // level operators take it point by point (the scalar h1 becomes 1)
  C.pc_nodal = h1L != nullptr;
  C.pc_h1L = h1L;
  if (h1L) {
    h1 = 1.0;
    for (int l = 0; l < C.nlevels; ++l) {
      Level& L = C.lev[l];
      SEM_TRY(alloc_once(&L.h1n, (size_t)L.nL));
      if (l == 0) SEM_CUDA_TRY(cudaMemcpyAsync(L.h1n, h1L, L.nL * sizeof(double), cudaMemcpyDeviceToDevice, s));
      else SEM_TRY(interp_nodal(C.lev[l - 1], L, C.lev[l - 1].h1n, L.h1n, s));
    }
  }
  for (int l = 0; l < C.nlevels; ++l) {
    Level& L = C.lev[l];
    L.pc_scaled = false;
    SEM_TRY(level_dinv(C, l, h1, h2, C.pc_nodal ? L.h1n : nullptr, L.dinv, L.dinv32, s));
    if (l == C.nlevels - 1) {
      if (C.opts.coarse_mode == SEM_COARSE_AUTO || C.opts.coarse_mode == SEM_COARSE_PIPE)
        SEM_TRY(coarse_pipe_build(L, s));
      if (C.pc_nodal) {
        // the one-launch coarse solve takes a scalar h1: give it h1-scaled factors
        const size_t nf = (size_t)7 * L.nL;
        SEM_TRY(alloc_once(&L.pcG, nf));
        if (L.G32) SEM_TRY(alloc_once(&L.pcG32, nf));
        if (L.G16) SEM_TRY(alloc_once(&L.pcG16, nf));
        k_scale_factors<<<vgrid(L.nL), 256, 0, s>>>(L.nL, L.NP * L.NP * L.NP, L.G, L.h1n, L.pcG,
                                                    L.G32 ? L.pcG32 : nullptr, L.G16 ? L.pcG16 : nullptr);
        SEM_LAUNCH_CHECK();
        L.pc_scaled = true;
      }
      continue;
    }
    if (C.opts.smoother == SEM_SMOOTH_ASM) {
      SEM_TRY(schwarz_build(C, L, s));
      k_lanczos_start<<<vgrid(L.nL), 256, 0, s>>>(L.nL, L.label, L.dmask, C.opts.lanczos_seed, L.vb);
      SEM_LAUNCH_CHECK();
      SEM_TRY(arnoldi_lmax_asm(C, l, h1, h2, L.vb, C.opts.lanczos_steps, s, &L.lmax));
    } else {
      SEM_TRY(lanczos(C, l, h1, h2, s, &L.lmax));
    }
  }
  SEM_CUDA_TRY(cudaStreamSynchronize(s));
  C.pc_h1 = h1;
  C.pc_h2 = h2;
  C.pc_prec = prec;
  C.pc_ready = true;
  return SEM_OK;
}

// Preconditioner step of a flexible-CG iteration: z = V-cycle(r) (input already in
// the finest level's b, output in its x), beta and the new direction. After the
// first call with given pointers it is captured once on the library's capture
// stream and replayed as a CUDA graph on s (about 45 launches become one). The
// caller runs the same step directly at least once before (the first V-cycle of
// the solve), so one-time set-up calls never happen inside a capture. A capture
// that fails (a coarse execution that waits on the host, say) switches the
// context to direct launches.
int precond_step(Ctx& C, int prec, const void* zx, int zprec, const double* w, double* sc, cudaStream_t s) {
  const Level& L = C.lev[0];
  auto direct = [&](cudaStream_t st) -> int {
    SEM_TRY(vcycle_level(C, 0, prec, st));
    SEM_TRY(kr_beta_flex(C, L, zx, zprec, C.r, w, sc, st));
    return kr_direction(L, C.p, zx, zprec, sc, st);
  };
  if (C.pc_graph_off || !C.cap_stream) return direct(s);
  const bool match = C.pc_graph && C.pc_graph_prec == prec && C.pc_graph_gen == C.pc_gen &&
                     C.pc_graph_key[0] == w && C.pc_graph_key[1] == sc && C.pc_graph_key[2] == zx;
  if (!match) {
    if (C.pc_graph) {
      cudaGraphExecDestroy(C.pc_graph);
      C.pc_graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(C.cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      C.pc_graph_off = true;
      return direct(s);
    }
    const int rc = direct(C.cap_stream);
    const cudaError_t e = cudaStreamEndCapture(C.cap_stream, &g);
    cudaError_t ei = cudaErrorUnknown;
    if (rc == SEM_OK && e == cudaSuccess && g) ei = cudaGraphInstantiate(&C.pc_graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      cudaGetLastError();
      C.pc_graph = nullptr;
      C.pc_graph_off = true;
      return direct(s);
    }
    C.pc_graph_prec = prec;
    C.pc_graph_gen = C.pc_gen;
    C.pc_graph_key[0] = w;
    C.pc_graph_key[1] = sc;
    C.pc_graph_key[2] = zx;
  }
  SEM_CUDA_TRY(cudaGraphLaunch(C.pc_graph, s));
  ++C.graph_steps;
  return SEM_OK;
}

int vcycle(Ctx& C, int prec, const double* r, double* z, cudaStream_t s) {
  Level& L = C.lev[0];
  VecSet v = vecs(L, prec);
  SEM_TRY(vec_copy_convert(r, SEM_FP64, v.b, prec == SEM_FP64 ? SEM_FP64 : SEM_FP32, L.nL, s));
  SEM_TRY(vcycle_level(C, 0, prec, s));
  return vec_copy_convert(v.x, prec == SEM_FP64 ? SEM_FP64 : SEM_FP32, z, SEM_FP64, L.nL, s);
}

}  // namespace sem

using namespace sem;

namespace {

Ctx* ctx_of(sem_ctx* h) { return reinterpret_cast<Ctx*>(h); }

int check_level(Ctx* C, int level) {
  if (!C) {
    set_detail("context is NULL");
    return SEM_EINVAL;
  }
  if (level < 0 || level >= C->nlevels) {
    set_detail("level %d outside 0..%d", level, C->nlevels - 1);
    return SEM_EINVAL;
  }
  return SEM_OK;
}

int check_prec(Ctx* C, int level, int prec) {
  const Level& L = C->lev[level];
  if (prec == SEM_FP64) return SEM_OK;
  if (prec == SEM_FP64P && L.G2) return SEM_OK;
  if (prec == SEM_FP32 && L.G32) return SEM_OK;
  if (prec == SEM_BF16G && L.G16) return SEM_OK;
  set_detail("precision %d not available (not built or unknown)", prec);
  return SEM_EINVAL;
}

}  // namespace

extern "C" {

int sem_ax(sem_ctx* h, const double* u, double* w, const sem_coef* c, int flags, void* stream) {
  Ctx* C = ctx_of(h);
  SEM_TRY(check_level(C, 0));
  if (!u || !w || !c || u == w || (flags & ~(SEM_AX_ASSEMBLE | SEM_AX_PAIRS))) {
    set_detail("sem_ax: NULL or aliased vector, NULL coefficients or unknown flag");
    return SEM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (flags & SEM_AX_PAIRS) SEM_TRY(ax_pairs_apply(C->lev[0], u, w, c->h1, c->h2, c->h1_L, s));
  else SEM_TRY(ax_apply(C->lev[0], SEM_FP64, u, w, c->h1, c->h2, c->h1_L, s));
  if (flags & SEM_AX_ASSEMBLE) SEM_TRY(gs_apply(C->lev[0], SEM_FP64, w, true, s));
  return SEM_OK;
}

int sem_gs(sem_ctx* h, double* w, int flags, void* stream) {
  Ctx* C = ctx_of(h);
  SEM_TRY(check_level(C, 0));
  if (!w || (flags & ~SEM_GS_ADD_MASK)) {
    set_detail("sem_gs: NULL vector or unknown flag");
    return SEM_EINVAL;
  }
  return gs_apply(C->lev[0], SEM_FP64, w, (flags & SEM_GS_ADD_MASK) != 0, (cudaStream_t)stream);
}

int sem_level_ax(sem_ctx* h, int level, int prec, const void* u, void* w, double h1, double h2, int flags,
                 void* stream) {
  Ctx* C = ctx_of(h);
  SEM_TRY(check_level(C, level));
  SEM_TRY(check_prec(C, level, prec));
  if (!u || !w || u == w || (flags & ~SEM_AX_ASSEMBLE)) {
    set_detail("sem_level_ax: NULL or aliased vector or unknown flag");
    return SEM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == SEM_FP64P) SEM_TRY(ax_pairs_apply(C->lev[level], (const double*)u, (double*)w, h1, h2, nullptr, s));
  else SEM_TRY(ax_apply(C->lev[level], prec, u, w, h1, h2, nullptr, s));
  const int vprec = (prec == SEM_FP64P) ? SEM_FP64 : prec;
  if (flags & SEM_AX_ASSEMBLE) SEM_TRY(gs_apply(C->lev[level], vprec, w, true, s));
  return SEM_OK;
}

int sem_level_gs(sem_ctx* h, int level, int prec, void* w, int flags, void* stream) {
  Ctx* C = ctx_of(h);
  SEM_TRY(check_level(C, level));
  if (!w || (flags & ~SEM_GS_ADD_MASK) || (prec != SEM_FP64 && prec != SEM_FP32)) {
    set_detail("sem_level_gs: NULL vector, unknown flag or precision");
    return SEM_EINVAL;
  }
  return gs_apply(C->lev[level], prec, w, (flags & SEM_GS_ADD_MASK) != 0, (cudaStream_t)stream);
}

int sem_level_dinv(sem_ctx* h, int level, double h1, double h2, double* dinv, void* stream) {
  Ctx* C = ctx_of(h);
  SEM_TRY(check_level(C, level));
  if (!dinv) {
    set_detail("sem_level_dinv: NULL output");
    return SEM_EINVAL;
  }
  return level_dinv(*C, level, h1, h2, nullptr, dinv, nullptr, (cudaStream_t)stream);
}

int sem_prolong_add(sem_ctx* h, int level, int prec, const void* ec, void* xf, void* stream) {
  Ctx* C = ctx_of(h);
  SEM_TRY(check_level(C, level));
  if (level + 1 >= C->nlevels || !ec || !xf || (prec != SEM_FP64 && prec != SEM_FP32)) {
    set_detail("sem_prolong_add: no coarser level, NULL vector or bad precision");
    return SEM_EINVAL;
  }
  return interp_add(C->lev[level], C->lev[level + 1], prec, ec, xf, (cudaStream_t)stream);
}

int sem_restrict(sem_ctx* h, int level, int prec, const void* rf, void* rc, void* stream) {
  Ctx* C = ctx_of(h);
  SEM_TRY(check_level(C, level));
  if (level + 1 >= C->nlevels || !rf || !rc || (prec != SEM_FP64 && prec != SEM_FP32)) {
    set_detail("sem_restrict: no coarser level, NULL vector or bad precision");
    return SEM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  SEM_TRY(restrict_residual(C->lev[level], C->lev[level + 1], prec, rf, nullptr, rc, s));
  return gs_apply(C->lev[level + 1], prec, rc, true, s);
}

int sem_precond_setup(sem_ctx* h, double h1, double h2, int prec, void* stream) {
  Ctx* C = ctx_of(h);
  SEM_TRY(check_level(C, 0));
  SEM_TRY(check_prec(C, 0, prec));
  return precond_setup(*C, h1, h2, prec, (cudaStream_t)stream);
}

int sem_precond_setup_nodal(sem_ctx* h, const double* h1_L, double h2, int prec, void* stream) {
  Ctx* C = ctx_of(h);
  SEM_TRY(check_level(C, 0));
  SEM_TRY(check_prec(C, 0, prec));
  if (!h1_L) {
    set_detail("sem_precond_setup_nodal: NULL h1_L");
    return SEM_EINVAL;
  }
  return precond_setup(*C, 1.0, h2, prec, (cudaStream_t)stream, h1_L);
}

int sem_cheb_smooth(sem_ctx* h, int level, const void* b, void* x, int x_is_zero, void* stream) {
  Ctx* C = ctx_of(h);
  SEM_TRY(check_level(C, level));
  if (!C->pc_ready || level >= C->nlevels - 1 || !b || !x) {
    set_detail("sem_cheb_smooth: preconditioner not set up, coarsest level, or NULL vector");
    return SEM_EINVAL;
  }
  return cheb(*C, level, C->pc_prec, b, x, x_is_zero != 0, (cudaStream_t)stream);
}

int sem_asm_apply(sem_ctx* h, int level, int prec, const void* r, void* z, double h1, double h2, void* stream) {
  Ctx* C = ctx_of(h);
  SEM_TRY(check_level(C, level));
  if (!r || !z || r == z || (prec != SEM_FP64 && prec != SEM_FP32 && prec != SEM_BF16G)) {
    set_detail("sem_asm_apply: NULL or aliased vector, or precision other than SEM_FP64/SEM_FP32/SEM_BF16G");
    return SEM_EINVAL;
  }
  Level& L = C->lev[level];
  if (prec != SEM_FP64 && !L.G32 && !L.G16) {
    set_detail("sem_asm_apply: FP32 copies were not built");
    return SEM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  SEM_TRY(schwarz_build(*C, L, s));
  SEM_TRY(asm_sum(L, prec, r, nullptr, z, h1, h2, s));
  return asm_weight(L, prec, z, s);
}

int sem_advect(sem_ctx* h, int prec, const void* c, const void* u, void* w, int ncomp, int flags, void* stream) {
  Ctx* C = ctx_of(h);
  SEM_TRY(check_level(C, 0));
  if (!c || !u || !w || w == u || w == c || ncomp < 1 || (prec != SEM_FP64 && prec != SEM_FP32 && prec != SEM_FP64P) ||
      (flags & ~SEM_ADV_ASSEMBLE)) {
    set_detail("sem_advect: NULL or aliased vector, ncomp < 1, precision other than FP64/FP32/FP64P, or unknown flag");
    return SEM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  SEM_TRY(advect_build(*C, s));
  SEM_TRY(advect_apply(*C, prec, c, u, w, ncomp, s));
  if (flags & SEM_ADV_ASSEMBLE) {
    const Level& L = C->lev[0];
    const int vp = prec == SEM_FP32 ? SEM_FP32 : SEM_FP64;
    const size_t esz = vp == SEM_FP64 ? 8 : 4;
    for (int q = 0; q < ncomp; ++q)
      SEM_TRY(gs_apply(L, vp, static_cast<char*>(w) + (size_t)q * L.nL * esz, false, s));
  }
  return SEM_OK;
}

int sem_char_advance(sem_ctx* h, int prec, const void* c0, const void* c1, void* w, int ncomp, double t0, double t1,
                     int nsub, void* stream) {
  Ctx* C = ctx_of(h);
  SEM_TRY(check_level(C, 0));
  if (!c0 || !w || w == c0 || (c1 && w == c1) || ncomp < 1 || nsub < 1 || !(t1 != t0) ||
      (prec != SEM_FP64 && prec != SEM_FP32 && prec != SEM_FP64P)) {
    set_detail("sem_char_advance: NULL or aliased vector, ncomp or nsub < 1, t1 == t0, or precision other than FP64/FP32/FP64P");
    return SEM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  SEM_TRY(advect_build(*C, s));
  return char_advance(*C, prec, c0, c1, w, ncomp, t0, t1, nsub, s);
}

int sem_vcycle(sem_ctx* h, const double* r, double* z, void* stream) {
  Ctx* C = ctx_of(h);
  SEM_TRY(check_level(C, 0));
  if (!C->pc_ready || !r || !z) {
    set_detail("sem_vcycle: preconditioner not set up or NULL vector");
    return SEM_EINVAL;
  }
  return vcycle(*C, C->pc_prec, r, z, (cudaStream_t)stream);
}

int sem_get_lmax(const sem_ctx* h, double* lmax, int n) {
  const Ctx* C = reinterpret_cast<const Ctx*>(h);
  if (!C || !lmax || !C->pc_ready) {
    set_detail("sem_get_lmax: preconditioner not set up");
    return SEM_EINVAL;
  }
  for (int l = 0; l < n && l < C->nlevels; ++l) lmax[l] = C->lev[l].lmax;
  return SEM_OK;
}

int sem_rhs(sem_ctx* h, const double* f, double* b, void* stream) {
  Ctx* C = ctx_of(h);
  SEM_TRY(check_level(C, 0));
  if (!f || !b) {
    set_detail("sem_rhs: NULL vector");
    return SEM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  SEM_TRY(rhs_mass(C->lev[0], f, b, s));
  return gs_apply(C->lev[0], SEM_FP64, b, true, s);
}

int sem_mass_local(sem_ctx* h, const double* f, double* out, void* stream) {
  Ctx* C = ctx_of(h);
  SEM_TRY(check_level(C, 0));
  if (!f || !out) {
    set_detail("sem_mass_local: NULL vector");
    return SEM_EINVAL;
  }
  return rhs_mass(C->lev[0], f, out, (cudaStream_t)stream);
}

int sem_dot(sem_ctx* h, const double* a, const double* b, double* out, void* stream) {
  Ctx* C = ctx_of(h);
  SEM_TRY(check_level(C, 0));
  if (!a || !b || !out) {
    set_detail("sem_dot: NULL argument");
    return SEM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  double* d = C->scal + 2 * S_NSLOTS;
  SEM_TRY(dot_owner(*C, C->lev[0], SEM_FP64, a, b, d, s));
  SEM_CUDA_TRY(cudaMemcpyAsync(out, d, 8, cudaMemcpyDeviceToHost, s));
  SEM_CUDA_TRY(cudaStreamSynchronize(s));
  return SEM_OK;
}

int sem_grad_h1(sem_ctx* h, const double* u, const double* lam, double* g, int flags, void* stream) {
  Ctx* C = ctx_of(h);
  SEM_TRY(check_level(C, 0));
  if (!u || !lam || !g || u == g || lam == g || (flags & ~SEM_GRAD_SUM)) {
    set_detail("sem_grad_h1: NULL or aliased vector or unknown flag");
    return SEM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  SEM_TRY(grad_h1_apply(C->lev[0], u, lam, g, s));
  if (flags & SEM_GRAD_SUM) SEM_TRY(gs_apply(C->lev[0], SEM_FP64, g, false, s));
  return SEM_OK;
}

}  // extern "C"

namespace {

// The body of sem_solve and sem_solve_proj. With a projection space P the
// right-hand side b is first projected (xbar, r0 = b - A xbar), the Krylov solve
// finds dx from r0 with x0 = 0 and stops at ||r|| <= tol ||b||, and afterwards
// u = xbar + dx and the space takes the new direction.
int solve_impl(Ctx* C, Proj* P, const double* f, const sem_coef* c, double tol, int maxit, int precond, int prec,
               int rhs_flags, double* u, sem_info* info, cudaStream_t s) {
  SEM_TRY(check_level(C, 0));
  C->graph_steps = 0;
  if (!f || !c || !u || f == u || !(tol >= 0.0) || maxit < 0 ||
      (precond != SEM_PC_JACOBI && precond != SEM_PC_PMG) ||
      (rhs_flags & ~(SEM_RHS_ASSEMBLED | SEM_X0_GIVEN | SEM_OUTER_PAIRS)) ||
      (P && (rhs_flags & SEM_X0_GIVEN))) {
    set_detail("sem_solve: bad argument (a projected solve takes no initial guess)");
    return SEM_EINVAL;
  }
  if (precond == SEM_PC_PMG) SEM_TRY(check_prec(C, 0, prec));
  if (precond == SEM_PC_PMG && c->h1_L && C->opts.smoother != SEM_SMOOTH_JACOBI) {
    set_detail("sem_solve: p-multigrid with a nodal h1 needs the Chebyshev-Jacobi smoother");
    return SEM_EINVAL;
  }
  const bool pairs = (rhs_flags & SEM_OUTER_PAIRS) != 0;
  if (pairs && !C->lev[0].G2) {
    set_detail("sem_solve: SEM_OUTER_PAIRS needs the pair factors (SEM_BUILD_PAIRS)");
    return SEM_EINVAL;
  }
  // outer operator R QQ^T A_L p (FP64 or FP32-pair element kernel)
  auto outer_ax = [&](const double* in, double* out, const double* skip, cudaStream_t st) -> int {
    if (pairs) SEM_TRY(ax_pairs_apply(C->lev[0], in, out, c->h1, c->h2, c->h1_L, st));
    else SEM_TRY(ax_apply(C->lev[0], SEM_FP64, in, out, c->h1, c->h2, c->h1_L, st, skip));
    return gs_apply_skip(C->lev[0], SEM_FP64, out, true, skip, st);
  };
  Level& L = C->lev[0];
  const int64_t n = L.nL;
  double* sc = C->scal;   // outer slot set
  double* b = C->t;
  if (rhs_flags & SEM_RHS_ASSEMBLED) {
    // replicated assembled values: average the copies (QQ^T W f) and mask
    SEM_TRY(mul_counting_weight(L, SEM_FP64, f, b, s));
  } else {
    // b = R QQ^T B_L f
    SEM_TRY(rhs_mass(L, f, b, s));
  }
  SEM_TRY(gs_apply(L, SEM_FP64, b, true, s));
  // projection onto earlier solutions: b <- r0 = b - A xbar (in place), reference norm (b, b)
  const double* bbref = nullptr;
  double* xbar = nullptr;
  if (P) {
    proj_bind_coef(*P, c, pairs);
    SEM_TRY(proj_state(*P, nullptr, nullptr, &xbar, &bbref, nullptr, s));
    SEM_TRY(proj_project(*P, b, xbar, b, s));
  }
  const bool x0 = (rhs_flags & SEM_X0_GIVEN) != 0;
  double* w = C->w;
  if (x0) SEM_TRY(outer_ax(u, w, nullptr, s));
  SEM_CUDA_TRY(cudaMemsetAsync(C->scal + 1 * S_NSLOTS + S_TOTAL, 0, sizeof(double), s));
  int iters = 0;
  double rr = 0, bb = 0;
  int rc = SEM_OK;
  if (precond == SEM_PC_JACOBI) {
    double* dinv = C->z;
    SEM_TRY(level_dinv(*C, 0, c->h1, c->h2, c->h1_L, dinv, nullptr, s));
    SEM_TRY(pcg_begin_tol(*C, L, SEM_FP64, b, x0 ? w : nullptr, u, C->r, dinv, C->p, sc, tol, s, bbref));
    const int batch = 8;
    int launched = 0;
    while (true) {
      SEM_TRY(read_scalars(*C, 0, s));
      const double* hs = C->h_scal;
      bb = hs[S_BB];
      rr = hs[S_RR];
      iters = (int)hs[S_ITER];
      if (hs[S_BREAK] != 0.0) {
        rc = SEM_EBREAKDOWN;
        break;
      }
      if (hs[S_DONE] != 0.0) break;
      if (launched >= maxit) {
        rc = SEM_ENOTCONV;
        break;
      }
      const int nb = std::min(batch, maxit - launched);
      for (int q = 0; q < nb; ++q) {
        SEM_TRY(outer_ax(C->p, w, sc + S_DONE, s));
        SEM_TRY(kr_alpha(*C, L, SEM_FP64, C->p, w, sc, s));
        SEM_TRY(kr_update_jacobi(*C, L, SEM_FP64, u, C->p, C->r, w, dinv, sc, s));
        SEM_TRY(kr_direction_jacobi(L, SEM_FP64, C->p, C->r, dinv, sc, s));
      }
      launched += nb;
    }
  } else {
    // the preconditioner is kept while the coefficients are the same (a nodal h1: the same
    // pointer; values changed behind it give a stale but still valid preconditioner)
    const bool same = C->pc_ready && C->pc_h2 == c->h2 && C->pc_prec == prec &&
                      (c->h1_L ? (C->pc_nodal && C->pc_h1L == c->h1_L) : (!C->pc_nodal && C->pc_h1 == c->h1));
    if (!same) SEM_TRY(precond_setup(*C, c->h1, c->h2, prec, s, c->h1_L));
    SEM_TRY(pcg_begin_tol(*C, L, SEM_FP64, b, x0 ? w : nullptr, u, C->r, nullptr, nullptr, sc, tol, s, bbref));
    SEM_CUDA_TRY(cudaMemsetAsync(C->p, 0, n * 8, s));
    SEM_TRY(read_scalars(*C, 0, s));
    bb = C->h_scal[S_BB];
    rr = C->h_scal[S_RR];
    if (C->h_scal[S_DONE] == 0.0) {
      // the V-cycle reads r from the finest level's b and leaves z in its x, both
      // in the V-cycle's type: the update kernel writes b, beta and the direction read x
      const VecSet v0 = vecs(C->lev[0], prec);
      const int vp = prec == SEM_FP64 ? SEM_FP64 : SEM_FP32;
      SEM_TRY(vec_copy_convert(C->r, SEM_FP64, v0.b, vp, n, s));
      SEM_TRY(vcycle_level(*C, 0, prec, s));
      SEM_TRY(kr_beta_flex(*C, L, v0.x, vp, C->r, nullptr, sc, s));
      SEM_TRY(kr_direction(L, C->p, v0.x, vp, sc, s));
      for (int k = 0; k < maxit; ++k) {
        SEM_TRY(outer_ax(C->p, w, nullptr, s));
        SEM_TRY(kr_alpha(*C, L, SEM_FP64, C->p, w, sc, s));
        SEM_TRY(kr_update_flex(*C, L, u, C->p, C->r, w, v0.b, vp, sc, s));
        SEM_TRY(read_scalars(*C, 0, s));
        const double* hs = C->h_scal;
        rr = hs[S_RR];
        iters = (int)hs[S_ITER];
        if (hs[S_BREAK] != 0.0) {
          rc = SEM_EBREAKDOWN;
          break;
        }
        if (hs[S_DONE] != 0.0) break;
        SEM_TRY(precond_step(*C, prec, v0.x, vp, w, sc, s));
      }
      if (rc == SEM_OK && C->h_scal[S_DONE] == 0.0) rc = SEM_ENOTCONV;
    }
  }
  double relres0 = -1.0;
  int pcount = 0;
  if (P) {
    // u holds dx: store it as the new direction (on restart the whole x is stored instead), then u = xbar + dx
    int count = 0, maxv = 0;
    SEM_TRY(proj_state(*P, &count, &maxv, nullptr, nullptr, nullptr, s));
    if (rc == SEM_OK || rc == SEM_ENOTCONV) {
      if (count < maxv) {
        SEM_TRY(proj_update(*P, c, pairs, nullptr, u, nullptr, s));
        SEM_TRY(proj_add_xbar(*P, u, s));
      } else {
        SEM_TRY(proj_add_xbar(*P, u, s));
        SEM_TRY(proj_update(*P, c, pairs, u, u, nullptr, s));
      }
    } else {
      SEM_TRY(proj_add_xbar(*P, u, s));
    }
    double h[2] = {0, 0};
    SEM_TRY(proj_state(*P, &pcount, nullptr, nullptr, nullptr, h, s));
    relres0 = h[0] > 0 ? std::sqrt(h[1] / h[0]) : 0.0;
  }
  if (info) {
    double ct = 0;
    SEM_CUDA_TRY(cudaMemcpyAsync(&ct, C->scal + 1 * S_NSLOTS + S_TOTAL, 8, cudaMemcpyDeviceToHost, s));
    SEM_CUDA_TRY(cudaStreamSynchronize(s));
    info->iters = iters;
    info->bnorm = std::sqrt(bb);
    info->relres = bb > 0 ? std::sqrt(rr / bb) : 0.0;
    info->coarse_iters = (int)ct;
    info->nlevels = C->nlevels;
    for (int l = 0; l < SEM_MAX_LEVELS; ++l) info->lmax[l] = (l < C->nlevels) ? C->lev[l].lmax : 0.0;
    info->relres0 = relres0;
    info->proj_count = pcount;
    info->graph_steps = C->graph_steps;
  }
  if (rc == SEM_ENOTCONV) set_detail("no convergence in %d iterations (relres %.3e)", maxit, bb > 0 ? std::sqrt(rr / bb) : 0.0);
  if (rc == SEM_EBREAKDOWN) set_detail("Krylov breakdown after %d iterations", iters);
  return rc;
}

}  // namespace

extern "C" {

int sem_solve(sem_ctx* h, const double* f, const sem_coef* c, double tol, int maxit, int precond, int prec,
              int rhs_flags, double* u, sem_info* info, void* stream) {
  return solve_impl(ctx_of(h), nullptr, f, c, tol, maxit, precond, prec, rhs_flags, u, info, (cudaStream_t)stream);
}

int sem_solve_proj(sem_ctx* h, sem_proj* pj, const double* f, const sem_coef* c, double tol, int maxit,
                   int precond, int prec, int rhs_flags, double* u, sem_info* info, void* stream) {
  Proj* P = reinterpret_cast<Proj*>(pj);
  if (!P || !proj_belongs(*P, ctx_of(h))) {
    set_detail("sem_solve_proj: NULL projection space or a space created for another context");
    return SEM_EINVAL;
  }
  return solve_impl(ctx_of(h), P, f, c, tol, maxit, precond, prec, rhs_flags, u, info, (cudaStream_t)stream);
}

}  // extern "C"
