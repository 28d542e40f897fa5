// sem_setup / sem_free and the setup products: GLL rule and D_hat per order
// (Section 2.3, eq. dh), device geometry (eq. grad, eq. gij, eq. vBu), the
// canonical gather-scatter maps (gs_setup, Section 3.2) and the p-multigrid
// levels (Section 3.4, "Poisson Solve Preconditioning": orders N, N/2, ..., 1).
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <vector>

#include "sem_internal.cuh"

namespace sem {

namespace {
thread_local char g_detail[512] = "";
}

void set_detail(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_detail, sizeof(g_detail), fmt, ap);
  va_end(ap);
}

// ---------------------------------------------------------------------------
// 1-D rules on the host
// ---------------------------------------------------------------------------
static void legendre(int N, double x, double* pn, double* pnm1) {
  double p0 = 1.0, p1 = x;
  if (N == 0) {
    *pn = 1.0;
    *pnm1 = 0.0;
    return;
  }
  for (int k = 1; k < N; ++k) {
    const double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
    p0 = p1;
    p1 = p2;
  }
  *pn = p1;
  *pnm1 = p0;
}

// GLL nodes: +-1 and the roots of P_N', by Newton's method on P_N' with
// P_N' = N (x P_N - P_{N-1}) / (x^2 - 1) and P_N'' from Legendre's equation,
// started at the Chebyshev-Gauss-Lobatto points. Weights 2 / (N(N+1) P_N^2).
void host_gll(int N, double* xi, double* rho) {
  xi[0] = -1.0;
  xi[N] = 1.0;
  for (int j = 1; j < N; ++j) {
    double x = -std::cos(M_PI * j / N);
    for (int it = 0; it < 100; ++it) {
      double P, Pm1;
      legendre(N, x, &P, &Pm1);
      const double dP = N * (x * P - Pm1) / (x * x - 1.0);
      const double d2P = (2.0 * x * dP - N * (N + 1) * P) / (1.0 - x * x);
      const double step = dP / d2P;
      x -= step;
      if (std::fabs(step) < 1e-16) break;
    }
    xi[j] = x;
  }
  for (int j = 0; j <= N / 2; ++j) {  // exact antisymmetry
    const double a = 0.5 * (xi[N - j] - xi[j]);
    xi[N - j] = a;
    xi[j] = -a;
  }
  if (N % 2 == 0) xi[N / 2] = 0.0;
  for (int j = 0; j <= N; ++j) {
    double P, Pm1;
    legendre(N, xi[j], &P, &Pm1);
    rho[j] = 2.0 / (N * (N + 1) * P * P);
  }
}

// D[a][b] = h_b'(xi_a): P_N(xi_a) / (P_N(xi_b)(xi_a - xi_b)) off the diagonal,
// -N(N+1)/4 and +N(N+1)/4 at the two corners, 0 elsewhere on the diagonal.
void host_dhat(int N, const double* xi, double* D) {
  const int NP = N + 1;
  double P[16];
  for (int a = 0; a < NP; ++a) {
    double pm1;
    legendre(N, xi[a], &P[a], &pm1);
  }
  for (int a = 0; a < NP; ++a)
    for (int b = 0; b < NP; ++b) D[a * NP + b] = (a == b) ? 0.0 : P[a] / (P[b] * (xi[a] - xi[b]));
  D[0] = -N * (N + 1) / 4.0;
  D[N * NP + N] = N * (N + 1) / 4.0;
}

void host_interp(int nc, const double* xi_from, int nt, const double* x_to, double* J) {
  for (int a = 0; a < nt; ++a)
    for (int b = 0; b < nc; ++b) {
      double v = 1.0;
      for (int c = 0; c < nc; ++c)
        if (c != b) v *= (x_to[a] - xi_from[c]) / (xi_from[b] - xi_from[c]);
      J[a * nc + b] = v;
    }
}

namespace {

// Coarse-level coordinates: the fine isoparametric map (eq. xijk) evaluated at
// the coarse GLL points, x_c = (J x J x J) x_f with J[a][b] = h^f_b(xi^c_a).
__global__ void k_interp_coords(int E, int NPf, int NPc, const double* __restrict__ xf, double* __restrict__ xc,
                                Mat64 J) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t C3 = (int64_t)NPc * NPc * NPc, F3 = (int64_t)NPf * NPf * NPf;
  if (p >= (int64_t)E * C3) return;
  const int64_t e = p / C3;
  const int loc = (int)(p - e * C3);
  const int k = loc / (NPc * NPc), j = (loc / NPc) % NPc, i = loc % NPc;
  const double* X = xf + e * F3;
  double acc = 0;
  for (int c = 0; c < NPf; ++c) {
    double t2 = 0;
    for (int b = 0; b < NPf; ++b) {
      double t1 = 0;
      for (int a = 0; a < NPf; ++a) t1 += J.a[i * NPf + a] * X[(c * NPf + b) * NPf + a];
      t2 += J.a[j * NPf + b] * t1;
    }
    acc += J.a[k * NPf + c] * t2;
  }
  xc[p] = acc;
}

// Global ids and Dirichlet flags at the order-Nc points from the order-Nf ones.
// Vertex: the fine vertex id. Edge: named by the smallest nonzero fine id on
// its interior; position counted from the endpoint with the smaller fine id.
// Face: named by the smallest nonzero fine id on its interior; position in the
// frame whose origin is the corner with the smallest fine id and whose first
// axis points to the origin's neighbour corner with the smaller fine id.
// key = (entity * 3 + type) * 256 + position; 0 (singleton) for interiors and
// unshared entities.
__global__ void k_coarse_ids(int E, int Nf, int Nc, const int64_t* __restrict__ gf, const uint8_t* __restrict__ df,
                             int64_t* __restrict__ gc, uint8_t* __restrict__ dc) {
  const int NPf = Nf + 1, NPc = Nc + 1;
  const int64_t C3 = (int64_t)NPc * NPc * NPc, F3 = (int64_t)NPf * NPf * NPf;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= (int64_t)E * C3) return;
  const int64_t e = p / C3;
  const int loc = (int)(p - e * C3);
  const int c[3] = {loc % NPc, (loc / NPc) % NPc, loc / (NPc * NPc)};
  const int64_t* G = gf + e * F3;
  const uint8_t* Df = df ? df + e * F3 : nullptr;
  auto at = [&](const int f[3]) { return (f[2] * NPf + f[1]) * NPf + f[0]; };
  int mids[3], nm = 0;
  for (int d = 0; d < 3; ++d)
    if (c[d] > 0 && c[d] < Nc) mids[nm++] = d;
  int base[3];
  for (int d = 0; d < 3; ++d) base[d] = (c[d] == 0) ? 0 : Nf;
  int64_t key = 0;
  uint8_t dir = 0;
  if (nm == 0) {
    const int64_t g = G[at(base)];
    key = g > 0 ? g * 3 * 256 : 0;
    dir = Df ? Df[at(base)] : 0;
  } else if (nm == 1) {
    const int d = mids[0];
    int fa[3] = {base[0], base[1], base[2]}, fb[3] = {base[0], base[1], base[2]};
    fa[d] = 0;
    fb[d] = Nf;
    const int64_t gA = G[at(fa)], gB = G[at(fb)];
    int64_t ent = 0;
    int f[3] = {base[0], base[1], base[2]};
    for (int t = 1; t < Nf; ++t) {
      f[d] = t;
      const int64_t g = G[at(f)];
      if (g > 0 && (ent == 0 || g < ent)) ent = g;
      if (Df && Df[at(f)]) dir = 1;
    }
    const int pos = (gA < gB) ? c[d] : Nc - c[d];
    key = ent > 0 ? (ent * 3 + 1) * 256 + pos : 0;
  } else if (nm == 2) {
    const int d1 = mids[0], d2 = mids[1];
    int64_t cg[4];
    for (int s2 = 0; s2 < 2; ++s2)
      for (int s1 = 0; s1 < 2; ++s1) {
        int f[3] = {base[0], base[1], base[2]};
        f[d1] = s1 * Nf;
        f[d2] = s2 * Nf;
        cg[s1 + 2 * s2] = G[at(f)];
      }
    int o = 0;
    for (int q = 1; q < 4; ++q)
      if (cg[q] < cg[o]) o = q;
    const int o1 = o % 2, o2 = o / 2;
    const int64_t n1 = cg[(1 - o1) + 2 * o2], n2 = cg[o1 + 2 * (1 - o2)];
    const int a_o = (o1 == 0) ? c[d1] : Nc - c[d1];
    const int b_o = (o2 == 0) ? c[d2] : Nc - c[d2];
    const int ap = (n1 < n2) ? a_o : b_o;
    const int bp = (n1 < n2) ? b_o : a_o;
    int64_t ent = 0;
    int f[3] = {base[0], base[1], base[2]};
    for (int t2 = 1; t2 < Nf; ++t2)
      for (int t1 = 1; t1 < Nf; ++t1) {
        f[d1] = t1;
        f[d2] = t2;
        const int64_t g = G[at(f)];
        if (g > 0 && (ent == 0 || g < ent)) ent = g;
        if (Df && Df[at(f)]) dir = 1;
      }
    key = ent > 0 ? (ent * 3 + 2) * 256 + ap * 16 + bp : 0;
  }
  gc[p] = key;
  dc[p] = dir;
}

template <typename T>
int dmalloc(T** p, size_t count) {
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T) + 16);
  if (e != cudaSuccess) {
    *p = nullptr;
    set_detail("cudaMalloc of %zu bytes: %s", count * sizeof(T), cudaGetErrorString(e));
    cudaGetLastError();
    return SEM_ENOMEM;
  }
  return SEM_OK;
}

void free_level(Level& L) {
  void* ptrs[] = {L.G, L.G32, L.G16, L.G2, L.x, L.y, L.z, L.gid, L.dflag, L.ids, L.off, L.idx, L.mult, L.node,
                  L.label, L.dmask, L.owner, L.cwt, L.cwt32, L.seg_off, L.seg_idx, L.seg_dir, L.dinv, L.dinv32,
                  L.vb, L.vx, L.vr, L.vd, L.vw, L.fb, L.fx, L.fr, L.fd, L.fw, L.cp, L.cpf,
                  L.sch_layer, L.sch_bt, L.sch_len, L.sch_len32, L.sch_ref, L.sch_ref32, L.sch_w, L.sch_w32,
                  L.sch_zf, L.sch_zf32, L.sch_woff, L.sch_witem, L.sch_wdir, L.sch_wpair, L.pp_el_off, L.pp_el,
                  L.pp_p2n, L.pp_nd_off, L.pp_nd_src, L.pp_nd_fl, L.pp_cp_off, L.pp_cp, L.pp_xbuf, L.pp_part,
                  L.h1n, L.pcG, L.pcG32, L.pcG16};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  L = Level();
}

int set_order(Level& L, int N, int E) {
  L.N = N;
  L.NP = N + 1;
  L.E = E;
  L.nL = (int64_t)E * np3(N);
  host_gll(N, L.xi, L.rho);
  double D[144];
  host_dhat(N, L.xi, D);
  for (int t = 0; t < L.NP * L.NP; ++t) {
    L.D.a[t] = D[t];
    L.Df.a[t] = (float)D[t];
  }
  return SEM_OK;
}

int build_level_products(Ctx& C, Level& L, cudaStream_t s) {
  const int64_t n = L.nL;
  SEM_TRY(dmalloc(&L.G, 7 * n));
  if (C.opts.prec_copies & SEM_BUILD_FP32) SEM_TRY(dmalloc(&L.G32, 7 * n));
  if (C.opts.prec_copies & SEM_BUILD_BF16G) SEM_TRY(dmalloc(&L.G16, 7 * n));
  int* d_bad = nullptr;
  SEM_TRY(dmalloc(&d_bad, 1));
  SEM_CUDA_TRY(cudaMemsetAsync(d_bad, 0, sizeof(int), s));
  int rc = geom_compute(L, d_bad, s);
  int bad = 0;
  if (rc == SEM_OK) {
    SEM_CUDA_TRY(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    SEM_CUDA_TRY(cudaStreamSynchronize(s));
  }
  cudaFree(d_bad);
  SEM_TRY(rc);
  if (bad) {
    set_detail("non-positive Jacobian at order %d", L.N);
    return SEM_EMESH;
  }
  if (C.opts.prec_copies & SEM_BUILD_PAIRS) SEM_TRY(pairs_build(L, s));
  SEM_TRY(build_maps(L, s));
  // preconditioner and V-cycle vectors
  SEM_TRY(dmalloc(&L.dinv, n));
  SEM_TRY(dmalloc(&L.vb, n));
  SEM_TRY(dmalloc(&L.vx, n));
  SEM_TRY(dmalloc(&L.vr, n));
  SEM_TRY(dmalloc(&L.vd, n));
  SEM_TRY(dmalloc(&L.vw, n));
  SEM_TRY(dmalloc(&L.cp, n));
  if (C.opts.prec_copies & (SEM_BUILD_FP32 | SEM_BUILD_BF16G)) {
    SEM_TRY(dmalloc(&L.dinv32, n));
    SEM_TRY(dmalloc(&L.fb, n));
    SEM_TRY(dmalloc(&L.fx, n));
    SEM_TRY(dmalloc(&L.fr, n));
    SEM_TRY(dmalloc(&L.fd, n));
    SEM_TRY(dmalloc(&L.fw, n));
    SEM_TRY(dmalloc(&L.cpf, n));
  }
  return SEM_OK;
}

int coarsen(Ctx& C, const Level& F, Level& L, int Nc, cudaStream_t s) {
  SEM_TRY(set_order(L, Nc, F.E));
  const int64_t n = L.nL;
  SEM_TRY(dmalloc(&L.x, n));
  SEM_TRY(dmalloc(&L.y, n));
  SEM_TRY(dmalloc(&L.z, n));
  SEM_TRY(dmalloc(&L.gid, n));
  SEM_TRY(dmalloc(&L.dflag, n));
  Mat64 J{};
  host_interp(F.NP, F.xi, L.NP, L.xi, J.a);
  const unsigned nb = (unsigned)((n + 255) / 256);
  k_interp_coords<<<nb, 256, 0, s>>>(L.E, F.NP, L.NP, F.x, L.x, J);
  k_interp_coords<<<nb, 256, 0, s>>>(L.E, F.NP, L.NP, F.y, L.y, J);
  k_interp_coords<<<nb, 256, 0, s>>>(L.E, F.NP, L.NP, F.z, L.z, J);
  SEM_LAUNCH_CHECK();
  k_coarse_ids<<<nb, 256, 0, s>>>(L.E, F.N, Nc, F.gid, F.dflag, L.gid, L.dflag);
  SEM_LAUNCH_CHECK();
  return build_level_products(C, L, s);
}

int validate_orders(const sem_mesh* m, const sem_opts& o, std::vector<int>& orders) {
  orders.clear();
  if (o.mg_nlevels == 0) {
    orders.push_back(m->N);
    while (orders.back() > 1 && (int)orders.size() < SEM_MAX_LEVELS) orders.push_back(std::max(1, orders.back() / 2));
    return SEM_OK;
  }
  if (o.mg_nlevels < 1 || o.mg_nlevels > SEM_MAX_LEVELS) {
    set_detail("mg_nlevels must be in 1..%d", SEM_MAX_LEVELS);
    return SEM_EINVAL;
  }
  for (int l = 0; l < o.mg_nlevels; ++l) {
    const int N = o.mg_orders[l];
    if (N < 1 || N > SEM_MAX_N || (l == 0 && N != m->N) || (l > 0 && N >= orders.back())) {
      set_detail("mg_orders must start at N and decrease strictly to >= 1");
      return SEM_EINVAL;
    }
    orders.push_back(N);
  }
  return SEM_OK;
}

}  // namespace

// a nodal field of level F at the GLL points of the next coarser level C
int interp_nodal(const Level& F, const Level& C, const double* f, double* c, cudaStream_t s) {
  Mat64 J{};
  host_interp(F.NP, F.xi, C.NP, C.xi, J.a);
  const int64_t n = C.nL;
  k_interp_coords<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(C.E, F.NP, C.NP, f, c, J);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}

}  // namespace sem

using namespace sem;

extern "C" {

void sem_default_opts(sem_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->mg_nlevels = 0;
  o->cheb_degree = 2;
  o->cheb_lmin_factor = 0.1;
  o->cheb_lmax_factor = 1.1;
  o->lanczos_steps = 10;
  o->lanczos_seed = 1;
  o->coarse_tol = 1e-1;
  o->coarse_maxit = 100;
  o->prec_copies = SEM_BUILD_FP32 | SEM_BUILD_BF16G | SEM_BUILD_PAIRS;
  o->smoother = SEM_SMOOTH_JACOBI;
  o->coarse_mode = SEM_COARSE_AUTO;
  o->spin_limit = 1ll << 31;
}

const char* sem_strerror(int code) {
  switch (code) {
    case SEM_OK: return "success";
    case SEM_EINVAL: return "invalid argument";
    case SEM_ENOMEM: return "device allocation failed";
    case SEM_ECUDA: return "CUDA error";
    case SEM_ENOTCONV: return "iteration limit reached before the tolerance";
    case SEM_EBREAKDOWN: return "Krylov breakdown (p^T A p <= 0 or non-finite scalar)";
    case SEM_EMESH: return "mesh rejected (non-positive Jacobian)";
  }
  return "unknown error";
}

const char* sem_last_error_detail(void) { return g_detail; }

void sem_free(sem_ctx* h) {
  Ctx* C = reinterpret_cast<Ctx*>(h);
  if (!C) return;
  for (int l = 0; l < SEM_MAX_LEVELS; ++l) free_level(C->lev[l]);
  advect_free(C->adv);
  void* ptrs[] = {C->red_part, C->red_ticket, C->scal, C->r, C->z, C->p, C->w, C->t,
                  C->cg_err};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (C->h_scal) cudaFreeHost(C->h_scal);
  if (C->ev) cudaEventDestroy(C->ev);
  for (auto& e : C->cev)
    if (e) cudaEventDestroy(e);
  if (C->h_done) cudaFreeHost(C->h_done);
  if (C->pc_graph) cudaGraphExecDestroy(C->pc_graph);
  if (C->cap_stream) cudaStreamDestroy(C->cap_stream);
  delete C;
}

int sem_setup(const sem_mesh* m, const sem_opts* opts_in, sem_ctx** out) {
  if (!out) {
    set_detail("out is NULL");
    return SEM_EINVAL;
  }
  *out = nullptr;
  if (!m || !m->x || !m->y || !m->z || !m->gid) {
    set_detail("mesh or one of its coordinate/id arrays is NULL");
    return SEM_EINVAL;
  }
  if (m->N < 1 || m->N > SEM_MAX_N) {
    set_detail("N = %d outside 1..%d", m->N, SEM_MAX_N);
    return SEM_EINVAL;
  }
  if (m->E < 1) {
    set_detail("E = %d must be >= 1", m->E);
    return SEM_EINVAL;
  }
  const int64_t nL = (int64_t)m->E * np3(m->N);
  if (nL >= ((int64_t)1 << 31) - 16) {
    set_detail("E*(N+1)^3 = %lld exceeds the 32-bit local index range", (long long)nL);
    return SEM_EINVAL;
  }
  sem_opts o;
  if (opts_in) o = *opts_in;
  else sem_default_opts(&o);
  if (o.cheb_degree < 1 || o.lanczos_steps < 1 || o.coarse_maxit < 0 || o.spin_limit < 0 ||
      !(o.cheb_lmax_factor > o.cheb_lmin_factor) ||
      (o.smoother != SEM_SMOOTH_JACOBI && o.smoother != SEM_SMOOTH_ASM) ||
      (o.coarse_mode != SEM_COARSE_AUTO && o.coarse_mode != SEM_COARSE_KERNELS && o.coarse_mode != SEM_COARSE_PIPE)) {
    set_detail("invalid smoother / Lanczos / coarse-solve options");
    return SEM_EINVAL;
  }
  std::vector<int> orders;
  SEM_TRY(validate_orders(m, o, orders));
  for (int64_t l = 0; l < nL; ++l)
    if (m->gid[l] < 0) {
      set_detail("negative global id at local point %lld", (long long)l);
      return SEM_EINVAL;
    }
  Ctx* C = new Ctx();
  C->opts = o;
  cudaGetDevice(&C->device);
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    delete C;
    set_detail("cudaStreamCreate failed");
    return SEM_ECUDA;
  }
  auto fail = [&](int rc) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    sem_free(reinterpret_cast<sem_ctx*>(C));
    return rc;
  };
#define STEP(expr)                   \
  do {                               \
    int rc_ = (expr);                \
    if (rc_ != SEM_OK) return fail(rc_); \
  } while (0)
#define CUSTEP(call)                                                              \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      set_detail("%s: %s", #call, cudaGetErrorString(e_));                        \
      return fail(SEM_ECUDA);                                                     \
    }                                                                             \
  } while (0)
  Level& F = C->lev[0];
  STEP(set_order(F, m->N, m->E));
  STEP(dmalloc(&F.x, nL));
  STEP(dmalloc(&F.y, nL));
  STEP(dmalloc(&F.z, nL));
  STEP(dmalloc(&F.gid, nL));
  STEP(dmalloc(&F.dflag, nL));
  CUSTEP(cudaMemcpyAsync(F.x, m->x, nL * 8, cudaMemcpyHostToDevice, s));
  CUSTEP(cudaMemcpyAsync(F.y, m->y, nL * 8, cudaMemcpyHostToDevice, s));
  CUSTEP(cudaMemcpyAsync(F.z, m->z, nL * 8, cudaMemcpyHostToDevice, s));
  CUSTEP(cudaMemcpyAsync(F.gid, m->gid, nL * 8, cudaMemcpyHostToDevice, s));
  if (m->dirichlet) {
    std::vector<uint8_t> d(m->dirichlet, m->dirichlet + nL);
    for (auto& v : d) v = v ? 1 : 0;
    CUSTEP(cudaMemcpyAsync(F.dflag, d.data(), nL, cudaMemcpyHostToDevice, s));
    CUSTEP(cudaStreamSynchronize(s));
  } else {
    CUSTEP(cudaMemsetAsync(F.dflag, 0, nL, s));
  }
  STEP(build_level_products(*C, F, s));
  C->nlevels = 1;
  for (size_t l = 1; l < orders.size(); ++l) {
    STEP(coarsen(*C, C->lev[l - 1], C->lev[l], orders[l], s));
    Level& Fi = C->lev[l - 1];
    Level& Co = C->lev[l];
    double J[144];
    host_interp(Co.NP, Co.xi, Fi.NP, Fi.xi, J);   // J[a*NPc + b] = h^c_b(xi^f_a)
    for (int t = 0; t < Fi.NP * Co.NP; ++t) {
      Fi.Jc.a[t] = J[t];
      Fi.Jcf.a[t] = (float)J[t];
    }
    C->nlevels = (int)l + 1;
  }
  for (int l = 0; l < C->nlevels; ++l) C->lev[l].spin_limit = o.spin_limit;
  // reduction scratch and fine-level solver workspace
  STEP(dmalloc(&C->red_part, RED_BLOCKS * 4));
  STEP(dmalloc(&C->red_ticket, 1));
  STEP(dmalloc(&C->cg_err, 1));
  CUSTEP(cudaMemsetAsync(C->red_ticket, 0, sizeof(unsigned), s));
  STEP(dmalloc(&C->scal, 4 * S_NSLOTS));
  CUSTEP(cudaMemsetAsync(C->scal, 0, 4 * S_NSLOTS * sizeof(double), s));
  CUSTEP(cudaMallocHost((void**)&C->h_scal, 4 * S_NSLOTS * sizeof(double)));
  STEP(dmalloc(&C->r, nL));
  STEP(dmalloc(&C->z, nL));
  STEP(dmalloc(&C->p, nL));
  STEP(dmalloc(&C->w, nL));
  STEP(dmalloc(&C->t, nL));
  CUSTEP(cudaEventCreateWithFlags(&C->ev, cudaEventDisableTiming));
  CUSTEP(cudaEventCreateWithFlags(&C->cev[0], cudaEventDisableTiming));
  CUSTEP(cudaEventCreateWithFlags(&C->cev[1], cudaEventDisableTiming));
  CUSTEP(cudaMallocHost((void**)&C->h_done, 2 * sizeof(double)));
  CUSTEP(cudaStreamCreateWithFlags(&C->cap_stream, cudaStreamNonBlocking));
  CUSTEP(cudaStreamSynchronize(s));
  cudaStreamDestroy(s);
#undef STEP
#undef CUSTEP
  *out = reinterpret_cast<sem_ctx*>(C);
  return SEM_OK;
}

int sem_num_levels(const sem_ctx* h) {
  const Ctx* C = reinterpret_cast<const Ctx*>(h);
  return C ? C->nlevels : 0;
}

int sem_level_info(const sem_ctx* h, int level, sem_level_desc* d) {
  const Ctx* C = reinterpret_cast<const Ctx*>(h);
  if (!C || !d || level < 0 || level >= C->nlevels) {
    set_detail("bad context, output or level");
    return SEM_EINVAL;
  }
  const Level& L = C->lev[level];
  d->N = L.N;
  d->E = L.E;
  d->nL = L.nL;
  d->nG = L.nG;
  d->n_ids = L.n_ids;
  d->n_idx = L.n_idx;
  d->n_seg = L.n_seg;
  d->n_seg_idx = L.n_seg_idx;
  return SEM_OK;
}

int sem_get_maps(const sem_ctx* h, int level, int64_t* ids, int64_t* off, int32_t* idx, int32_t* mult,
                 int64_t* node, int64_t* label, uint8_t* dmask) {
  const Ctx* C = reinterpret_cast<const Ctx*>(h);
  if (!C || level < 0 || level >= C->nlevels) {
    set_detail("bad context or level");
    return SEM_EINVAL;
  }
  const Level& L = C->lev[level];
  if (ids) SEM_CUDA_TRY(cudaMemcpy(ids, L.ids, L.n_ids * 8, cudaMemcpyDeviceToHost));
  if (off) SEM_CUDA_TRY(cudaMemcpy(off, L.off, (L.n_ids + 1) * 8, cudaMemcpyDeviceToHost));
  if (idx) SEM_CUDA_TRY(cudaMemcpy(idx, L.idx, L.n_idx * 4, cudaMemcpyDeviceToHost));
  if (mult) SEM_CUDA_TRY(cudaMemcpy(mult, L.mult, L.nL * 4, cudaMemcpyDeviceToHost));
  if (dmask) SEM_CUDA_TRY(cudaMemcpy(dmask, L.dmask, L.nL, cudaMemcpyDeviceToHost));
  std::vector<int32_t> tmp;
  if (node || label) tmp.resize(L.nL);
  if (node) {
    SEM_CUDA_TRY(cudaMemcpy(tmp.data(), L.node, L.nL * 4, cudaMemcpyDeviceToHost));
    for (int64_t l = 0; l < L.nL; ++l) node[l] = tmp[l];
  }
  if (label) {
    SEM_CUDA_TRY(cudaMemcpy(tmp.data(), L.label, L.nL * 4, cudaMemcpyDeviceToHost));
    for (int64_t l = 0; l < L.nL; ++l) label[l] = tmp[l];
  }
  return SEM_OK;
}

int sem_get_geom(const sem_ctx* h, int level, double* G) {
  const Ctx* C = reinterpret_cast<const Ctx*>(h);
  if (!C || !G || level < 0 || level >= C->nlevels) {
    set_detail("bad context, output or level");
    return SEM_EINVAL;
  }
  const Level& L = C->lev[level];
  SEM_CUDA_TRY(cudaMemcpy(G, L.G, 7 * L.nL * 8, cudaMemcpyDeviceToHost));
  return SEM_OK;
}

int sem_get_geom_lowp(const sem_ctx* h, int level, int prec, void* G) {
  const Ctx* C = reinterpret_cast<const Ctx*>(h);
  if (!C || !G || level < 0 || level >= C->nlevels) {
    set_detail("bad context, output or level");
    return SEM_EINVAL;
  }
  const Level& L = C->lev[level];
  if (prec == SEM_FP32 && L.G32) SEM_CUDA_TRY(cudaMemcpy(G, L.G32, 7 * L.nL * 4, cudaMemcpyDeviceToHost));
  else if (prec == SEM_BF16G && L.G16) SEM_CUDA_TRY(cudaMemcpy(G, L.G16, 7 * L.nL * 2, cudaMemcpyDeviceToHost));
  else {
    set_detail("requested low-precision copy was not built");
    return SEM_EINVAL;
  }
  return SEM_OK;
}

int sem_get_coords(const sem_ctx* h, int level, double* x, double* y, double* z, int64_t* gid) {
  const Ctx* C = reinterpret_cast<const Ctx*>(h);
  if (!C || level < 0 || level >= C->nlevels) {
    set_detail("bad context or level");
    return SEM_EINVAL;
  }
  const Level& L = C->lev[level];
  if (x) SEM_CUDA_TRY(cudaMemcpy(x, L.x, L.nL * 8, cudaMemcpyDeviceToHost));
  if (y) SEM_CUDA_TRY(cudaMemcpy(y, L.y, L.nL * 8, cudaMemcpyDeviceToHost));
  if (z) SEM_CUDA_TRY(cudaMemcpy(z, L.z, L.nL * 8, cudaMemcpyDeviceToHost));
  if (gid) SEM_CUDA_TRY(cudaMemcpy(gid, L.gid, L.nL * 8, cudaMemcpyDeviceToHost));
  return SEM_OK;
}

int sem_gll(int N, double* xi, double* rho, double* D) {
  if (N < 1 || N > SEM_MAX_N) {
    set_detail("N = %d outside 1..%d", N, SEM_MAX_N);
    return SEM_EINVAL;
  }
  double x[16], r[16], d[144];
  host_gll(N, x, r);
  host_dhat(N, x, d);
  if (xi) std::memcpy(xi, x, (N + 1) * 8);
  if (rho) std::memcpy(rho, r, (N + 1) * 8);
  if (D) std::memcpy(D, d, (N + 1) * (N + 1) * 8);
  return SEM_OK;
}

}  // extern "C"
