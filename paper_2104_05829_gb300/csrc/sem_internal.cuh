// Internal declarations shared by the libsem translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "sem.h"

namespace sem {

// ----------------------------------------------------------------------------
// Error plumbing: every entry point returns a status; the last failure's text
// is kept per host thread for sem_last_error_detail.
// ----------------------------------------------------------------------------
void set_detail(const char* fmt, ...);

#define SEM_CUDA_TRY(call)                                                             \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      ::sem::set_detail("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
      return SEM_ECUDA;                                                                \
    }                                                                                  \
  } while (0)

#define SEM_LAUNCH_CHECK() SEM_CUDA_TRY(cudaGetLastError())

#define SEM_TRY(expr)          \
  do {                         \
    int rc_ = (expr);          \
    if (rc_ != SEM_OK) return rc_; \
  } while (0)

// Small dense matrices passed to kernels by value (they land in the kernel's
// constant parameter bank; kernels copy them to shared memory where the index
// depends on the thread).
struct Mat64 {
  double a[144];
};
struct Mat32 {
  float a[144];
};

inline int np3(int N) { return (N + 1) * (N + 1) * (N + 1); }

// Host-side 1-D rule for order N (GLL nodes ascending, weights, D_hat row-major
// D[a*(N+1)+b] = h_b'(xi_a), eq. dh).
void host_gll(int N, double* xi, double* rho);
void host_dhat(int N, const double* xi, double* D);
// J[a*nc + b] = h_b(x_a) for cardinal polynomials on xi_from (nc nodes) at points x_to.
void host_interp(int nc, const double* xi_from, int nt, const double* x_to, double* J);

struct Level {
  int N = 0, NP = 0, E = 0;
  long long spin_limit = 1ll << 31;   // SM clocks a device-side wait of this level's kernels may spin
  // nodal h1 of a preconditioner set up with a nodal coefficient: the fine values,
  // carried level by level to the coarser GLL points (allocated on first use)
  double* h1n = nullptr;              // [nL]
  // the coarsest level's factors with G11..G33 times h1n (B kept), for the one-launch
  // coarse solve, which takes a scalar h1; current while pc_scaled is set
  double* pcG = nullptr;
  float* pcG32 = nullptr;
  __nv_bfloat16* pcG16 = nullptr;
  bool pc_scaled = false;
  int64_t nL = 0, nG = 0, n_ids = 0, n_idx = 0, n_seg = 0, n_seg_idx = 0;
  Mat64 D{};                 // D_hat of this order
  Mat32 Df{};
  double xi[16] = {0}, rho[16] = {0};
  // geometry: [E][7][NP^3] with components G11 G12 G13 G22 G23 G33 B
  double* G = nullptr;
  float* G32 = nullptr;
  __nv_bfloat16* G16 = nullptr;
  float2* G2 = nullptr;        // (hi, lo) FP32 split of G for the pair-arithmetic kernel
  // coordinates, ids and Dirichlet flags as given (fine) or derived (coarse)
  double *x = nullptr, *y = nullptr, *z = nullptr;
  int64_t* gid = nullptr;
  uint8_t* dflag = nullptr;
  // canonical gather-scatter maps
  int64_t* ids = nullptr;    // [n_ids]
  int64_t* off = nullptr;    // [n_ids+1]
  int32_t* idx = nullptr;    // [n_idx]
  int32_t* mult = nullptr;   // [nL]
  int32_t* node = nullptr;   // [nL]
  int32_t* label = nullptr;  // [nL]
  uint8_t* dmask = nullptr;  // [nL] 1 at Dirichlet nodes
  uint8_t* owner = nullptr;  // [nL] 1 at the smallest-index copy of each non-Dirichlet node
  double* cwt = nullptr;     // [nL] counting weight 1/m
  float* cwt32 = nullptr;
  // gather-scatter segments: nodes that are shared or Dirichlet
  int32_t* seg_off = nullptr;  // [n_seg+1]
  int32_t* seg_idx = nullptr;  // [n_seg_idx]
  uint8_t* seg_dir = nullptr;  // [n_seg]
  // interpolation from level+1 (coarse) to this level: J[a*NPc + b] = h^c_b(xi^f_a)
  Mat64 Jc{};
  Mat32 Jcf{};
  // preconditioner state
  double* dinv = nullptr;
  float* dinv32 = nullptr;
  double lmax = 0.0;
  // V-cycle work vectors (allocated in the precision of the build: FP64 and FP32 sets)
  double *vb = nullptr, *vx = nullptr, *vr = nullptr, *vd = nullptr, *vw = nullptr;
  float *fb = nullptr, *fx = nullptr, *fr = nullptr, *fd = nullptr, *fw = nullptr;
  double *cp = nullptr;      // extra FP64 vector (coarse PCG direction)
  float *cpf = nullptr;
  // overlapping Schwarz smoother (asm.cu; built on first use)
  bool sch_ready = false;
  int32_t* sch_layer = nullptr;   // [E][6][NP*NP] local index of each face-layer node, -1 without neighbour
  uint8_t* sch_bt = nullptr;      // [E][6] side types: 0 neighbour, 1 Dirichlet boundary, 2 Neumann boundary
  double* sch_len = nullptr;      // [E][3] mean element lengths along r, s, t
  float* sch_len32 = nullptr;
  double* sch_ref = nullptr;      // [9][(N+3)^2 + (N+3)] reference 1-D eigenvectors and eigenvalues per side pair
  float* sch_ref32 = nullptr;
  double* sch_w = nullptr;        // [nL] Schwarz weights 1/count, 0 at Dirichlet nodes
  float* sch_w32 = nullptr;
  double* sch_zf = nullptr;       // [E][6][NP*NP] staged face-layer outputs
  float* sch_zf32 = nullptr;
  int32_t* sch_woff = nullptr;    // [nw+1] CSR offsets of the work nodes of the Schwarz sum
  int32_t* sch_witem = nullptr;   // copies (local index >= 0), then staged slots (-slot - 1)
  uint8_t* sch_wdir = nullptr;    // [nw] Dirichlet work nodes (written as zero)
  int2* sch_wpair = nullptr;      // [np] (copy, slot) of the nodes with one copy and one staged value
  int64_t sch_nw = 0, sch_np = 0;
  // sub-domain coarse solve (coarse_pipe.cu; built on first use at order 1)
  int pp_blocks = 0;              // sub-domains, one block each; 0 not built, -1 does not apply
  int pp_max_el = 0, pp_max_nd = 0, pp_max_cp = 0;   // largest sub-domain: elements, nodes, copy entries
  int pp_nsm = 0;                 // SMs of the device the sub-domains were built for
  int32_t* pp_el_off = nullptr;   // [B+1] offsets into pp_el
  int32_t* pp_el = nullptr;       // [E] elements grouped by sub-domain, ascending within one
  int32_t* pp_p2n = nullptr;      // [nL] per point in pp_el order: sub-domain node | bit 31 when published
  int32_t* pp_nd_off = nullptr;   // [B+1] offsets into the node arrays
  int32_t* pp_nd_src = nullptr;   // one local point of each sub-domain node (b and D^-1 are read there)
  uint8_t* pp_nd_fl = nullptr;    // bit 0: the sub-domain holds the owner copy; bit 1: Dirichlet
  int32_t* pp_cp_off = nullptr;   // [nodes + 1] offsets into pp_cp
  int32_t* pp_cp = nullptr;       // copies in canonical order: >= 0 sub-domain point, < 0 -(local point + 1)
  double* pp_xbuf = nullptr;      // [2][nL] exchange buffer of tagged words (16 bytes per value)
  double* pp_part = nullptr;      // [2][3][B] tagged block partials (16 bytes each)
};

// Device scalar slots (double) used by the Krylov kernels.
enum Scal {
  S_RZ = 0,      // (r, z)
  S_PW,          // (p, w)
  S_ALPHA,
  S_RR,          // (r, r)
  S_RZN,         // (r, z) new
  S_ZDR,         // (z, r_new - r_old)
  S_BETA,
  S_BB,          // (b, b)
  S_DONE,        // nonzero: the loop has converged; kernels become no-ops
  S_BREAK,       // nonzero: breakdown seen
  S_TOL2,        // tol^2 * (b,b) for device-side convergence tests
  S_ITER,        // iterations counted on the device
  S_TOTAL,       // iterations summed over every loop started since the last reset
  S_NSLOTS
};

// Dealiased advection data of level 0 (advect.cu; built on first use)
struct AdvData {
  bool ready = false;
  int nq = 0;
  double* Gq = nullptr;      // [E][9][nq^3] w J dr_d/dx_m at the Gauss points
  float* Gq32 = nullptr;
  float2* Gq2 = nullptr;      // FP32-pair split of Gq (built on the first pair evaluation)
  double *Im = nullptr, *Dq = nullptr, *wq = nullptr;   // GLL -> Gauss interpolation, Gauss derivative, weights
  float *Im32 = nullptr, *Dq32 = nullptr;
  float2 *Im2 = nullptr, *Dq2 = nullptr;
  double hIm[14 * 9] = {0};   // host copies (nq <= 14, N + 1 <= 9)
  double hDq[14 * 14] = {0};
  // characteristics substeps: inverse assembled mass and RK workspace (allocated on first use)
  double* minv = nullptr;     // [nL] 1 / (QQ^T B_L)
  float* minv32 = nullptr;
  void* ws = nullptr;         // bytes: 3 stage arrays of ncomp L-vectors + one wind (3 L-vectors)
  size_t ws_bytes = 0;
};

struct Ctx {
  int device = 0;
  int nlevels = 0;
  Level lev[SEM_MAX_LEVELS];
  sem_opts opts{};
  // deterministic reduction scratch
  double* red_part = nullptr;       // [RED_BLOCKS * 4]
  unsigned int* red_ticket = nullptr;
  double* scal = nullptr;           // [4 * S_NSLOTS]: outer, coarse, spare
  double* h_scal = nullptr;         // pinned mirror
  // fine-level FP64 solver workspace
  double *r = nullptr, *z = nullptr, *p = nullptr, *w = nullptr, *t = nullptr;
  // preconditioner
  bool pc_ready = false;
  int pc_prec = SEM_FP64;
  double pc_h1 = 0, pc_h2 = 0;
  cudaEvent_t ev = nullptr;
  cudaEvent_t cev[2] = {nullptr, nullptr};   // coarse-solve batch markers
  double* h_done = nullptr;                  // pinned, 2 slots
  AdvData adv;
  // the preconditioner step of a flexible-CG iteration (V-cycle, beta, direction)
  // as a CUDA graph, captured on a library stream and replayed on the caller's
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t pc_graph = nullptr;
  const void* pc_graph_key[3] = {nullptr, nullptr, nullptr};   // w, sc, level-0 x the graph was captured with
  int pc_graph_prec = -1;
  uint64_t pc_graph_gen = 0;                 // pc_gen at capture
  uint64_t pc_gen = 0;                       // bumped by every preconditioner set-up
  bool pc_graph_off = false;                 // a capture failed: direct launches from then on
  int graph_steps = 0;                       // graph replays in the current solve
  bool pc_nodal = false;                     // the preconditioner was set up with a nodal h1
  const double* pc_h1L = nullptr;            // the caller's fine-level h1 it was set up with
  // error flag of the one-launch coarse solve (set when a bounded wait gives up)
  int* cg_err = nullptr;                     // [1]
};

// 8 per SM on a 152-SM GB300 (64 warps: enough loads in flight while warps wait on
// the narrow FP64 pipe); fixed for determinism
constexpr int RED_BLOCKS = 1216;
constexpr int RED_THREADS = 256;

// ---- ax.cu
int ax_apply(const Level& L, int prec, const void* u, void* w, double h1, double h2, const double* h1L,
             cudaStream_t s, const double* skip = nullptr);
// a nodal field of level F at the GLL points of the next coarser level C (setup.cu), the way
// the coarse coordinates are formed (the fine element interpolant at the coarse points)
int interp_nodal(const Level& F, const Level& C, const double* f, double* c, cudaStream_t s);
int diag_local(const Level& L, double h1, double h2, const double* h1L, double* d, cudaStream_t s);
int grad_h1_apply(const Level& L, const double* u, const double* lam, double* g, cudaStream_t s);
int geom_compute(Level& L, int* d_bad, cudaStream_t s);

// ---- ax_eo.cu (FP64 element operator, even-odd contractions)
int ax_eo_apply(const Level& L, const double* u, double* w, double h1, double h2, const double* h1L,
                const double* skip, cudaStream_t s);

// elements [e0, e1) of the level only (u, w, h1L: whole-level L-vectors)
int ax_eo_apply_range(const Level& L, int e0, int e1, const double* u, double* w, double h1, double h2,
                      const double* h1L, bool pairs, cudaStream_t s);

// ---- ax_eo.cu (FP32-pair variant)
int pairs_build(Level& L, cudaStream_t s);
int ax_pairs_apply(const Level& L, const double* u, double* w, double h1, double h2, const double* h1L,
                   cudaStream_t s);

// ---- coarse_pipe.cu: recursive coordinate bisection (host): el[0..n) goes to parts
// part0 .. part0 + parts - 1 (el_off[part] = first position), sizes within one of each
// other, each part's elements ascending; c[3][E] are the element centroids
void rcb(int32_t* el, int n, int parts, int part0, int32_t base, const std::vector<double>* c,
         std::vector<int32_t>& el_off);

// ---- coarse_pipe.cu: one-launch pipelined coarse Jacobi-PCG on sub-domains (cooperative launch)
int coarse_pipe_build(Level& L, cudaStream_t s);
// outer_sc: the calling solve's scalar slots (S_BREAK and S_DONE are set there when a wait gives up)
int coarse_pipe_solve(Level& L, int prec, const void* b, void* x, const void* dinv, double h1, double h2,
                      double tol, int maxit, double* sc, int* err, double* outer_sc, cudaStream_t s, bool* used);

// ---- gs.cu
int gs_apply(const Level& L, int prec, void* w, bool mask, cudaStream_t s);
int gs_apply_skip(const Level& L, int prec, void* w, bool mask, const double* skip, cudaStream_t s);

// ---- gsmap.cu
int build_maps(Level& L, cudaStream_t s);

// ---- blas.cu
int vec_fill(void* v, int prec, int64_t n, double val, cudaStream_t s);
int vec_copy_convert(const void* src, int sprec, void* dst, int dprec, int64_t n, cudaStream_t s);
int dot_owner(Ctx& C, const Level& L, int prec, const void* a, const void* b, double* d_out, cudaStream_t s);
int dinv_finalize(const Level& L, double* d, cudaStream_t s);
int dinv_finalize(const Level& L, double* d, float* d32, cudaStream_t s);
int rhs_mass(const Level& L, const double* f, double* b, cudaStream_t s);
int mul_counting_weight(const Level& L, int prec, const void* in, void* out, cudaStream_t s);

// Krylov / smoother kernels (blas.cu)
int pcg_begin_tol(Ctx& C, const Level& L, int prec, const void* b, const void* w, void* x, void* r,
                  const void* dinv, void* p, double* sc, double tol, cudaStream_t s,
                  const double* bbref = nullptr);
int kr_alpha(Ctx& C, const Level& L, int prec, const void* p, const void* w, double* sc, cudaStream_t s);
int kr_update_jacobi(Ctx& C, const Level& L, int prec, void* x, const void* p, void* r, const void* w,
                     const void* dinv, double* sc, cudaStream_t s);
int kr_direction_jacobi(const Level& L, int prec, void* p, const void* r, const void* dinv, double* sc,
                        cudaStream_t s);
// flexible CG: rb (may be null) receives r in the V-cycle's type rb_prec; z is the
// V-cycle's output in type z_prec; w = null in kr_beta_flex gives beta = 0
int kr_update_flex(Ctx& C, const Level& L, double* x, const double* p, double* r, const double* w, void* rb,
                   int rb_prec, double* sc, cudaStream_t s);
int kr_beta_flex(Ctx& C, const Level& L, const void* z, int z_prec, const double* r, const double* w, double* sc,
                 cudaStream_t s);
int kr_direction(const Level& L, double* p, const void* z, int z_prec, double* sc, cudaStream_t s);
int cheb_first(const Level& L, int prec, const void* b, const void* w, void* x, void* d, bool x_zero,
               double inv_theta, cudaStream_t s);
int cheb_step(const Level& L, int prec, const void* b, const void* w, void* x, void* d, double c1, double c2,
              cudaStream_t s);
int residual_weighted(const Level& L, int prec, const void* b, const void* w, void* out, cudaStream_t s);

// ---- asm.cu: overlapping Schwarz smoother with fast-diagonalisation local solves
int schwarz_build(Ctx& C, Level& L, cudaStream_t s);
int asm_sum(const Level& L, int prec, const void* b, const void* w, void* z, double h1, double h2, cudaStream_t s);
int asm_weight(const Level& L, int prec, void* z, cudaStream_t s);
int cheb_w_update(const Level& L, int prec, const void* z, void* x, void* d, double c1, double c2, bool first,
                  bool x_zero, cudaStream_t s);
int arnoldi_lmax_asm(Ctx& C, int l, double h1, double h2, const double* v0, int steps, cudaStream_t s,
                     double* lam);

// ---- advect.cu: dealiased advection operator
int advect_build(Ctx& C, cudaStream_t s);
void advect_free(AdvData& A);
int advect_apply(Ctx& C, int prec, const void* c, const void* u, void* w, int ncomp, cudaStream_t s);
int char_advance(Ctx& C, int prec, const void* c0, const void* c1, void* w, int ncomp, double t0, double t1,
                 int nsub, cudaStream_t s);

// ---- proj.cu: projection of successive right-hand sides
struct Proj;
void proj_bind_coef(Proj& P, const sem_coef* c, bool pairs);
int proj_project(Proj& P, const double* b, double* xbar, double* r0, cudaStream_t s);
int proj_update(Proj& P, const sem_coef* c, bool pairs, const double* x, const double* dx, int* added,
                cudaStream_t s);
int proj_add_xbar(Proj& P, double* u, cudaStream_t s);
int proj_state(const Proj& P, int* count, int* maxv, double** xbar, const double** bb_dev, double* h_bb_rr0,
               cudaStream_t s);
bool proj_belongs(const Proj& P, const Ctx* C);

// ---- solve.cu
// h1L: NULL for the scalar h1, else the fine-level nodal h1 (DEVICE; CHEBY-JAC only)
int precond_setup(Ctx& C, double h1, double h2, int prec, cudaStream_t s, const double* h1L = nullptr);
int vcycle(Ctx& C, int prec, const double* r, double* z, cudaStream_t s);

// ---- transfer (ax.cu)
int interp_add(const Level& F, const Level& Cl, int prec, const void* ec, void* xf, cudaStream_t s);
int interp_T(const Level& F, const Level& Cl, int prec, const void* rf, void* rc, cudaStream_t s);
// rc = J^T (cwt_f * (bf - wf)) without assembly (wf may be null)
int restrict_residual(const Level& F, const Level& Cl, int prec, const void* bf, const void* wf, void* rc,
                      cudaStream_t s);

// helpers
inline size_t prec_size(int prec) { return prec == SEM_FP64 ? 8 : 4; }

// Launch set-up that is done once per device and remembered (a kernel's shared-
// memory attribute, an occupancy query), so that launches later captured into a
// CUDA graph issue no such calls. Each device keeps its own entry, filled under a
// lock: a second device, or another host thread, does its own set-up.
constexpr int MAX_DEVICES = 64;
template <typename V>
struct PerDevice {
  std::mutex m;
  V v[MAX_DEVICES] = {};
};
inline int current_device(int* dev) {
  SEM_CUDA_TRY(cudaGetDevice(dev));
  if (*dev < 0 || *dev >= MAX_DEVICES) {
    set_detail("device ordinal %d out of range", *dev);
    return SEM_EINVAL;
  }
  return SEM_OK;
}
// Set the dynamic shared-memory limit of kernel f to `bytes` on the current device,
// once per device.
inline int smem_attr_once(PerDevice<bool>& cache, const void* f, size_t bytes) {
  int dev = 0;
  SEM_TRY(current_device(&dev));
  std::lock_guard<std::mutex> lock(cache.m);
  if (!cache.v[dev]) {
    SEM_CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    cache.v[dev] = true;
  }
  return SEM_OK;
}

}  // namespace sem
