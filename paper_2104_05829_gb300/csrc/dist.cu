// Element partitioning across GPUs and the interface exchange of the gather-scatter
// (Section 3.1, "Domain Partitioning", and Section 3.2, "Parallel Communication").
//
// A rank holds a subset of the elements with their global node ids. QQ^T of the whole
// mesh is then the rank's own gather-scatter plus, at the nodes it shares with other
// ranks (the interface), the other ranks' partial sums. The calls here are the
// rank-local pieces of that exchange:
//  * sem_partition_rcb: recursive coordinate bisection of element centroids (host),
//  * sem_ax_elements: the element operator on a range of elements, so that a rank can
//    apply it to the elements that touch the interface first and start the exchange
//    while the other elements are computed (the nonlocal-first overlap of Section 3.2),
//  * a halo: for a list of interface global ids, sem_halo_gather writes the rank's
//    partial sum of every interface node into a caller buffer at a caller-given
//    position, and sem_halo_scatter writes the completed sums back to every local copy.
// The exchange between the two (a sum over ranks of the buffers) is the caller's
// collective.
#include <algorithm>
#include <cmath>
#include <vector>

#include "sem_internal.cuh"

namespace sem {

struct Halo {
  Ctx* ctx = nullptr;
  int64_t n = 0;            // interface nodes held by this rank
  int64_t nbuf = 0;         // entries of the exchange buffer
  int64_t* seg = nullptr;   // [n] index of the node in the level's id list (copies idx[off[seg] .. off[seg+1]))
  int64_t* pos = nullptr;   // [n] position of the node in the exchange buffer
  int* bad = nullptr;       // [1] ids not found on this rank
};

namespace {

// seg[i] = k with ids[k] == gid[i] (ids ascending), or -1 when absent
__global__ void k_halo_find(int64_t n, const int64_t* __restrict__ gid, const int64_t* __restrict__ ids,
                            int64_t n_ids, int64_t* __restrict__ seg, int* bad) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t g = gid[i];
  int64_t lo = 0, hi = n_ids;   // first index with ids[k] >= g
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (ids[mid] < g) lo = mid + 1;
    else hi = mid;
  }
  if (lo < n_ids && ids[lo] == g) {
    seg[i] = lo;
  } else {
    seg[i] = -1;
    atomicExch(bad, 1);
  }
}

// buf[pos[i]] = sum of the local copies of node i, in ascending local index
__global__ void k_halo_gather(int64_t n, const int64_t* __restrict__ seg, const int64_t* __restrict__ pos,
                              const int64_t* __restrict__ off, const int32_t* __restrict__ idx,
                              const double* __restrict__ w, double* __restrict__ buf) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t k = seg[i];
  double s = 0.0;
  for (int64_t p = off[k]; p < off[k + 1]; ++p) s += w[idx[p]];
  buf[pos[i]] = s;
}

// every local copy of node i <- buf[pos[i]] (0 at Dirichlet nodes when mask is set)
__global__ void k_halo_scatter(int64_t n, const int64_t* __restrict__ seg, const int64_t* __restrict__ pos,
                               const int64_t* __restrict__ off, const int32_t* __restrict__ idx,
                               const uint8_t* __restrict__ dmask, const double* __restrict__ buf,
                               double* __restrict__ w, int mask) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t k = seg[i];
  const int64_t b = off[k], e = off[k + 1];
  const double v = (mask && dmask[idx[b]]) ? 0.0 : buf[pos[i]];
  for (int64_t p = b; p < e; ++p) w[idx[p]] = v;
}

inline unsigned nblk(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + 255) / 256); }

}  // namespace

}  // namespace sem

using namespace sem;

extern "C" {

int sem_partition_rcb(int32_t E, const double* cx, const double* cy, const double* cz, int32_t nparts,
                      int32_t* part) {
  if (E < 1 || nparts < 1 || nparts > E || !cx || !cy || !cz || !part) {
    set_detail("sem_partition_rcb: need 1 <= nparts <= E and non-NULL arrays");
    return SEM_EINVAL;
  }
  std::vector<double> c[3] = {std::vector<double>(cx, cx + E), std::vector<double>(cy, cy + E),
                              std::vector<double>(cz, cz + E)};
  std::vector<int32_t> el(E), el_off(nparts + 1);
  for (int32_t e = 0; e < E; ++e) el[e] = e;
  rcb(el.data(), E, nparts, 0, 0, c, el_off);
  el_off[nparts] = E;
  for (int32_t p = 0; p < nparts; ++p)
    for (int32_t q = el_off[p]; q < el_off[p + 1]; ++q) part[el[q]] = p;
  return SEM_OK;
}

int sem_ax_elements(sem_ctx* h, int32_t e0, int32_t e1, const double* u, double* w, const sem_coef* c, int flags,
                    void* stream) {
  Ctx* C = reinterpret_cast<Ctx*>(h);
  if (!C || !u || !w || !c || u == w || e0 < 0 || e1 < e0 || e1 > C->lev[0].E || (flags & ~SEM_AX_PAIRS)) {
    set_detail("sem_ax_elements: NULL or aliased vector, element range outside 0..E, or unknown flag");
    return SEM_EINVAL;
  }
  return ax_eo_apply_range(C->lev[0], e0, e1, u, w, c->h1, c->h2, c->h1_L, (flags & SEM_AX_PAIRS) != 0,
                           (cudaStream_t)stream);
}

int sem_halo_create(sem_ctx* h, int64_t n, const int64_t* gid, const int64_t* pos, int64_t nbuf,
                    sem_halo** out) {
  Ctx* C = reinterpret_cast<Ctx*>(h);
  if (out) *out = nullptr;
  if (!C || !out || n < 0 || nbuf < 0 || (n > 0 && (!gid || !pos))) {
    set_detail("sem_halo_create: NULL argument or negative size");
    return SEM_EINVAL;
  }
  for (int64_t i = 0; i < n; ++i)
    if (gid[i] <= 0 || pos[i] < 0 || pos[i] >= nbuf) {
      set_detail("sem_halo_create: id %lld must be positive and position %lld inside 0..%lld", (long long)gid[i],
                 (long long)pos[i], (long long)nbuf);
      return SEM_EINVAL;
    }
  Halo* H = new Halo();
  H->ctx = C;
  H->n = n;
  H->nbuf = nbuf;
  const Level& L = C->lev[0];
  cudaStream_t s = nullptr;
  int64_t* d_gid = nullptr;
  int bad = 0;
  auto fail = [&](int rc) {
    if (d_gid) cudaFree(d_gid);
    sem_halo_free(reinterpret_cast<sem_halo*>(H));
    return rc;
  };
  const size_t bytes = (size_t)std::max<int64_t>(n, 1) * sizeof(int64_t);
  if (cudaMalloc(&H->seg, bytes) != cudaSuccess || cudaMalloc(&H->pos, bytes) != cudaSuccess ||
      cudaMalloc(&H->bad, sizeof(int)) != cudaSuccess || cudaMalloc(&d_gid, bytes) != cudaSuccess) {
    cudaGetLastError();
    set_detail("sem_halo_create: cudaMalloc failed");
    return fail(SEM_ENOMEM);
  }
  cudaError_t e = cudaMemsetAsync(H->bad, 0, sizeof(int), s);
  if (e == cudaSuccess && n > 0) e = cudaMemcpyAsync(d_gid, gid, n * sizeof(int64_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && n > 0) e = cudaMemcpyAsync(H->pos, pos, n * sizeof(int64_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && n > 0) {
    k_halo_find<<<nblk(n), 256, 0, s>>>(n, d_gid, L.ids, L.n_ids, H->seg, H->bad);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, H->bad, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_detail("sem_halo_create: %s", cudaGetErrorString(e));
    return fail(SEM_ECUDA);
  }
  if (bad) {
    set_detail("sem_halo_create: an interface id is not held by this context");
    return fail(SEM_EINVAL);
  }
  cudaFree(d_gid);
  *out = reinterpret_cast<sem_halo*>(H);
  return SEM_OK;
}

void sem_halo_free(sem_halo* hh) {
  Halo* H = reinterpret_cast<Halo*>(hh);
  if (!H) return;
  if (H->seg) cudaFree(H->seg);
  if (H->pos) cudaFree(H->pos);
  if (H->bad) cudaFree(H->bad);
  delete H;
}

int sem_halo_gather(sem_halo* hh, const double* w, double* buf, void* stream) {
  Halo* H = reinterpret_cast<Halo*>(hh);
  if (!H || !w || !buf) {
    set_detail("sem_halo_gather: NULL argument");
    return SEM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (H->nbuf > 0) SEM_CUDA_TRY(cudaMemsetAsync(buf, 0, H->nbuf * sizeof(double), s));
  if (H->n == 0) return SEM_OK;
  const Level& L = H->ctx->lev[0];
  k_halo_gather<<<nblk(H->n), 256, 0, s>>>(H->n, H->seg, H->pos, L.off, L.idx, w, buf);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}

int sem_halo_scatter(sem_halo* hh, const double* buf, double* w, int flags, void* stream) {
  Halo* H = reinterpret_cast<Halo*>(hh);
  if (!H || !w || !buf || (flags & ~SEM_GS_ADD_MASK)) {
    set_detail("sem_halo_scatter: NULL argument or unknown flag");
    return SEM_EINVAL;
  }
  if (H->n == 0) return SEM_OK;
  const Level& L = H->ctx->lev[0];
  k_halo_scatter<<<nblk(H->n), 256, 0, (cudaStream_t)stream>>>(H->n, H->seg, H->pos, L.off, L.idx, L.dmask, buf,
                                                               w, (flags & SEM_GS_ADD_MASK) ? 1 : 0);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}

}  // extern "C"
