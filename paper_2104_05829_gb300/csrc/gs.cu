// Gather-scatter w_L <- QQ^T w_L (gs_op with +, Section 3.2) and
// the Dirichlet mask R^T R (footnote below eq. dssum).
//
// The segments are the global nodes that need work: nodes with more than one
// local copy and Dirichlet nodes. Interior (singleton) points are never touched.
// Every segment's copies are summed in ascending local-index order (a fixed
// order, so results are reproducible) and the sum is written back to every copy;
// a Dirichlet segment writes zeros when the mask is requested.
//
// One launch covers four classes of segments, one class per thread block: the
// non-Dirichlet nodes with 2, 4 and 8 copies (face, edge and vertex nodes of a
// conforming hexahedral mesh) read their copies' local indices from fixed-stride
// tables (one 8- or 16-byte load, no offsets, no branches), and every other segment
// (Dirichlet nodes, other multiplicities) takes the general CSR path. With one
// thread per segment each thread issues all its loads before its first add.
#include "sem_internal.cuh"

namespace sem {

namespace {

constexpr int GS_T = 256;

struct GsTables {
  const int2* t2;
  const int4* t4;
  const int4* t8;
  const int32_t* tr;
  const int32_t* off;
  const int32_t* idx;
  const uint8_t* sdir;
  int64_t n2, n4, n8, nr;
  int64_t b2, b4, b8;   // blocks of the first three classes
};

template <typename T>
__global__ void __launch_bounds__(GS_T) k_gs(GsTables t, T* __restrict__ w, int mask, const double* skip) {
  if (skip && *skip != 0.0) return;
  int64_t b = blockIdx.x;
  if (b < t.b2) {
    const int64_t i = b * GS_T + threadIdx.x;
    if (i >= t.n2) return;
    const int2 q = t.t2[i];
    const T v0 = w[q.x], v1 = w[q.y];
    const T sum = v0 + v1;
    w[q.x] = sum;
    w[q.y] = sum;
    return;
  }
  b -= t.b2;
  if (b < t.b4) {
    const int64_t i = b * GS_T + threadIdx.x;
    if (i >= t.n4) return;
    const int4 q = t.t4[i];
    const T v0 = w[q.x], v1 = w[q.y], v2 = w[q.z], v3 = w[q.w];
    T sum = v0 + v1;
    sum += v2;
    sum += v3;
    w[q.x] = sum;
    w[q.y] = sum;
    w[q.z] = sum;
    w[q.w] = sum;
    return;
  }
  b -= t.b4;
  if (b < t.b8) {
    const int64_t i = b * GS_T + threadIdx.x;
    if (i >= t.n8) return;
    const int4 q = t.t8[2 * i], r = t.t8[2 * i + 1];
    const int id[8] = {q.x, q.y, q.z, q.w, r.x, r.y, r.z, r.w};
    T v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = w[id[k]];
    T sum = v[0];
#pragma unroll
    for (int k = 1; k < 8; ++k) sum += v[k];
#pragma unroll
    for (int k = 0; k < 8; ++k) w[id[k]] = sum;
    return;
  }
  b -= t.b8;
  const int64_t i = b * GS_T + threadIdx.x;
  if (i >= t.nr) return;
  const int32_t sgi = t.tr[i];
  const int bo = t.off[sgi], e = t.off[sgi + 1], m = e - bo;
  if (mask && t.sdir[sgi]) {
    for (int p = bo; p < e; ++p) w[t.idx[p]] = T(0);
    return;
  }
  if (m < 2) return;
  if (m <= 8) {
    int id[8];
    T v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) id[k] = k < m ? t.idx[bo + k] : 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = k < m ? w[id[k]] : T(0);
    T sum = v[0];
#pragma unroll
    for (int k = 1; k < 8; ++k)
      if (k < m) sum += v[k];
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (k < m) w[id[k]] = sum;
    return;
  }
  T sum = w[t.idx[bo]];
  for (int p = bo + 1; p < e; ++p) sum += w[t.idx[p]];
  for (int p = bo; p < e; ++p) w[t.idx[p]] = sum;
}

inline int64_t blocks_for(int64_t n) { return (n + GS_T - 1) / GS_T; }

}  // namespace

int gs_apply_skip(const Level& L, int prec, void* w, bool mask, const double* skip, cudaStream_t s) {
  if (L.n_seg == 0) return SEM_OK;
  GsTables t{L.gs2, L.gs4, L.gs8, L.gsr, L.seg_off, L.seg_idx, L.seg_dir, L.n_gs2, L.n_gs4, L.n_gs8, L.n_gsr,
             blocks_for(L.n_gs2), blocks_for(L.n_gs4), blocks_for(L.n_gs8)};
  const int64_t nb = t.b2 + t.b4 + t.b8 + blocks_for(L.n_gsr);
  if (nb == 0) return SEM_OK;
  if (prec == SEM_FP64)
    k_gs<double><<<(unsigned)nb, GS_T, 0, s>>>(t, (double*)w, mask ? 1 : 0, skip);
  else
    k_gs<float><<<(unsigned)nb, GS_T, 0, s>>>(t, (float*)w, mask ? 1 : 0, skip);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}

int gs_apply(const Level& L, int prec, void* w, bool mask, cudaStream_t s) {
  return gs_apply_skip(L, prec, w, mask, nullptr, s);
}

}  // namespace sem
