// Gather-scatter w_L <- QQ^T w_L (gs_op with +, Section 3.2) and
// the Dirichlet mask R^T R (footnote below eq. dssum).
//
// The segments are the global nodes that need work: nodes with more than one
// local copy and Dirichlet nodes. Interior (singleton) points are never touched.
// One thread per segment sums its copies in ascending local-index order (a
// fixed order, so results are reproducible) and writes the sum back to every
// copy; a Dirichlet segment writes zeros when the mask is requested. Segments of
// up to eight copies (every node of a conforming hexahedral mesh) issue all their
// index and value loads before the first add.
#include "sem_internal.cuh"

namespace sem {

namespace {

template <typename T>
__global__ void k_gs(int64_t nseg, const int32_t* __restrict__ off, const int32_t* __restrict__ idx,
                     const uint8_t* __restrict__ sdir, T* __restrict__ w, int mask, const double* skip) {
  if (skip && *skip != 0.0) return;
  const int64_t sgi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (sgi >= nseg) return;
  const int b = off[sgi], e = off[sgi + 1], m = e - b;
  if (mask && sdir[sgi]) {
    for (int p = b; p < e; ++p) w[idx[p]] = T(0);
    return;
  }
  if (m < 2) return;
  if (m <= 8) {
    int id[8];
    T v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) id[t] = t < m ? idx[b + t] : 0;
#pragma unroll
    for (int t = 0; t < 8; ++t) v[t] = t < m ? w[id[t]] : T(0);
    T s = v[0];
#pragma unroll
    for (int t = 1; t < 8; ++t)
      if (t < m) s += v[t];
#pragma unroll
    for (int t = 0; t < 8; ++t)
      if (t < m) w[id[t]] = s;
    return;
  }
  T s = w[idx[b]];
  for (int p = b + 1; p < e; ++p) s += w[idx[p]];
  for (int p = b; p < e; ++p) w[idx[p]] = s;
}

}  // namespace

int gs_apply_skip(const Level& L, int prec, void* w, bool mask, const double* skip, cudaStream_t s) {
  if (L.n_seg == 0) return SEM_OK;
  const int T = 256;
  const unsigned nb = (unsigned)((L.n_seg + T - 1) / T);
  if (prec == SEM_FP64)
    k_gs<double><<<nb, T, 0, s>>>(L.n_seg, L.seg_off, L.seg_idx, L.seg_dir, (double*)w, mask ? 1 : 0, skip);
  else
    k_gs<float><<<nb, T, 0, s>>>(L.n_seg, L.seg_off, L.seg_idx, L.seg_dir, (float*)w, mask ? 1 : 0, skip);
  SEM_LAUNCH_CHECK();
  return SEM_OK;
}

int gs_apply(const Level& L, int prec, void* w, bool mask, cudaStream_t s) {
  return gs_apply_skip(L, prec, w, mask, nullptr, s);
}

}  // namespace sem
