// gs_setup on the device: canonical gather-scatter maps from per-point global
// ids (Section 3.2, "Parallel Communication": ids are global pointers, positions are local
// pointers, 0 marks a singleton).
//
// The (id, local index) pairs with a nonzero id are sorted by a stable LSD
// radix sort on the id (8-bit digits, as many passes as the largest id needs).
// The input is in ascending local-index order and every pass is stable, so the
// result is ordered by (id, local index): the canonical order. Runs of equal
// ids are the global nodes.
#include "sem_internal.cuh"

namespace sem {

namespace {

constexpr int SCAN_T = 256, SCAN_I = 8, SCAN_TILE = SCAN_T * SCAN_I;

// Exclusive scan of int64 values, tile by tile; tile totals go to `sums`.
__global__ void k_scan_tiles(const int64_t* __restrict__ in, int64_t* __restrict__ out, int64_t n,
                             int64_t* __restrict__ sums) {
  __shared__ int64_t s_w[SCAN_T / 32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_I;
  int64_t v[SCAN_I];
  int64_t tot = 0;
#pragma unroll
  for (int q = 0; q < SCAN_I; ++q) {
    const int64_t p = base + q;
    v[q] = p < n ? in[p] : 0;
    tot += v[q];
  }
  // inclusive warp scan of thread totals
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t x = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[warp] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t run = 0;
    for (int w = 0; w < SCAN_T / 32; ++w) {
      const int64_t t = s_w[w];
      s_w[w] = run;
      run += t;
    }
    sums[blockIdx.x] = run;
  }
  __syncthreads();
  int64_t run = s_w[warp] + x - tot;
#pragma unroll
  for (int q = 0; q < SCAN_I; ++q) {
    const int64_t p = base + q;
    if (p < n) out[p] = run;
    run += v[q];
  }
}

__global__ void k_scan_add(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ offs) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p < n) out[p] += offs[p / SCAN_TILE];
}

// Exclusive scan; *total (host) receives the sum. Allocates its scratch.
int scan_excl(const int64_t* in, int64_t* out, int64_t n, int64_t* total, cudaStream_t s) {
  if (n == 0) {
    if (total) *total = 0;
    return SEM_OK;
  }
  const int64_t nt = (n + SCAN_TILE - 1) / SCAN_TILE;
  int64_t* sums = nullptr;
  int64_t* soff = nullptr;
  SEM_CUDA_TRY(cudaMallocAsync(&sums, nt * sizeof(int64_t), s));
  SEM_CUDA_TRY(cudaMallocAsync(&soff, nt * sizeof(int64_t), s));
  k_scan_tiles<<<(unsigned)nt, SCAN_T, 0, s>>>(in, out, n, sums);
  SEM_LAUNCH_CHECK();
  int64_t sub_total = 0;
  int rc = SEM_OK;
  if (nt > 1) {
    rc = scan_excl(sums, soff, nt, &sub_total, s);
    if (rc == SEM_OK) {
      k_scan_add<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, n, soff);
      SEM_LAUNCH_CHECK();
    }
  } else {
    SEM_CUDA_TRY(cudaMemcpyAsync(&sub_total, sums, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SEM_CUDA_TRY(cudaStreamSynchronize(s));
  }
  if (total) *total = sub_total;
  SEM_CUDA_TRY(cudaFreeAsync(sums, s));
  SEM_CUDA_TRY(cudaFreeAsync(soff, s));
  return rc;
}

// ---- radix sort pieces -------------------------------------------------------
constexpr int RAD_T = 256, RAD_CHUNKS = 16, RAD_TILE = RAD_T * RAD_CHUNKS, RAD_W = RAD_T / 32;

__global__ void k_rad_hist(const int64_t* __restrict__ key, int64_t n, int shift, int64_t* __restrict__ hist,
                           int64_t nblk) {
  __shared__ int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RAD_TILE;
  for (int c = 0; c < RAD_CHUNKS; ++c) {
    const int64_t p = base + c * RAD_T + threadIdx.x;
    if (p < n) atomicAdd(&h[((uint64_t)key[p] >> shift) & 0xFF], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_rad_scatter(const int64_t* __restrict__ key, const int32_t* __restrict__ val, int64_t n,
                              int shift, const int64_t* __restrict__ offs, int64_t nblk,
                              int64_t* __restrict__ key2, int32_t* __restrict__ val2) {
  __shared__ int s_wc[RAD_W][256];
  __shared__ int s_base[256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  s_base[threadIdx.x] = 0;
  const int64_t base = (int64_t)blockIdx.x * RAD_TILE;
  const unsigned lt = (1u << lane) - 1u;
  for (int c = 0; c < RAD_CHUNKS; ++c) {
#pragma unroll
    for (int w = 0; w < RAD_W; ++w) s_wc[w][threadIdx.x] = 0;
    __syncthreads();
    const int64_t p = base + c * RAD_T + threadIdx.x;
    const int d = p < n ? (int)(((uint64_t)key[p] >> shift) & 0xFF) : 256;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & lt);
    if (d < 256 && rank == 0) s_wc[warp][d] = __popc(peers);
    __syncthreads();
    {
      const int dg = threadIdx.x;
      int run = s_base[dg];
#pragma unroll
      for (int w = 0; w < RAD_W; ++w) {
        const int t = s_wc[w][dg];
        s_wc[w][dg] = run;
        run += t;
      }
      s_base[dg] = run;
    }
    __syncthreads();
    if (d < 256) {
      const int64_t dest = offs[(int64_t)d * nblk + blockIdx.x] + s_wc[warp][d] + rank;
      key2[dest] = key[p];
      val2[dest] = val[p];
    }
    __syncthreads();
  }
}

// ---- map construction kernels -------------------------------------------------
__global__ void k_nonzero_flags(const int64_t* __restrict__ gid, int64_t n, int64_t* __restrict__ fnz,
                                int64_t* __restrict__ fz, int* bad) {
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= n) return;
  const int64_t g = gid[l];
  if (g < 0) atomicExch(bad, 1);
  fnz[l] = g > 0;
  fz[l] = g == 0;
}

__global__ void k_compact_nz(const int64_t* __restrict__ gid, int64_t n, const int64_t* __restrict__ pos,
                             int64_t* __restrict__ key, int32_t* __restrict__ val) {
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= n) return;
  const int64_t g = gid[l];
  if (g > 0) {
    key[pos[l]] = g;
    val[pos[l]] = (int32_t)l;
  }
}

__global__ void k_max_key(const int64_t* __restrict__ key, int64_t n, unsigned long long* out) {
  uint64_t m = 0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    m = max(m, (uint64_t)key[p]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, (uint64_t)__shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)m);
}

__global__ void k_heads(const int64_t* __restrict__ key, int64_t n, int64_t* __restrict__ head) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= n) return;
  head[p] = (p == 0 || key[p] != key[p - 1]) ? 1 : 0;
}

// seg id of position p = inclusive count of heads up to p, minus one
__global__ void k_ids_off(const int64_t* __restrict__ key, const int64_t* __restrict__ head,
                          const int64_t* __restrict__ hscan, int64_t n, int64_t* __restrict__ ids,
                          int64_t* __restrict__ off, int64_t nids) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p == 0) off[nids] = n;
  if (p >= n) return;
  if (head[p]) {
    const int64_t s = hscan[p];
    ids[s] = key[p];
    off[s] = p;
  }
}

__global__ void k_per_point_nz(const int64_t* __restrict__ off, const int32_t* __restrict__ idx, int64_t nids,
                               const uint8_t* __restrict__ dflag, int32_t* __restrict__ mult,
                               int32_t* __restrict__ node, int32_t* __restrict__ label, uint8_t* __restrict__ dmask,
                               int64_t* __restrict__ segflag, int64_t* __restrict__ seglen) {
  const int64_t sg = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (sg >= nids) return;
  const int64_t b = off[sg], e = off[sg + 1];
  const int m = (int)(e - b);
  const int32_t lab = idx[b];
  uint8_t dir = 0;
  for (int64_t p = b; p < e; ++p) dir |= (dflag ? dflag[idx[p]] : 0);
  dir = dir ? 1 : 0;
  for (int64_t p = b; p < e; ++p) {
    const int32_t l = idx[p];
    mult[l] = m;
    node[l] = (int32_t)sg;
    label[l] = lab;
    dmask[l] = dir;
  }
  const bool keep = m > 1 || dir;
  segflag[sg] = keep;
  seglen[sg] = keep ? m : 0;
}

__global__ void k_per_point_zero(const int64_t* __restrict__ gid, int64_t n, const int64_t* __restrict__ zpos,
                                 int64_t nids, const uint8_t* __restrict__ dflag, int32_t* __restrict__ mult,
                                 int32_t* __restrict__ node, int32_t* __restrict__ label,
                                 uint8_t* __restrict__ dmask) {
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= n || gid[l] != 0) return;
  mult[l] = 1;
  node[l] = (int32_t)(nids + zpos[l]);
  label[l] = (int32_t)l;
  dmask[l] = dflag ? (dflag[l] ? 1 : 0) : 0;
}

__global__ void k_owner_cwt(int64_t n, const int32_t* __restrict__ mult, const int32_t* __restrict__ label,
                            const uint8_t* __restrict__ dmask, uint8_t* __restrict__ owner, double* __restrict__ cwt,
                            float* __restrict__ cwt32) {
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= n) return;
  owner[l] = (label[l] == (int32_t)l && !dmask[l]) ? 1 : 0;
  const double c = 1.0 / (double)mult[l];
  cwt[l] = c;
  cwt32[l] = (float)c;
}

// gs segments: kept nonzero-id segments first (id order), then Dirichlet singletons (local order)
__global__ void k_seg_fill_nz(const int64_t* __restrict__ off, const int32_t* __restrict__ idx, int64_t nids,
                              const int64_t* __restrict__ segflag, const int64_t* __restrict__ segpos,
                              const int64_t* __restrict__ lenpos, const uint8_t* __restrict__ dmask,
                              int32_t* __restrict__ seg_off, int32_t* __restrict__ seg_idx,
                              uint8_t* __restrict__ seg_dir) {
  const int64_t sg = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (sg >= nids || !segflag[sg]) return;
  const int64_t q = segpos[sg];
  const int64_t o = lenpos[sg];
  seg_off[q] = (int32_t)o;
  const int64_t b = off[sg], e = off[sg + 1];
  for (int64_t p = b; p < e; ++p) seg_idx[o + (p - b)] = idx[p];
  seg_dir[q] = dmask[idx[b]];
}

__global__ void k_zero_dir_flags(const int64_t* __restrict__ gid, const uint8_t* __restrict__ dflag, int64_t n,
                                 int64_t* __restrict__ f) {
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= n) return;
  f[l] = (gid[l] == 0 && dflag && dflag[l]) ? 1 : 0;
}

__global__ void k_seg_fill_zero(int64_t n, const int64_t* __restrict__ f, const int64_t* __restrict__ fpos,
                                int64_t q0, int64_t o0, int32_t* __restrict__ seg_off, int32_t* __restrict__ seg_idx,
                                uint8_t* __restrict__ seg_dir) {
  const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (l >= n || !f[l]) return;
  const int64_t k = fpos[l];
  seg_off[q0 + k] = (int32_t)(o0 + k);
  seg_idx[o0 + k] = (int32_t)l;
  seg_dir[q0 + k] = 1;
}

__global__ void k_set_last(int32_t* seg_off, int64_t q, int64_t v) { seg_off[q] = (int32_t)v; }

inline unsigned nblocks(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

#define MALLOC(ptr, count) SEM_CUDA_TRY(cudaMalloc((void**)&(ptr), (size_t)(count) * sizeof(*(ptr)) + 16))

int build_maps(Level& L, cudaStream_t s) {
  const int64_t n = L.nL;
  int* d_bad = nullptr;
  SEM_CUDA_TRY(cudaMallocAsync((void**)&d_bad, sizeof(int), s));
  SEM_CUDA_TRY(cudaMemsetAsync(d_bad, 0, sizeof(int), s));
  int64_t *fnz, *fz, *pnz, *pz;
  SEM_CUDA_TRY(cudaMallocAsync((void**)&fnz, n * 8, s));
  SEM_CUDA_TRY(cudaMallocAsync((void**)&fz, n * 8, s));
  SEM_CUDA_TRY(cudaMallocAsync((void**)&pnz, n * 8, s));
  SEM_CUDA_TRY(cudaMallocAsync((void**)&pz, n * 8, s));
  k_nonzero_flags<<<nblocks(n), 256, 0, s>>>(L.gid, n, fnz, fz, d_bad);
  SEM_LAUNCH_CHECK();
  int64_t n_idx = 0, n_zero = 0;
  SEM_TRY(scan_excl(fnz, pnz, n, &n_idx, s));
  SEM_TRY(scan_excl(fz, pz, n, &n_zero, s));
  int bad = 0;
  SEM_CUDA_TRY(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  SEM_CUDA_TRY(cudaStreamSynchronize(s));
  if (bad) {
    set_detail("negative global id");
    return SEM_EINVAL;
  }
  L.n_idx = n_idx;
  // compact and sort the nonzero ids
  int64_t *k1, *k2;
  int32_t *v1, *v2;
  SEM_CUDA_TRY(cudaMallocAsync((void**)&k1, (n_idx + 1) * 8, s));
  SEM_CUDA_TRY(cudaMallocAsync((void**)&k2, (n_idx + 1) * 8, s));
  SEM_CUDA_TRY(cudaMallocAsync((void**)&v1, (n_idx + 1) * 4, s));
  SEM_CUDA_TRY(cudaMallocAsync((void**)&v2, (n_idx + 1) * 4, s));
  k_compact_nz<<<nblocks(n), 256, 0, s>>>(L.gid, n, pnz, k1, v1);
  SEM_LAUNCH_CHECK();
  if (n_idx > 0) {
    unsigned long long* d_max;
    SEM_CUDA_TRY(cudaMallocAsync((void**)&d_max, 8, s));
    SEM_CUDA_TRY(cudaMemsetAsync(d_max, 0, 8, s));
    k_max_key<<<1024, 256, 0, s>>>(k1, n_idx, d_max);
    SEM_LAUNCH_CHECK();
    unsigned long long mx = 0;
    SEM_CUDA_TRY(cudaMemcpyAsync(&mx, d_max, 8, cudaMemcpyDeviceToHost, s));
    SEM_CUDA_TRY(cudaStreamSynchronize(s));
    SEM_CUDA_TRY(cudaFreeAsync(d_max, s));
    int bits = 0;
    while (bits < 64 && (mx >> bits) != 0) ++bits;
    const int64_t nblk = (n_idx + RAD_TILE - 1) / RAD_TILE;
    int64_t *hist, *hoff;
    SEM_CUDA_TRY(cudaMallocAsync((void**)&hist, 256 * nblk * 8, s));
    SEM_CUDA_TRY(cudaMallocAsync((void**)&hoff, 256 * nblk * 8, s));
    for (int shift = 0; shift < bits; shift += 8) {
      k_rad_hist<<<(unsigned)nblk, RAD_T, 0, s>>>(k1, n_idx, shift, hist, nblk);
      SEM_LAUNCH_CHECK();
      SEM_TRY(scan_excl(hist, hoff, 256 * nblk, nullptr, s));
      k_rad_scatter<<<(unsigned)nblk, RAD_T, 0, s>>>(k1, v1, n_idx, shift, hoff, nblk, k2, v2);
      SEM_LAUNCH_CHECK();
      std::swap(k1, k2);
      std::swap(v1, v2);
    }
    SEM_CUDA_TRY(cudaFreeAsync(hist, s));
    SEM_CUDA_TRY(cudaFreeAsync(hoff, s));
  }
  // segments (= nodes with a nonzero id)
  int64_t *head, *hscan;
  SEM_CUDA_TRY(cudaMallocAsync((void**)&head, (n_idx + 1) * 8, s));
  SEM_CUDA_TRY(cudaMallocAsync((void**)&hscan, (n_idx + 1) * 8, s));
  k_heads<<<nblocks(n_idx), 256, 0, s>>>(k1, n_idx, head);
  SEM_LAUNCH_CHECK();
  int64_t nids = 0;
  SEM_TRY(scan_excl(head, hscan, n_idx, &nids, s));
  L.n_ids = nids;
  L.nG = nids + n_zero;
  MALLOC(L.ids, nids + 1);
  MALLOC(L.off, nids + 1);
  MALLOC(L.idx, n_idx + 1);
  MALLOC(L.mult, n);
  MALLOC(L.node, n);
  MALLOC(L.label, n);
  MALLOC(L.dmask, n);
  MALLOC(L.owner, n);
  MALLOC(L.cwt, n);
  MALLOC(L.cwt32, n);
  k_ids_off<<<nblocks(n_idx > 0 ? n_idx : 1), 256, 0, s>>>(k1, head, hscan, n_idx, L.ids, L.off, nids);
  SEM_LAUNCH_CHECK();
  SEM_CUDA_TRY(cudaMemcpyAsync(L.idx, v1, n_idx * 4, cudaMemcpyDeviceToDevice, s));
  int64_t *segflag, *seglen, *segpos, *lenpos;
  SEM_CUDA_TRY(cudaMallocAsync((void**)&segflag, (nids + 1) * 8, s));
  SEM_CUDA_TRY(cudaMallocAsync((void**)&seglen, (nids + 1) * 8, s));
  SEM_CUDA_TRY(cudaMallocAsync((void**)&segpos, (nids + 1) * 8, s));
  SEM_CUDA_TRY(cudaMallocAsync((void**)&lenpos, (nids + 1) * 8, s));
  k_per_point_nz<<<nblocks(nids > 0 ? nids : 1), 256, 0, s>>>(L.off, L.idx, nids, L.dflag, L.mult, L.node,
                                                              L.label, L.dmask, segflag, seglen);
  SEM_LAUNCH_CHECK();
  k_per_point_zero<<<nblocks(n), 256, 0, s>>>(L.gid, n, pz, nids, L.dflag, L.mult, L.node, L.label, L.dmask);
  SEM_LAUNCH_CHECK();
  k_owner_cwt<<<nblocks(n), 256, 0, s>>>(n, L.mult, L.label, L.dmask, L.owner, L.cwt, L.cwt32);
  SEM_LAUNCH_CHECK();
  // gather-scatter segment list
  int64_t nkeep = 0, nkeep_idx = 0;
  SEM_TRY(scan_excl(segflag, segpos, nids, &nkeep, s));
  SEM_TRY(scan_excl(seglen, lenpos, nids, &nkeep_idx, s));
  int64_t *zf, *zfp;
  SEM_CUDA_TRY(cudaMallocAsync((void**)&zf, n * 8, s));
  SEM_CUDA_TRY(cudaMallocAsync((void**)&zfp, n * 8, s));
  k_zero_dir_flags<<<nblocks(n), 256, 0, s>>>(L.gid, L.dflag, n, zf);
  SEM_LAUNCH_CHECK();
  int64_t nzd = 0;
  SEM_TRY(scan_excl(zf, zfp, n, &nzd, s));
  L.n_seg = nkeep + nzd;
  L.n_seg_idx = nkeep_idx + nzd;
  if (L.n_seg_idx >= (int64_t)INT32_MAX) {
    set_detail("too many local points for 32-bit gather-scatter indices");
    return SEM_EINVAL;
  }
  MALLOC(L.seg_off, L.n_seg + 1);
  MALLOC(L.seg_idx, L.n_seg_idx + 1);
  MALLOC(L.seg_dir, L.n_seg + 1);
  if (nids > 0) {
    k_seg_fill_nz<<<nblocks(nids), 256, 0, s>>>(L.off, L.idx, nids, segflag, segpos, lenpos, L.dmask, L.seg_off,
                                                L.seg_idx, L.seg_dir);
    SEM_LAUNCH_CHECK();
  }
  k_seg_fill_zero<<<nblocks(n), 256, 0, s>>>(n, zf, zfp, nkeep, nkeep_idx, L.seg_off, L.seg_idx, L.seg_dir);
  SEM_LAUNCH_CHECK();
  k_set_last<<<1, 1, 0, s>>>(L.seg_off, L.n_seg, L.n_seg_idx);
  SEM_LAUNCH_CHECK();
  for (void* ptr : {(void*)d_bad, (void*)fnz, (void*)fz, (void*)pnz, (void*)pz, (void*)k1, (void*)k2, (void*)v1,
                    (void*)v2, (void*)head, (void*)hscan, (void*)segflag, (void*)seglen, (void*)segpos,
                    (void*)lenpos, (void*)zf, (void*)zfp})
    SEM_CUDA_TRY(cudaFreeAsync(ptr, s));
  SEM_CUDA_TRY(cudaStreamSynchronize(s));
  return SEM_OK;
}

}  // namespace sem
