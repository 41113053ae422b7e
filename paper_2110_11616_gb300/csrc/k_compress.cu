// The compression pieces of Sec. V-D on a CGA, and the G-Arrays form of its
// X pointer that Sec. V sets against the CGA's:
//   k_km_init / k_bbox / k_km_seed   the bounding box of the stored voxels
//                     and the eight centres at its corners
//   k_km_assign       one Lloyd pass over a tile: every voxel's nearest
//                     centre (ties to the lower cluster), the count of changed
//                     labels and the per-cluster coordinate sums
//   k_km_update       the centres from the sums (round half up to 1/256
//                     voxel), convergence when a pass changed no label
//   k_motion          mv = ref - pred for clusters non-empty in both frames
//   k_reconstruct     every voxel moved by its cluster's vector rounded half
//                     up to whole voxels
//   k_residual        the residual frame: each reconstructed point's
//                     attributes minus those of its corresponding reference
//                     point
//   k_garrays_x       the dense X pointer, one cell per x value of the axis
//   k_lookup          the Sec. V-A point lookup of integer voxels, through
//                     X_index (CGA) or through the dense X pointer (G-Arrays)
// Centres are integers in 1/256 voxel and every sum is an exact integer, so
// the results do not depend on the order in which voxels are visited.
#include <algorithm>

#include "k_common.cuh"

namespace libcga {

namespace {

// Per-block partial sums fit 32 bits: a tile of kTile voxels of coordinates
// below 2^16.
static_assert((uint64_t)kTile * 65535u < (1ull << 32), "tile sums");

__global__ void k_km_init(KmState* st, uint32_t max_iter) {
  const uint32_t t = threadIdx.x;
  if (t < 3) {
    st->box[t] = 0xffffffffu;
    st->box[3 + t] = 0;
  }
  if (t < kKmClusters * 4) (&st->sum[0][0])[t] = 0;
  if (t == 0) {
    st->changed = 0;
    st->pass = 0;
    st->done = 0;
    st->max_iter = max_iter;
  }
}

// Least and greatest y over Y_index and z over Z_index (x: the ends of the
// sorted X_index).
__global__ void k_bbox(Levels a, KmState* st) {
  const uint32_t u = (uint32_t)a.hdr->cnt[0], g = (uint32_t)a.hdr->cnt[1];
  const uint32_t stride = gridDim.x * blockDim.x;
  uint32_t lo[2] = {0xffffffffu, 0xffffffffu}, hi[2] = {0, 0};
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < g; i += stride) {
    const uint32_t y = __ldg(a.idx1 + i);
    lo[0] = min(lo[0], y);
    hi[0] = max(hi[0], y);
  }
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < u; i += stride) {
    const uint32_t z = __ldg(a.idx0 + i);
    lo[1] = min(lo[1], z);
    hi[1] = max(hi[1], z);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    lo[k] = __reduce_min_sync(0xffffffffu, lo[k]);
    hi[k] = __reduce_max_sync(0xffffffffu, hi[k]);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&st->box[1], lo[0]);
    atomicMin(&st->box[2], lo[1]);
    atomicMax(&st->box[4], hi[0]);
    atomicMax(&st->box[5], hi[1]);
  }
}

// Corner c of the box: the greatest coordinate of axis a where bit a of c is
// set, else the least, in 1/256 voxel.
__global__ void k_km_seed(Levels a, KmState* st, long long* centres, unsigned long long* counts,
                          uint32_t* iters) {
  const uint32_t t = threadIdx.x;
  const uint32_t u = (uint32_t)a.hdr->cnt[0], h = (uint32_t)a.hdr->cnt[2];
  if (t < kKmClusters * 3) {
    const uint32_t c = t / 3, ax = t % 3;
    long long v = 0;
    if (u > 0) {
      const uint32_t lo = ax == 0 ? (uint32_t)__ldg(a.idx2) : st->box[ax];
      const uint32_t hi = ax == 0 ? (uint32_t)__ldg(a.idx2 + h - 1) : st->box[3 + ax];
      v = 256ll * (long long)(((c >> ax) & 1u) ? hi : lo);
    }
    centres[t] = v;
  }
  if (t < kKmClusters) counts[t] = 0;
  if (t == 0) {
    *iters = 0;
    if (u == 0) st->done = 1;
  }
}

__global__ void __launch_bounds__(kThreads) k_km_assign(Levels a, KmState* st,
                                                        const long long* __restrict__ centres,
                                                        uint8_t* __restrict__ labels) {
  __shared__ Window s_win;
  __shared__ uint16_t s_col[kTile], s_slab[kTile];
  __shared__ uint32_t s_warp[kWarps];
  __shared__ int s_c[kKmClusters * 3];
  __shared__ uint32_t s_sum[kKmClusters][4];
  __shared__ uint32_t s_changed;
  if (st->done) return;
  const uint32_t u = (uint32_t)a.hdr->cnt[0];
  const uint32_t start = blockIdx.x * kTile;
  if (start >= u) return;
  const uint32_t cnt = min((uint32_t)kTile, u - start);
  const uint32_t tid = threadIdx.x, lane = tid & 31;
  const bool later_pass = st->pass > 0;
  if (tid < kKmClusters * 3) s_c[tid] = (int)centres[tid];  // below 2^24
  if (tid < kKmClusters * 4) (&s_sum[0][0])[tid] = 0;
  if (tid == 0) s_changed = 0;
  if (tid < 32) {
    const Window wv =
        warp_window_of(a, (uint32_t)a.hdr->cnt[1], (uint32_t)a.hdr->cnt[2], start, start + cnt - 1);
    if (tid == 0) s_win = wv;
  }
  __syncthreads();
  const Window w = s_win;
  expand_window(a, w, start, cnt, s_col, s_slab, s_warp);
  uint32_t changed = 0;
  for (uint32_t base = 0; base < cnt; base += kThreads) {
    const uint32_t e = base + tid;
    const bool valid = e < cnt;
    uint32_t x = 0, y = 0, z = 0, best = 0;
    if (valid) {
      const uint32_t cr = s_col[e];
      x = __ldg(a.idx2 + w.x0 + s_slab[cr]);
      y = __ldg(a.idx1 + w.c0 + cr);
      z = __ldg(a.idx0 + start + e);
      const int vx = (int)(x << 8), vy = (int)(y << 8), vz = (int)(z << 8);
      unsigned long long bd = ~0ull;
#pragma unroll
      for (uint32_t c = 0; c < kKmClusters; ++c) {
        const int dx = vx - s_c[3 * c], dy = vy - s_c[3 * c + 1], dz = vz - s_c[3 * c + 2];
        const unsigned long long d = (unsigned long long)((long long)dx * dx) +
                                     (unsigned long long)((long long)dy * dy) +
                                     (unsigned long long)((long long)dz * dz);
        if (d < bd) {
          bd = d;
          best = c;
        }
      }
      if (later_pass && labels[start + e] != best) ++changed;
      labels[start + e] = (uint8_t)best;
    }
    // one shared-memory update per distinct label of the warp
    uint32_t todo = __ballot_sync(0xffffffffu, valid);
    while (todo) {
      const uint32_t leader = __ffs(todo) - 1;
      const uint32_t L = __shfl_sync(0xffffffffu, best, leader);
      const bool mine = valid && best == L;
      const uint32_t mask = __ballot_sync(0xffffffffu, mine);
      todo &= ~mask;
      const uint32_t sx = __reduce_add_sync(0xffffffffu, mine ? x : 0u);
      const uint32_t sy = __reduce_add_sync(0xffffffffu, mine ? y : 0u);
      const uint32_t sz = __reduce_add_sync(0xffffffffu, mine ? z : 0u);
      if (lane == leader) {
        atomicAdd(&s_sum[L][0], sx);
        atomicAdd(&s_sum[L][1], sy);
        atomicAdd(&s_sum[L][2], sz);
        atomicAdd(&s_sum[L][3], (uint32_t)__popc(mask));
      }
    }
  }
  changed = __reduce_add_sync(0xffffffffu, changed);
  if (lane == 0 && changed) atomicAdd(&s_changed, changed);
  __syncthreads();
  if (tid < kKmClusters * 4) {
    const uint32_t v = (&s_sum[0][0])[tid];
    if (v) atomicAdd(&(&st->sum[0][0])[tid], (unsigned long long)v);
  }
  if (tid == 0 && s_changed) atomicAdd(&st->changed, (unsigned long long)s_changed);
}

__global__ void k_km_update(KmState* st, long long* centres, unsigned long long* counts,
                            uint32_t* iters) {
  if (threadIdx.x != 0 || st->done) return;
  const uint32_t pass = ++st->pass;
  const bool converged = pass > 1 && st->changed == 0;
  for (uint32_t c = 0; c < kKmClusters; ++c) {
    const unsigned long long n = st->sum[c][3];
    counts[c] = n;
    if (!converged && n > 0) {
      for (int ax = 0; ax < 3; ++ax) {
        centres[3 * c + ax] = (long long)((256ull * st->sum[c][ax] + n / 2) / n);
      }
    }
  }
  *iters = pass;
  if (converged || pass >= st->max_iter) st->done = 1;
  for (uint32_t i = 0; i < kKmClusters * 4; ++i) (&st->sum[0][0])[i] = 0;
  st->changed = 0;
}

__global__ void k_motion(const long long* ref_c, const unsigned long long* ref_n,
                         const long long* pred_c, const unsigned long long* pred_n,
                         long long* mv) {
  const uint32_t t = threadIdx.x;
  if (t < kKmClusters * 3) {
    const uint32_t c = t / 3;
    mv[t] = (ref_n[c] > 0 && pred_n[c] > 0) ? ref_c[t] - pred_c[t] : 0;
  }
}

__global__ void __launch_bounds__(kThreads) k_reconstruct(Levels a, const uint8_t* __restrict__ labels,
                                                          const long long* __restrict__ mv,
                                                          int* __restrict__ out) {
  __shared__ Window s_win;
  __shared__ uint16_t s_col[kTile], s_slab[kTile];
  __shared__ uint32_t s_warp[kWarps];
  __shared__ int s_step[kKmClusters * 3];
  const uint32_t u = (uint32_t)a.hdr->cnt[0];
  const uint32_t start = blockIdx.x * kTile;
  if (start >= u) return;
  const uint32_t cnt = min((uint32_t)kTile, u - start);
  const uint32_t tid = threadIdx.x;
  // floor((mv + 128) / 256): the arithmetic shift rounds toward -infinity
  if (tid < kKmClusters * 3) s_step[tid] = (int)((mv[tid] + 128) >> 8);
  if (tid < 32) {
    const Window wv =
        warp_window_of(a, (uint32_t)a.hdr->cnt[1], (uint32_t)a.hdr->cnt[2], start, start + cnt - 1);
    if (tid == 0) s_win = wv;
  }
  __syncthreads();
  const Window w = s_win;
  expand_window(a, w, start, cnt, s_col, s_slab, s_warp);
  for (uint32_t e = tid; e < cnt; e += kThreads) {
    const uint32_t cr = s_col[e];
    const uint32_t L = min((uint32_t)__ldg(labels + start + e), kKmClusters - 1);
    int* o = out + 3 * (size_t)(start + e);
    o[0] = (int)__ldg(a.idx2 + w.x0 + s_slab[cr]) + s_step[3 * L];
    o[1] = (int)__ldg(a.idx1 + w.c0 + cr) + s_step[3 * L + 1];
    o[2] = (int)__ldg(a.idx0 + start + e) + s_step[3 * L + 2];
  }
}

// res[i*C + c] = pred[i*C + c] - ref[idx[i]*C + c], or pred[i*C + c] when
// idx[i] >= u_ref (no corresponding point).  One thread per output entry.
__global__ void k_residual(const uint8_t* __restrict__ pred, uint64_t u_pred,
                           const uint8_t* __restrict__ ref, uint64_t u_ref,
                           const uint32_t* __restrict__ idx, uint32_t C, int16_t* __restrict__ res) {
  const uint64_t total = u_pred * C;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < total; e += stride) {
    const uint64_t i = e / C;
    const uint32_t c = (uint32_t)(e - i * C);
    const uint32_t j = __ldg(idx + i);
    const int p = __ldg(pred + e);
    res[e] = (int16_t)(j < u_ref ? p - (int)__ldg(ref + (uint64_t)j * C + c) : p);
  }
}

__global__ void k_garrays_x(Levels a, uint32_t* xptr) {
  const uint32_t h = (uint32_t)a.hdr->cnt[2];
  const uint32_t n = 1u << a.bits;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += stride) {
    xptr[v] = __ldg(a.ptr2 + lower_bound_u16(a.idx2, 0, h, v));
  }
}

// xptr == nullptr: the CGA lookup (x searched in X_index); else the G-Arrays
// lookup (the x value indexes the dense pointer).
__global__ void k_lookup(Levels a, const uint32_t* __restrict__ xptr, const int* __restrict__ qv,
                         uint32_t m, uint32_t* __restrict__ idx) {
  const uint32_t h = (uint32_t)a.hdr->cnt[2];
  const int side = 1 << a.bits;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride) {
    const int x = __ldg(qv + 3 * (size_t)j), y = __ldg(qv + 3 * (size_t)j + 1),
              z = __ldg(qv + 3 * (size_t)j + 2);
    uint32_t r = 0xffffffffu;
    if (x >= 0 && y >= 0 && z >= 0 && x < side && y < side && z < side) {
      if (xptr == nullptr) {
        bool found = false;
        const uint32_t b = a.bits;
        const unsigned long long key = ((unsigned long long)x << (2 * b)) |
                                       ((unsigned long long)y << b) | (unsigned long long)z;
        const uint32_t p = rank_of_found(a, h, key, found);
        if (found) r = p;
      } else {
        const uint32_t ys = __ldg(xptr + x), ye = __ldg(xptr + x + 1);
        const uint32_t c = lower_bound_u16(a.idx1, ys, ye, (uint32_t)y);
        if (c < ye && __ldg(a.idx1 + c) == (uint32_t)y) {
          const uint32_t zs = __ldg(a.ptr1 + c), ze = __ldg(a.ptr1 + c + 1);
          const uint32_t p = lower_bound_u16(a.idx0, zs, ze, (uint32_t)z);
          if (p < ze && __ldg(a.idx0 + p) == (uint32_t)z) r = p;
        }
      }
    }
    idx[j] = r;
  }
}

unsigned grid_for(uint64_t work) {
  return (unsigned)std::min<uint64_t>((std::max<uint64_t>(work, 1) + 255) / 256,
                                      (uint64_t)device_sm_count() * 8);
}

}  // namespace

cudaError_t run_kmeans(const Levels& a, uint32_t max_iter, KmState* st, uint8_t* labels,
                       long long* centres, unsigned long long* counts, uint32_t* iters,
                       cudaStream_t stream) {
  k_km_init<<<1, 32, 0, stream>>>(st, max_iter);
  k_bbox<<<grid_for(a.cap), 256, 0, stream>>>(a, st);
  k_km_seed<<<1, 32, 0, stream>>>(a, st, centres, counts, iters);
  const unsigned tiles = (unsigned)std::max<uint64_t>((a.cap + kTile - 1) / kTile, 1);
  for (uint32_t t = 0; t < max_iter; ++t) {
    k_km_assign<<<tiles, kThreads, 0, stream>>>(a, st, centres, labels);
    k_km_update<<<1, 32, 0, stream>>>(st, centres, counts, iters);
  }
  count_launch(3 + 2 * (uint64_t)max_iter);
  return cudaGetLastError();
}

cudaError_t run_motion(const long long* ref_c, const unsigned long long* ref_n,
                       const long long* pred_c, const unsigned long long* pred_n, long long* mv,
                       cudaStream_t stream) {
  k_motion<<<1, 32, 0, stream>>>(ref_c, ref_n, pred_c, pred_n, mv);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t run_reconstruct(const Levels& a, const uint8_t* labels, const long long* mv, int* out,
                            cudaStream_t stream) {
  const uint64_t tiles = (a.cap + kTile - 1) / kTile;
  if (tiles == 0) return cudaSuccess;
  k_reconstruct<<<(unsigned)tiles, kThreads, 0, stream>>>(a, labels, mv, out);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t run_residual(const uint8_t* pred, uint64_t u_pred, const uint8_t* ref, uint64_t u_ref,
                         const uint32_t* idx, uint32_t channels, int16_t* res,
                         cudaStream_t stream) {
  if (u_pred == 0) return cudaSuccess;
  k_residual<<<grid_for(u_pred * channels), 256, 0, stream>>>(pred, u_pred, ref, u_ref, idx,
                                                              channels, res);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t run_garrays_x(const Levels& a, uint32_t* xptr, cudaStream_t stream) {
  k_garrays_x<<<grid_for((1ull << a.bits) + 1), 256, 0, stream>>>(a, xptr);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t run_lookup(const Levels& a, const uint32_t* xptr, const int* qv, uint32_t m,
                       uint32_t* idx, cudaStream_t stream) {
  if (m == 0) return cudaSuccess;
  k_lookup<<<grid_for(m), 256, 0, stream>>>(a, xptr, qv, m, idx);
  count_launch(1);
  return cudaGetLastError();
}

}  // namespace libcga
