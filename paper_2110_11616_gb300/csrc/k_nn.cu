// Exact nearest-neighbour search on a CGA (Eq. 7-8, Sec. III-C).
//
// The search is the paper's window search, with the bound shrinking as
// closer voxels are found.  It visits x slabs outward from the query's x, and
// in each slab the columns outward from the query's y.  A slab is skipped once
// dx^2 exceeds the best squared distance found so far, and a column once
// dx^2 + dy^2 does.  Each visited column contributes its two z neighbours of
// the query (binary search).  Every voxel that could lie at or below the final
// distance is examined, and ties go to the smaller key, so the result is
// exactly Eq. 8's set reduced by the smaller-key rule.
//
// GPU mapping: one warp per query.  In each round the 32 lanes take 16 slabs
// on each side of the query (lane parity picks the side).  Phase A: every lane
// finds its slab's nearest column and that column's nearest voxel.  A warp
// minimum then sets the bound.  Phase B: each lane scans its slab's remaining
// columns under that bound, and a second warp minimum follows.  Queries are
// visited in Morton order of their voxel (a 4-pass radix sort of
// (morton << 32 | index) keys), so neighbouring warps read neighbouring slabs.
#include <algorithm>
#include <new>

#include "k_common.cuh"

namespace libcga {

namespace {

size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

__device__ __forceinline__ int find_nn_seg(const NnSeg* __restrict__ segs, int S, uint32_t t) {
  int lo = 0, hi = S - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (segs[mid].tile_base <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ long long quantize_query(float v, float scale, float off) {
  float f = floorf(__fmaf_rn(v, scale, off));
  f = fminf(fmaxf(f, -1073741824.0f), 1073741824.0f);
  return (long long)f;
}

__device__ __forceinline__ unsigned long long absdiff(long long a, long long b) {
  return (unsigned long long)(a > b ? a - b : b - a);
}

__device__ __forceinline__ uint32_t spread3(uint32_t v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

// Sort keys (morton30 << 32 | query index) and per-segment digit histograms
// of the four passes over bits 32..63.  A block covers 256 slots of one tile.
__global__ void __launch_bounds__(256) k_nn_keys(const NnSeg* __restrict__ segs, int S,
                                                 unsigned long long* __restrict__ keys,
                                                 uint32_t* __restrict__ hist) {
  __shared__ uint32_t s_hist[4][kRadix];
  for (int i = threadIdx.x; i < 4 * kRadix; i += blockDim.x) (&s_hist[0][0])[i] = 0;
  __syncthreads();
  const uint32_t slot = blockIdx.x * 256u + threadIdx.x;
  const uint32_t tile = blockIdx.x / (kTile / 256);
  const int s = find_nn_seg(segs, S, tile);
  const NnSeg& sg = segs[s];
  const uint32_t local = slot - sg.tile_base * (uint32_t)kTile;
  if (local < sg.m) {
    const float* p = sg.q + 3 * (size_t)local;
    const float px = p[0], py = p[1], pz = p[2];
    uint32_t mort = 0x3fffffffu;
    if (isfinite(px) && isfinite(py) && isfinite(pz)) {
      const uint32_t bits = sg.a.bits;
      const float top = (float)((1u << bits) - 1u);
      const float v[3] = {px, py, pz};
      uint32_t c[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        float f = floorf(__fmaf_rn(v[a], sg.scale, sg.off[a]));
        f = fminf(fmaxf(f, 0.0f), top);
        const uint32_t u = (uint32_t)f;
        c[a] = bits >= 10 ? (u >> (bits - 10)) : (u << (10 - bits));
      }
      mort = (spread3(c[0]) << 2) | (spread3(c[1]) << 1) | spread3(c[2]);
    }
    keys[slot] = ((unsigned long long)mort << 32) | local;
#pragma unroll
    for (int k = 0; k < 4; ++k) atomicAdd(&s_hist[k][(mort >> (8 * k)) & (kRadix - 1)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 4 * kRadix; i += blockDim.x) {
    const uint32_t v = (&s_hist[0][0])[i];
    if (v) atomicAdd(hist + (size_t)s * kMaxPasses * kRadix + i, v);
  }
}

struct Best {
  unsigned long long d2, key;
  uint32_t idx;
  __device__ __forceinline__ void offer(unsigned long long d, unsigned long long k, uint32_t i) {
    if (d < d2 || (d == d2 && k < key)) {
      d2 = d;
      key = k;
      idx = i;
    }
  }
  __device__ __forceinline__ void warp_min() {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long od = __shfl_xor_sync(0xffffffffu, d2, o);
      const unsigned long long ok = __shfl_xor_sync(0xffffffffu, key, o);
      const uint32_t oi = __shfl_xor_sync(0xffffffffu, idx, o);
      offer(od, ok, oi);
    }
  }
};

// The two z neighbours of the query in column c.
__device__ __forceinline__ void visit_column(const Levels& a, uint32_t c, unsigned long long kxy,
                                             unsigned long long dxy, long long qz, uint32_t cqz,
                                             Best& b) {
  const uint32_t zs = __ldg(a.ptr1 + c), ze = __ldg(a.ptr1 + c + 1);
  const uint32_t zr = lower_bound_u16(a.idx0, zs, ze, cqz);
  if (zr < ze) {
    const uint32_t z = __ldg(a.idx0 + zr);
    const unsigned long long dz = absdiff(z, qz);
    b.offer(dxy + dz * dz, kxy | z, zr);
  }
  if (zr > zs) {
    const uint32_t z = __ldg(a.idx0 + zr - 1);
    const unsigned long long dz = absdiff(z, qz);
    b.offer(dxy + dz * dz, kxy | z, zr - 1);
  }
}

// Window search over the fine CGA alone (one warp, 16 slabs per side per round).
__device__ __forceinline__ void search_fine(const Levels& a, const uint32_t* xdir, uint32_t h,
                                            long long qx, long long qy, long long qz,
                                            uint32_t cqx, uint32_t cqy, uint32_t cqz,
                                            uint32_t lane, Best& best) {
  const uint32_t b = a.bits;
  const uint32_t xr0 = xdir != nullptr ? __ldg(xdir + cqx) : lower_bound_u16(a.idx2, 0, h, cqx);
  const bool right = (lane & 1u) == 0u;
  for (uint32_t r = 0;; ++r) {
    const long long k = (long long)r * 16 + (lane >> 1);
    const long long slab = right ? (long long)xr0 + k : (long long)xr0 - 1 - k;
    const bool valid = slab >= 0 && slab < (long long)h;
    unsigned long long dx2 = ~0ull;
    uint32_t x = 0;
    if (valid) {
      x = __ldg(a.idx2 + slab);
      const unsigned long long dx = absdiff(x, qx);
      dx2 = dx * dx;
    }
    const bool active = valid && dx2 <= best.d2;
    if (!__any_sync(0xffffffffu, active)) break;
    uint32_t ys = 0, ye = 0, yr0 = 0;
    const unsigned long long kx = (unsigned long long)x << (2 * b);
    if (active) {
      ys = __ldg(a.ptr2 + slab);
      ye = __ldg(a.ptr2 + slab + 1);
      yr0 = lower_bound_u16(a.idx1, ys, ye, cqy);
      if (yr0 < ye) {
        const uint32_t y = __ldg(a.idx1 + yr0);
        const unsigned long long dy = absdiff(y, qy);
        const unsigned long long dxy = dx2 + dy * dy;
        if (dxy <= best.d2) visit_column(a, yr0, kx | ((unsigned long long)y << b), dxy, qz, cqz, best);
      }
      if (yr0 > ys) {
        const uint32_t y = __ldg(a.idx1 + yr0 - 1);
        const unsigned long long dy = absdiff(y, qy);
        const unsigned long long dxy = dx2 + dy * dy;
        if (dxy <= best.d2) visit_column(a, yr0 - 1, kx | ((unsigned long long)y << b), dxy, qz, cqz, best);
      }
    }
    best.warp_min();
    if (active) {
      long long R2 = (long long)yr0 + 1, L2 = (long long)yr0 - 2;
      while (true) {
        const bool hR = R2 < (long long)ye, hL = L2 >= (long long)ys;
        if (!hR && !hL) break;
        const unsigned long long eR = hR ? absdiff(__ldg(a.idx1 + R2), qy) : ~0ull;
        const unsigned long long eL = hL ? absdiff(__ldg(a.idx1 + L2), qy) : ~0ull;
        const bool gR = hR && (!hL || eR <= eL);
        const unsigned long long dy = gR ? eR : eL;
        const unsigned long long dxy = dx2 + dy * dy;
        if (dxy > best.d2) break;
        const uint32_t c = (uint32_t)(gR ? R2 : L2);
        if (gR) ++R2; else --L2;
        const uint32_t y = __ldg(a.idx1 + c);
        visit_column(a, c, kx | ((unsigned long long)y << b), dxy, qz, cqz, best);
      }
    }
    best.warp_min();
  }
}

// Distance from q to the voxel interval [lo, lo + s - 1] (0 inside).
__device__ __forceinline__ unsigned long long interval_dist(long long q, uint32_t lo, uint32_t s) {
  const long long l = lo, hi = (long long)lo + s - 1;
  return q < l ? (unsigned long long)(l - q) : (q > hi ? (unsigned long long)(q - hi) : 0ull);
}

// Every fine column inside the footprint of one coarse column: fine slabs
// [fx0, fx1) (the fine slabs of the coarse slab), y in [ylo, ylo + s).
__device__ __forceinline__ void refine_footprint(const Levels& a, uint32_t fx0, uint32_t fx1,
                                                 uint32_t ylo, uint32_t s, long long qx,
                                                 long long qy, long long qz, uint32_t cqz,
                                                 Best& best) {
  const uint32_t b = a.bits;
  for (uint32_t xi = fx0; xi < fx1; ++xi) {
    const uint32_t x = __ldg(a.idx2 + xi);
    const unsigned long long dx = absdiff(x, qx);
    const unsigned long long dx2 = dx * dx;
    if (dx2 > best.d2) continue;
    const uint32_t ys = __ldg(a.ptr2 + xi), ye = __ldg(a.ptr2 + xi + 1);
    const unsigned long long kx = (unsigned long long)x << (2 * b);
    for (uint32_t c = lower_bound_u16(a.idx1, ys, ye, ylo); c < ye; ++c) {
      const uint32_t y = __ldg(a.idx1 + c);
      if (y >= ylo + s) break;
      const unsigned long long dy = absdiff(y, qy);
      const unsigned long long dxy = dx2 + dy * dy;
      if (dxy > best.d2) continue;
      visit_column(a, c, kx | ((unsigned long long)y << b), dxy, qz, cqz, best);
    }
  }
}

// A coarse column (cx, cy): its nearest occupied coarse cell along z bounds
// every point below it; refine the fine footprint only if that bound can beat
// the best distance so far.
__device__ __forceinline__ void visit_coarse_column(const NnSeg& sg, uint32_t cc, uint32_t cy,
                                                    unsigned long long dxl2,
                                                    unsigned long long dyl2, uint32_t fx0,
                                                    uint32_t fx1, long long qx, long long qy,
                                                    long long qz, uint32_t cqz, Best& best) {
  if (dxl2 + dyl2 > best.d2) return;
  const Levels& c = sg.c;
  const uint32_t L = sg.shift, s = 1u << L;
  const uint32_t zs = __ldg(c.ptr1 + cc), ze = __ldg(c.ptr1 + cc + 1);
  const uint32_t zr = lower_bound_u16(c.idx0, zs, ze, cqz >> L);
  unsigned long long dzl = ~0ull;
  if (zr < ze) dzl = min(dzl, interval_dist(qz, (uint32_t)__ldg(c.idx0 + zr) << L, s));
  if (zr > zs) dzl = min(dzl, interval_dist(qz, (uint32_t)__ldg(c.idx0 + zr - 1) << L, s));
  if (dxl2 + dyl2 + dzl * dzl > best.d2) return;
  refine_footprint(sg.a, fx0, fx1, cy << L, s, qx, qy, qz, cqz, best);
}

// Two-level window search: the same round structure over the coarse CGA (the
// occupied cells of 2^shift voxels), with box lower bounds deciding which
// cells' fine footprints are searched.  A point lies in an occupied cell whose
// bound never exceeds the point's distance, so pruning by "bound > best"
// never drops a point at or below the final distance.
__device__ __forceinline__ void search_two_level(const NnSeg& sg, long long qx, long long qy,
                                                 long long qz, uint32_t cqx, uint32_t cqy,
                                                 uint32_t cqz, uint32_t lane, Best& best) {
  const Levels& c = sg.c;
  const uint32_t L = sg.shift, s = 1u << L;
  const uint32_t hc = (uint32_t)c.hdr->cnt[2];
  const uint32_t xr0 = sg.cxdir != nullptr ? __ldg(sg.cxdir + (cqx >> L))
                                            : lower_bound_u16(c.idx2, 0, hc, cqx >> L);
  const uint32_t cqy_c = cqy >> L;
  const bool right = (lane & 1u) == 0u;
  for (uint32_t r = 0;; ++r) {
    const long long k = (long long)r * 16 + (lane >> 1);
    const long long slab = right ? (long long)xr0 + k : (long long)xr0 - 1 - k;
    const bool valid = slab >= 0 && slab < (long long)hc;
    unsigned long long dxl2 = ~0ull;
    if (valid) {
      const unsigned long long dxl = interval_dist(qx, (uint32_t)__ldg(c.idx2 + slab) << L, s);
      dxl2 = dxl * dxl;
    }
    const bool active = valid && dxl2 <= best.d2;
    if (!__any_sync(0xffffffffu, active)) break;
    uint32_t ys = 0, ye = 0, yr0 = 0, fx0 = 0, fx1 = 0;
    if (active) {
      ys = __ldg(c.ptr2 + slab);
      ye = __ldg(c.ptr2 + slab + 1);
      yr0 = lower_bound_u16(c.idx1, ys, ye, cqy_c);
      fx0 = __ldg(sg.xs + slab);
      fx1 = __ldg(sg.xs + slab + 1);
      if (yr0 < ye) {
        const uint32_t cy = __ldg(c.idx1 + yr0);
        const unsigned long long dyl = interval_dist(qy, cy << L, s);
        visit_coarse_column(sg, yr0, cy, dxl2, dyl * dyl, fx0, fx1, qx, qy, qz, cqz, best);
      }
      if (yr0 > ys) {
        const uint32_t cy = __ldg(c.idx1 + yr0 - 1);
        const unsigned long long dyl = interval_dist(qy, cy << L, s);
        visit_coarse_column(sg, yr0 - 1, cy, dxl2, dyl * dyl, fx0, fx1, qx, qy, qz, cqz, best);
      }
    }
    best.warp_min();
    if (active) {
      long long R2 = (long long)yr0 + 1, L2 = (long long)yr0 - 2;
      while (true) {
        const bool hR = R2 < (long long)ye, hL = L2 >= (long long)ys;
        if (!hR && !hL) break;
        const unsigned long long eR =
            hR ? interval_dist(qy, (uint32_t)__ldg(c.idx1 + R2) << L, s) : ~0ull;
        const unsigned long long eL =
            hL ? interval_dist(qy, (uint32_t)__ldg(c.idx1 + L2) << L, s) : ~0ull;
        const bool gR = hR && (!hL || eR <= eL);
        const unsigned long long dyl = gR ? eR : eL;
        if (dxl2 + dyl * dyl > best.d2) break;
        const uint32_t cc = (uint32_t)(gR ? R2 : L2);
        if (gR) ++R2; else --L2;
        visit_coarse_column(sg, cc, __ldg(c.idx1 + cc), dxl2, dyl * dyl, fx0, fx1, qx, qy, qz,
                            cqz, best);
      }
    }
    best.warp_min();
  }
}

// COARSE: compiled with the two-level search (used when a segment carries a
// coarse companion); the fine-only instantiation keeps fewer registers.
template <bool COARSE>
__global__ void __launch_bounds__(256) k_nn_warp(const NnSeg* __restrict__ segs, int S,
                                                 NnSeg inline_seg, uint32_t total_slots,
                                                 const unsigned long long* __restrict__ order,
                                                 const unsigned int* __restrict__ order_err) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const bool sorted = order != nullptr && (order_err == nullptr || *order_err == 0u);
  for (uint32_t slot = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; slot < total_slots;
       slot += nwarps) {
    const uint32_t tile = slot / (uint32_t)kTile;
    const NnSeg& sg = segs != nullptr ? segs[find_nn_seg(segs, S, tile)] : inline_seg;
    const uint32_t local = slot - sg.tile_base * (uint32_t)kTile;
    if (local >= sg.m) continue;
    const uint32_t j = sorted ? (uint32_t)order[slot] : local;
    if (j >= sg.m) continue;  // a caller-given order that is not a permutation
    const Levels& a = sg.a;
    const float* p = sg.q + 3 * (size_t)j;
    const float px = p[0], py = p[1], pz = p[2];
    const uint32_t u = (uint32_t)a.hdr->cnt[0], h = (uint32_t)a.hdr->cnt[2];
    if (!(isfinite(px) && isfinite(py) && isfinite(pz)) || u == 0) {
      if (lane == 0) {
        sg.idx[j] = 0xffffffffu;
        sg.d2[j] = ~0ull;
      }
      continue;
    }
    const uint32_t b = a.bits;
    const long long top = (1ll << b) - 1;
    const long long qx = quantize_query(px, sg.scale, sg.off[0]);
    const long long qy = quantize_query(py, sg.scale, sg.off[1]);
    const long long qz = quantize_query(pz, sg.scale, sg.off[2]);
    const uint32_t cqx = (uint32_t)min(max(qx, 0ll), top);
    const uint32_t cqy = (uint32_t)min(max(qy, 0ll), top);
    const uint32_t cqz = (uint32_t)min(max(qz, 0ll), top);
    Best best{~0ull, ~0ull, 0xffffffffu};
    if (COARSE && sg.has_coarse) {
      search_two_level(sg, qx, qy, qz, cqx, cqy, cqz, lane, best);
    } else {
      search_fine(a, sg.xdir, h, qx, qy, qz, cqx, cqy, cqz, lane, best);
    }
    if (lane == 0) {
      sg.idx[j] = best.idx;
      sg.d2[j] = best.d2;
    }
  }
}

}  // namespace

size_t nn_scratch_bytes(uint32_t total_tiles, int S) {
  return align_up(sizeof(Header)) + align_up((size_t)S * sizeof(NnSeg)) +
         sort_scratch_bytes((uint64_t)total_tiles * kTile, total_tiles, S, true);
}

NnTables nn_tables(void* scratch, uint32_t total_tiles, int S) {
  char* p = static_cast<char*>(scratch);
  NnTables t{};
  t.err = reinterpret_cast<Header*>(p);
  p += align_up(sizeof(Header));
  t.segs = reinterpret_cast<NnSeg*>(p);
  p += align_up((size_t)S * sizeof(NnSeg));
  t.sort = sort_scratch_carve(p, (uint64_t)total_tiles * kTile, total_tiles, S, true);
  return t;
}

cudaError_t nn_upload(const NnSeg* h_segs, int S, const NnTables& t, cudaStream_t stream) {
  SortSeg* ss = new (std::nothrow) SortSeg[S]();
  if (ss == nullptr) return cudaErrorMemoryAllocation;
  for (int s = 0; s < S; ++s) {
    ss[s].n_host = h_segs[s].m;
    ss[s].passes = 4;
    ss[s].bit0 = 32;
    ss[s].key_base = (uint64_t)h_segs[s].tile_base * kTile;
    ss[s].tile_base = h_segs[s].tile_base;
    ss[s].num_tiles = h_segs[s].num_tiles;
    ss[s].out.hdr = t.err;
  }
  cudaError_t e = cudaMemcpyAsync(t.segs, h_segs, sizeof(NnSeg) * S, cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) {
    e = cudaMemcpyAsync(t.sort.segs, ss, sizeof(SortSeg) * S, cudaMemcpyHostToDevice, stream);
  }
  delete[] ss;
  return e;
}

cudaError_t nn_upload_one(const NnSeg& h_seg, const NnTables& t, cudaStream_t stream) {
  SortSeg ss{};
  ss.n_host = h_seg.m;
  ss.passes = 4;
  ss.bit0 = 32;
  ss.key_base = (uint64_t)h_seg.tile_base * kTile;
  ss.tile_base = h_seg.tile_base;
  ss.num_tiles = h_seg.num_tiles;
  ss.out.hdr = t.err;
  cudaError_t e = cudaMemcpyAsync(t.segs, &h_seg, sizeof(NnSeg), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) {
    e = cudaMemcpyAsync(t.sort.segs, &ss, sizeof(SortSeg), cudaMemcpyHostToDevice, stream);
  }
  return e;
}

static void launch_search(const NnSeg* d_segs, int S, const NnSeg& inline_seg,
                          uint32_t total_tiles, const unsigned long long* order,
                          const unsigned int* order_err, bool coarse, cudaStream_t stream) {
  const uint32_t total_slots = total_tiles * (uint32_t)kTile;
  const uint32_t blocks =
      std::min<uint32_t>((total_slots + 7) / 8, (uint32_t)device_sm_count() * 8);
  if (coarse) {
    k_nn_warp<true><<<blocks, 256, 0, stream>>>(d_segs, S, inline_seg, total_slots, order,
                                                order_err);
  } else {
    k_nn_warp<false><<<blocks, 256, 0, stream>>>(d_segs, S, inline_seg, total_slots, order,
                                                 order_err);
  }
  count_launch(1);
}

cudaError_t run_nn_sort_device(int S, uint32_t total_tiles, const NnTables& t,
                               cudaStream_t stream) {
  if (total_tiles == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(t.err, 0, sizeof(Header), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(t.sort.hist, 0, t.sort.zero_bytes, stream);
  if (e != cudaSuccess) return e;
  k_nn_keys<<<total_tiles * (kTile / 256), 256, 0, stream>>>(
      t.segs, S, static_cast<unsigned long long*>(t.sort.keys0), t.sort.hist);
  count_launch(1);
  return run_radix_passes(S, total_tiles, 4, true, t.sort, stream);
}

cudaError_t run_nn_search(const NnSeg& seg, const unsigned long long* order, cudaStream_t stream) {
  if (seg.m == 0) return cudaSuccess;
  launch_search(nullptr, 1, seg, seg.num_tiles, order, nullptr, seg.has_coarse != 0, stream);
  return cudaGetLastError();
}

cudaError_t run_nn_device(int S, uint32_t total_tiles, const NnTables& t, cudaStream_t stream,
                          bool any_coarse) {
  if (total_tiles == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(t.err, 0, sizeof(Header), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(t.sort.hist, 0, t.sort.zero_bytes, stream);
  if (e != cudaSuccess) return e;
  k_nn_keys<<<total_tiles * (kTile / 256), 256, 0, stream>>>(
      t.segs, S, static_cast<unsigned long long*>(t.sort.keys0), t.sort.hist);
  count_launch(1);
  e = run_radix_passes(S, total_tiles, 4, true, t.sort, stream);
  if (e != cudaSuccess) return e;
  // four passes leave the sorted keys in keys0
  launch_search(t.segs, S, NnSeg{}, total_tiles,
                static_cast<const unsigned long long*>(t.sort.keys0), &t.err->err, any_coarse,
                stream);
  return cudaGetLastError();
}

cudaError_t run_nn(const NnSeg* h_segs, int S, uint32_t total_tiles, void* scratch,
                   cudaStream_t stream) {
  if (total_tiles == 0) return cudaSuccess;
  if (scratch == nullptr) {
    if (S != 1) return cudaErrorInvalidValue;
    launch_search(nullptr, 1, h_segs[0], total_tiles, nullptr, nullptr,
                  h_segs[0].has_coarse != 0, stream);
    return cudaGetLastError();
  }
  const NnTables t = nn_tables(scratch, total_tiles, S);
  const cudaError_t e = nn_upload(h_segs, S, t, stream);
  if (e != cudaSuccess) return e;
  bool any_coarse = false;
  for (int s = 0; s < S; ++s) any_coarse = any_coarse || h_segs[s].has_coarse != 0;
  return run_nn_device(S, total_tiles, t, stream, any_coarse);
}

}  // namespace libcga
