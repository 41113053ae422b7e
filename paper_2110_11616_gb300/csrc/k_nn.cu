// Exact nearest-neighbour search on a CGA (Eq. 7-8, Sec. V-C).
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
#include <atomic>
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

// |v - q| of a stored coordinate and a query coordinate (clamped to +-2^30,
// so the difference fits 31 bits; its square is one widening multiply).
__device__ __forceinline__ uint32_t absdiff(uint32_t v, int q) {
  const int d = (int)v - q;
  return (uint32_t)(d < 0 ? -d : d);
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
  if (local < sg.m && sg.qv != nullptr) {
    // integer query voxels: clamped to the grid for the ordering only
    const uint32_t bits = sg.a.bits;
    const int top = (1 << bits) - 1;
    uint32_t c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const uint32_t u = (uint32_t)min(max(__ldg(sg.qv + 3 * (size_t)local + a), 0), top);
      c[a] = bits >= 10 ? (u >> (bits - 10)) : (u << (10 - bits));
    }
    const uint32_t mort = (spread3(c[0]) << 2) | (spread3(c[1]) << 1) | spread3(c[2]);
    keys[slot] = ((unsigned long long)mort << 32) | local;
#pragma unroll
    for (int k = 0; k < 4; ++k) atomicAdd(&s_hist[k][(mort >> (8 * k)) & (kRadix - 1)], 1u);
  } else if (local < sg.m) {
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

// The best (distance^2, index) so far.  The CGA index of a voxel rises with
// its key, so the least index among equal distances is the smallest key
// (Eq. 8's tie rule).
struct Best {
  unsigned long long d2;
  uint32_t idx;
  __device__ __forceinline__ void offer(unsigned long long d, uint32_t i) {
    if (d < d2 || (d == d2 && i < idx)) {
      d2 = d;
      idx = i;
    }
  }
  // Lexicographic minimum of (d2, idx) over the warp, by 32-bit warp
  // reductions of the high then the low distance word, then the index.
  __device__ __forceinline__ void warp_min() {
    const uint32_t full = 0xffffffffu;
    const uint32_t dh = (uint32_t)(d2 >> 32), dl = (uint32_t)d2;
    const uint32_t mh = __reduce_min_sync(full, dh);
    const uint32_t ml = __reduce_min_sync(full, dh == mh ? dl : full);
    idx = __reduce_min_sync(full, dh == mh && dl == ml ? idx : full);
    d2 = ((unsigned long long)mh << 32) | ml;
  }
};

// The two z neighbours of the query in column c.  ctab (or null): the column
// table, whose entry holds the column's voxel range and its lowest | highest
// z << 16 in one 16-byte load; when the query lies below or above the whole
// column, that end is the only neighbour and no search is needed.
__device__ __forceinline__ void visit_column(const Levels& a, const uint4* ctab, uint32_t c,
                                             unsigned long long dxy, int qz, uint32_t cqz,
                                             Best& b) {
  uint32_t zs, ze;
  if (ctab != nullptr) {
    const uint4 e = __ldg(ctab + c);
    zs = e.x;
    ze = e.y;
    const uint32_t zz = e.z;
    const uint32_t zlo = zz & 0xffffu, zhi = zz >> 16;
    if (cqz <= zlo) {
      const unsigned long long dz = absdiff(zlo, qz);
      b.offer(dxy + dz * dz, zs);
      return;
    }
    if (cqz >= zhi) {
      const unsigned long long dz = absdiff(zhi, qz);
      b.offer(dxy + dz * dz, ze - 1);
      return;
    }
  } else {
    zs = __ldg(a.ptr1 + c);
    ze = __ldg(a.ptr1 + c + 1);
  }
  const uint32_t zr = lower_bound_u16(a.idx0, zs, ze, cqz);
  if (zr < ze) {
    const uint32_t z = __ldg(a.idx0 + zr);
    const unsigned long long dz = absdiff(z, qz);
    b.offer(dxy + dz * dz, zr);
  }
  if (zr > zs) {
    const uint32_t z = __ldg(a.idx0 + zr - 1);
    const unsigned long long dz = absdiff(z, qz);
    b.offer(dxy + dz * dz, zr - 1);
  }
}

// Window search over the fine CGA alone (one warp, 16 slabs per side per round).
__device__ __forceinline__ void search_fine(const Levels& a, const uint32_t* xdir,
                                            const uint4* ctab, uint32_t h,
                                            int qx, int qy, int qz,
                                            uint32_t cqx, uint32_t cqy, uint32_t cqz,
                                            uint32_t lane, Best& best) {
  const uint32_t xr0 = xdir != nullptr ? __ldg(xdir + cqx) : lower_bound_u16(a.idx2, 0, h, cqx);
  const bool right = (lane & 1u) == 0u;
  for (uint32_t r = 0;; ++r) {
    const int k = (int)(r * 16u + (lane >> 1));
    const int slab = right ? (int)xr0 + k : (int)xr0 - 1 - k;
    const bool valid = slab >= 0 && slab < (int)h;
    unsigned long long dx2 = ~0ull;
    uint32_t x = 0, ys = 0, ye = 0, yr0 = 0;
    if (valid) {
      // the slab's column range is loaded together with its x value
      x = __ldg(a.idx2 + slab);
      ys = __ldg(a.ptr2 + slab);
      ye = __ldg(a.ptr2 + slab + 1);
      const unsigned long long dx = absdiff(x, qx);
      dx2 = dx * dx;
    }
    const bool active = valid && dx2 <= best.d2;
    if (!__any_sync(0xffffffffu, active)) break;
    if (active) {
      yr0 = lower_bound_u16(a.idx1, ys, ye, cqy);
      if (yr0 < ye) {
        const uint32_t y = __ldg(a.idx1 + yr0);
        const unsigned long long dy = absdiff(y, qy);
        const unsigned long long dxy = dx2 + dy * dy;
        if (dxy <= best.d2) {
          visit_column(a, ctab, yr0, dxy, qz, cqz, best);
        }
      }
      if (yr0 > ys) {
        const uint32_t y = __ldg(a.idx1 + yr0 - 1);
        const unsigned long long dy = absdiff(y, qy);
        const unsigned long long dxy = dx2 + dy * dy;
        if (dxy <= best.d2) {
          visit_column(a, ctab, yr0 - 1, dxy, qz, cqz, best);
        }
      }
    }
    best.warp_min();
    if (active) {
      int R2 = (int)yr0 + 1, L2 = (int)yr0 - 2;
      while (true) {
        const bool hR = R2 < (int)ye, hL = L2 >= (int)ys;
        if (!hR && !hL) break;
        const uint32_t eR = hR ? absdiff(__ldg(a.idx1 + R2), qy) : 0xffffffffu;
        const uint32_t eL = hL ? absdiff(__ldg(a.idx1 + L2), qy) : 0xffffffffu;
        const bool gR = hR && (!hL || eR <= eL);
        const unsigned long long dy = gR ? eR : eL;
        const unsigned long long dxy = dx2 + dy * dy;
        if (dxy > best.d2) break;
        const uint32_t c = (uint32_t)(gR ? R2 : L2);
        if (gR) ++R2; else --L2;
        visit_column(a, ctab, c, dxy, qz, cqz, best);
      }
    }
    best.warp_min();
  }
}

// Distance from q to the voxel interval [lo, lo + s - 1] (0 inside).
__device__ __forceinline__ uint32_t interval_dist(int q, uint32_t lo, uint32_t s) {
  const int l = (int)lo, hi = (int)(lo + s - 1);
  return q < l ? (uint32_t)(l - q) : (q > hi ? (uint32_t)(q - hi) : 0u);
}

// A query in voxel units: unclamped (x, y, z) for distances, clamped
// (cx, cy, cz) inside the grid for searches.
constexpr int kQueryLimit = 1 << 30;

// Blocks per SM the fine-only and the coarse searches are compiled for (their
// register budgets; measured on GB300: fine 6 beats 5 and 8, coarse 5 beats
// 4 and 6).
#ifndef CGA_NN_FINE_BLOCKS
#define CGA_NN_FINE_BLOCKS 6
#endif
#ifndef CGA_NN_COARSE_BLOCKS
#define CGA_NN_COARSE_BLOCKS 5
#endif
#ifndef CGA_NN_TREE_BLOCKS
#define CGA_NN_TREE_BLOCKS 4
#endif
// 1: a frame's child bounds are kept in shared memory for the way back
#ifndef CGA_NN_TREE_CACHE
#define CGA_NN_TREE_CACHE 1
#endif

struct Qry {
  int x, y, z;
  uint32_t cx, cy, cz;
};

// Level K of a segment: 0 is the CGA itself, 1..ncoarse its coarse levels.
template <int K>
__device__ __forceinline__ const Levels& level(const NnSeg& sg) {
  if constexpr (K == 0) return sg.a; else return sg.c[K - 1];
}
template <int K>
__device__ __forceinline__ uint32_t level_shift(const NnSeg& sg) {
  if constexpr (K == 0) return 0u; else return sg.shift[K - 1];
}

template <int K>
__device__ void visit_cell_column(const NnSeg& sg, uint32_t c, uint32_t cy,
                                  unsigned long long dxl2, unsigned long long dyl2, uint32_t cx0,
                                  uint32_t cx1, const Qry& q, Best& best);

// The slabs [x0, x1) of level K restricted to columns with y in [ylo, ylo +
// ysz) (level-K units): slabs are taken nearest to the query first, and the
// columns of a slab nearest first, so the best distance tightens early and
// each walk stops once its lower bound exceeds it.  Level 0 visits the fine
// columns; a column of a coarse level is refined one level down.
template <int K>
__device__ void refine_level(const NnSeg& sg, uint32_t x0, uint32_t x1, uint32_t ylo,
                             uint32_t ysz, const uint32_t* starts, const Qry& q, Best& best) {
  if constexpr (K == 0) {
    // the fine columns of one cell: few enough that a plain ascending scan
    // with the bound test per slab and per column beats ordering them
    const Levels& a = sg.a;
    for (uint32_t xi = x0; xi < x1; ++xi) {
      const uint32_t x = __ldg(a.idx2 + xi);
      const unsigned long long dx = absdiff(x, q.x);
      const unsigned long long dx2 = dx * dx;
      if (dx2 > best.d2) continue;
      const uint32_t ys = __ldg(a.ptr2 + xi), ye = __ldg(a.ptr2 + xi + 1);
      const uint32_t c0 = starts != nullptr ? __ldg(starts + (xi - x0))
                                            : lower_bound_u16(a.idx1, ys, ye, ylo);
      for (uint32_t c = c0; c < ye; ++c) {
        const uint32_t y = __ldg(a.idx1 + c);
        if (y >= ylo + ysz) break;
        const unsigned long long dy = absdiff(y, q.y);
        const unsigned long long dxy = dx2 + dy * dy;
        if (dxy > best.d2) continue;
        visit_column(a, sg.ctab, c, dxy, q.z, q.cz, best);
      }
    }
    return;
  }
  const Levels& L = level<K>(sg);
  const uint32_t sh = level_shift<K>(sg), cell = 1u << sh;
  const uint32_t qyc = q.cy >> sh;
  const uint32_t split = lower_bound_u16(L.idx2, x0, x1, q.cx >> sh);
  int r = (int)split, l = (int)split - 1;
  while (true) {
    const bool hr = r < (int)x1, hl = l >= (int)x0;
    if (!hr && !hl) break;
    const uint32_t vr = hr ? (uint32_t)__ldg(L.idx2 + r) : 0u;
    const uint32_t vl = hl ? (uint32_t)__ldg(L.idx2 + l) : 0u;
    const uint32_t er = hr ? interval_dist(q.x, vr << sh, cell) : 0xffffffffu;
    const uint32_t el = hl ? interval_dist(q.x, vl << sh, cell) : 0xffffffffu;
    const bool gr = hr && (!hl || er <= el);
    const unsigned long long dxl = gr ? er : el;
    const unsigned long long dxl2 = dxl * dxl;
    if (dxl2 > best.d2) break;
    const uint32_t xi = (uint32_t)(gr ? r : l), xv = gr ? vr : vl;
    if (gr) ++r; else --l;
    const uint32_t ys = __ldg(L.ptr2 + xi), ye = __ldg(L.ptr2 + xi + 1);
    // columns [c0, c1) of this slab lie in the y range; cs: the first at or
    // beyond the query's row
    const uint32_t c0 = starts != nullptr ? __ldg(starts + (xi - x0))
                                          : lower_bound_u16(L.idx1, ys, ye, ylo);
    uint32_t cs = c0, c1 = c0;
    while (c1 < ye) {
      const uint32_t y = __ldg(L.idx1 + c1);
      if (y >= ylo + ysz) break;
      if (y < qyc) cs = c1 + 1;
      ++c1;
    }
    if (c0 == c1) continue;
    uint32_t fx0 = 0, fx1 = 0;
    if constexpr (K > 0) {
      fx0 = __ldg(sg.xs[K - 1] + xi);
      fx1 = __ldg(sg.xs[K - 1] + xi + 1);
    }
    int R = (int)cs, Lc = (int)cs - 1;
    while (true) {
      const bool hR = R < (int)c1, hL = Lc >= (int)c0;
      if (!hR && !hL) break;
      const uint32_t yR = hR ? (uint32_t)__ldg(L.idx1 + R) : 0u;
      const uint32_t yL = hL ? (uint32_t)__ldg(L.idx1 + Lc) : 0u;
      const uint32_t eR = hR ? interval_dist(q.y, yR << sh, cell) : 0xffffffffu;
      const uint32_t eL = hL ? interval_dist(q.y, yL << sh, cell) : 0xffffffffu;
      const bool gR = hR && (!hL || eR <= eL);
      const unsigned long long dyl = gR ? eR : eL;
      if (dxl2 + dyl * dyl > best.d2) break;
      const uint32_t c = (uint32_t)(gR ? R : Lc), yv = gR ? yR : yL;
      if (gR) ++R; else --Lc;
      if constexpr (K == 0) {
        visit_column(L, sg.ctab, c, dxl2 + dyl * dyl, q.z, q.cz, best);
      } else {
        visit_cell_column<K>(sg, c, yv, dxl2, dyl * dyl, fx0, fx1, q, best);
      }
    }
  }
}

// Distance along z from the query to the nearest occupied cell of column c
// of level K >= 1.
template <int K>
__device__ __forceinline__ unsigned long long cell_z_dist(const NnSeg& sg, uint32_t c,
                                                          const Qry& q) {
  const Levels& L = level<K>(sg);
  const uint32_t sh = level_shift<K>(sg), cell = 1u << sh;
  const uint4* ctab = sg.zr[K - 1];
  uint32_t zs, ze;
  if (ctab != nullptr) {
    // one load: the column's cell range and z range; below or above the whole
    // column, the nearest cell is its lowest or highest
    const uint4 e = __ldg(ctab + c);
    const uint32_t qc = q.cz >> sh;
    const uint32_t zlo = e.z & 0xffffu, zhi = e.z >> 16;
    if (qc <= zlo) return interval_dist(q.z, zlo << sh, cell);
    if (qc >= zhi) return interval_dist(q.z, zhi << sh, cell);
    zs = e.x;
    ze = e.y;
  } else {
    zs = __ldg(L.ptr1 + c);
    ze = __ldg(L.ptr1 + c + 1);
  }
  const uint32_t zr = lower_bound_u16(L.idx0, zs, ze, q.cz >> sh);
  unsigned long long dzl = ~0ull;
  if (zr < ze) dzl = min(dzl, (unsigned long long)interval_dist(q.z, (uint32_t)__ldg(L.idx0 + zr) << sh, cell));
  if (zr > zs) {
    dzl = min(dzl, (unsigned long long)interval_dist(q.z, (uint32_t)__ldg(L.idx0 + zr - 1) << sh, cell));
  }
  return dzl;
}

// Column c (y = cy) of level K >= 1: its nearest occupied cells along z bound
// every point below it; refine the column's footprint one level down (the
// finer slabs [cx0, cx1), y range of the cell) only if that bound can beat the
// best distance so far.
template <int K>
__device__ void visit_cell_column(const NnSeg& sg, uint32_t c, uint32_t cy,
                                  unsigned long long dxl2, unsigned long long dyl2, uint32_t cx0,
                                  uint32_t cx1, const Qry& q, Best& best) {
  if (dxl2 + dyl2 > best.d2) return;
  const unsigned long long dzl = cell_z_dist<K>(sg, c, q);
  if (dxl2 + dyl2 + dzl * dzl > best.d2) return;
  const uint32_t dsh = level_shift<K>(sg) - level_shift<K - 1>(sg);
  const uint32_t* child = sg.child[K - 1];
  refine_level<K - 1>(sg, cx0, cx1, cy << dsh, 1u << dsh,
                      child != nullptr ? child + ((size_t)c << dsh) : nullptr, q, best);
}

// Window search whose rounds run over the coarsest level TOP (cells of
// 2^shift voxels) with box lower bounds; surviving cells are refined level by
// level down to the fine columns.  A point lies in an occupied cell at every
// level whose bound never exceeds the point's distance, so pruning by
// "bound > best" never drops a point at or below the final distance.
template <int TOP>
__device__ void search_levels(const NnSeg& sg, const Qry& q, uint32_t lane, Best& best) {
  const Levels& c = level<TOP>(sg);
  const uint32_t L = level_shift<TOP>(sg), s = 1u << L;
  const uint32_t* xs = sg.xs[TOP - 1];
  const uint32_t* cxdir = sg.cxdir[TOP - 1];
  const uint32_t hc = (uint32_t)c.hdr->cnt[2];
  const uint32_t xr0 = cxdir != nullptr ? __ldg(cxdir + (q.cx >> L))
                                        : lower_bound_u16(c.idx2, 0, hc, q.cx >> L);
  const uint32_t cqy_c = q.cy >> L;
  const bool right = (lane & 1u) == 0u;
  {
    // Seed: each lane bounds the two columns of one nearest slab that are
    // nearest in y (box lower bound with z from the column's nearest cells);
    // only the column with the least bound in the warp is refined, so the
    // rounds below start from a real candidate instead of an infinite bound.
    const int slab = right ? (int)xr0 + (int)(lane >> 1) : (int)xr0 - 1 - (int)(lane >> 1);
    unsigned long long lb = ~0ull, sdx2 = 0, sdy2 = 0;
    uint32_t sc = 0, scy = 0, sfx0 = 0, sfx1 = 0;
    if (slab >= 0 && slab < (int)hc) {
      const unsigned long long dxl = interval_dist(q.x, (uint32_t)__ldg(c.idx2 + slab) << L, s);
      const uint32_t ys = __ldg(c.ptr2 + slab), ye = __ldg(c.ptr2 + slab + 1);
      const uint32_t yr0 = lower_bound_u16(c.idx1, ys, ye, cqy_c);
      sfx0 = __ldg(xs + slab);
      sfx1 = __ldg(xs + slab + 1);
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const uint32_t cc = yr0 - (uint32_t)t;
        if (t == 0 ? yr0 >= ye : yr0 <= ys) continue;
        const uint32_t cy = __ldg(c.idx1 + cc);
        const unsigned long long dyl = interval_dist(q.y, cy << L, s);
        const unsigned long long dzl = cell_z_dist<TOP>(sg, cc, q);
        const unsigned long long bnd = dxl * dxl + dyl * dyl + dzl * dzl;
        if (bnd < lb) {
          lb = bnd;
          sc = cc;
          scy = cy;
          sdx2 = dxl * dxl;
          sdy2 = dyl * dyl;
        }
      }
    }
    unsigned long long v = lb;
    uint32_t win = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ov = __shfl_xor_sync(0xffffffffu, v, o);
      const uint32_t ol = __shfl_xor_sync(0xffffffffu, win, o);
      if (ov < v || (ov == v && ol < win)) {
        v = ov;
        win = ol;
      }
    }
    if (v != ~0ull && lane == win) {
      visit_cell_column<TOP>(sg, sc, scy, sdx2, sdy2, sfx0, sfx1, q, best);
    }
    best.warp_min();
  }
  for (uint32_t r = 0;; ++r) {
    const int k = (int)(r * 16u + (lane >> 1));
    const int slab = right ? (int)xr0 + k : (int)xr0 - 1 - k;
    const bool valid = slab >= 0 && slab < (int)hc;
    unsigned long long dxl2 = ~0ull;
    if (valid) {
      const unsigned long long dxl = interval_dist(q.x, (uint32_t)__ldg(c.idx2 + slab) << L, s);
      dxl2 = dxl * dxl;
    }
    const bool active = valid && dxl2 <= best.d2;
    if (!__any_sync(0xffffffffu, active)) break;
    uint32_t ys = 0, ye = 0, yr0 = 0, fx0 = 0, fx1 = 0;
    if (active) {
      ys = __ldg(c.ptr2 + slab);
      ye = __ldg(c.ptr2 + slab + 1);
      yr0 = lower_bound_u16(c.idx1, ys, ye, cqy_c);
      fx0 = __ldg(xs + slab);
      fx1 = __ldg(xs + slab + 1);
      if (yr0 < ye) {
        const uint32_t cy = __ldg(c.idx1 + yr0);
        const unsigned long long dyl = interval_dist(q.y, cy << L, s);
        visit_cell_column<TOP>(sg, yr0, cy, dxl2, dyl * dyl, fx0, fx1, q, best);
      }
      if (yr0 > ys) {
        const uint32_t cy = __ldg(c.idx1 + yr0 - 1);
        const unsigned long long dyl = interval_dist(q.y, cy << L, s);
        visit_cell_column<TOP>(sg, yr0 - 1, cy, dxl2, dyl * dyl, fx0, fx1, q, best);
      }
    }
    best.warp_min();
    if (active) {
      int R2 = (int)yr0 + 1, L2 = (int)yr0 - 2;
      while (true) {
        const bool hR = R2 < (int)ye, hL = L2 >= (int)ys;
        if (!hR && !hL) break;
        const uint32_t eR =
            hR ? interval_dist(q.y, (uint32_t)__ldg(c.idx1 + R2) << L, s) : 0xffffffffu;
        const uint32_t eL =
            hL ? interval_dist(q.y, (uint32_t)__ldg(c.idx1 + L2) << L, s) : 0xffffffffu;
        const bool gR = hR && (!hL || eR <= eL);
        const unsigned long long dyl = gR ? eR : eL;
        if (dxl2 + dyl * dyl > best.d2) break;
        const uint32_t cc = (uint32_t)(gR ? R2 : L2);
        if (gR) ++R2; else --L2;
        visit_cell_column<TOP>(sg, cc, __ldg(c.idx1 + cc), dxl2, dyl * dyl, fx0, fx1, q, best);
      }
    }
    best.warp_min();
  }
}

// ---- occupancy-tree search (cga_nn_prepare_levels with CGA_NN_TREE) -------
//
// A depth-first descent of the 64-ary occupancy tree (k_tree.cu), nearest
// child first.  The warp keeps one frame per level on the path: the node's
// child set, the children still to visit and the node's cell.  Each step the
// lanes bound two children each (box distance of the child cell; lane i takes
// children i and i + 32), drop every child whose bound exceeds the best
// distance so far, and the warp enters the remaining child with the least
// bound.  Children of a level-2 node are bricks: their 64 voxels are examined
// at once (two per lane).  A child is dropped only when its bound exceeds the
// best distance, and the best distance never falls below the final one, so
// every cell holding a voxel at the final distance is entered: the result is
// Eq. 8's nearest voxel, ties to the smaller key.

// Squared distance from q to the cell [lo, lo + s - 1] along one axis, in D
// (uint32_t when every squared distance of the search fits 32 bits: a grid of
// at most 15 bits per axis and a query inside it; else 64 bits).
template <typename D>
__device__ __forceinline__ D axis_lb2(int q, uint32_t lo, uint32_t s) {
  const D d = interval_dist(q, lo, s);
  return d * d;
}

struct TreeFrame {
  unsigned long long mask, rem;
  uint32_t first, ox, oy, oz, lvl, pad;
};

// Warp minimum of a D value (32-bit words, high first).
__device__ __forceinline__ uint32_t warp_min_d(uint32_t v) {
  return __reduce_min_sync(0xffffffffu, v);
}
__device__ __forceinline__ unsigned long long warp_min_d(unsigned long long v) {
  const uint32_t full = 0xffffffffu;
  const uint32_t vh = (uint32_t)(v >> 32), vl = (uint32_t)v;
  const uint32_t mh = __reduce_min_sync(full, vh);
  const uint32_t ml = __reduce_min_sync(full, vh == mh ? vl : full);
  return ((unsigned long long)mh << 32) | ml;
}

// The best (distance^2, key) of the tree search.
template <typename D>
struct BestKey {
  D d2;
  unsigned long long key;
  // Lexicographic minimum of the lanes' (d, k).
  __device__ __forceinline__ void warp_min_of(D d, unsigned long long k) {
    const uint32_t full = 0xffffffffu;
    const D md = warp_min_d(d);
    const bool at = d == md;
    const uint32_t kh = __reduce_min_sync(full, at ? (uint32_t)(k >> 32) : full);
    const uint32_t kl = __reduce_min_sync(full, at && (uint32_t)(k >> 32) == kh ? (uint32_t)k : full);
    d2 = md;
    key = ((unsigned long long)kh << 32) | kl;
  }
};

// The voxels of the brick at brick coordinates (bx, by, bz) with occupancy
// m: lane i takes voxels i and i + 32 (bit c = cx << 4 | cy << 2 | cz).
template <typename D>
__device__ __forceinline__ void tree_brick(unsigned long long m, uint32_t bx, uint32_t by,
                                           uint32_t bz, const Qry& q, uint32_t b, uint32_t lane,
                                           BestKey<D>& best) {
  const uint32_t y = (by << 2) + ((lane >> 2) & 3u), z = (bz << 2) + (lane & 3u);
  const uint32_t x0 = (bx << 2) + (lane >> 4);
  const D dy = absdiff(y, q.y), dz = absdiff(z, q.z);
  const D dyz = dy * dy + dz * dz;
  const unsigned long long yz = ((unsigned long long)y << b) | z;
  D cd = (D)~(D)0;
  unsigned long long ck = ~0ull;
  if ((m >> lane) & 1ull) {
    const D dx = absdiff(x0, q.x);
    cd = dx * dx + dyz;
    ck = ((unsigned long long)x0 << (2 * b)) | yz;
  }
  if ((m >> (lane + 32)) & 1ull) {
    const D dx = absdiff(x0 + 2, q.x);
    const D d = dx * dx + dyz;
    if (d < cd) {  // on a tie the smaller x (smaller key) stays
      cd = d;
      ck = ((unsigned long long)(x0 + 2) << (2 * b)) | yz;
    }
  }
  const bool better = cd < best.d2 || (cd == best.d2 && ck < best.key);
  if (__any_sync(0xffffffffu, better)) {
    best.warp_min_of(better ? cd : best.d2, better ? ck : best.key);
  }
}

// Bound of a child cell from its box code: the box of its occupied voxels
// (FB-bit bounds in cells of 2^ss voxels) inside the cell at voxel origin
// (X, Y, Z).
template <typename D, int FB>
__device__ __forceinline__ D child_lb(const Qry& q, uint32_t X, uint32_t Y, uint32_t Z,
                                      uint32_t k, uint32_t ss) {
  constexpr uint32_t fm = (1u << FB) - 1u;
  const uint32_t lx = k & fm, hx = (k >> FB) & fm, ly = (k >> (2 * FB)) & fm,
                 hy = (k >> (3 * FB)) & fm, lz = (k >> (4 * FB)) & fm, hz = (k >> (5 * FB)) & fm;
  return axis_lb2<D>(q.x, X + (lx << ss), (hx - lx + 1) << ss) +
         axis_lb2<D>(q.y, Y + (ly << ss), (hy - ly + 1) << ss) +
         axis_lb2<D>(q.z, Z + (lz << ss), (hz - lz + 1) << ss);
}
template <typename D>
__device__ __forceinline__ D child_lb_any(bool brick, const Qry& q, uint32_t X, uint32_t Y,
                                          uint32_t Z, uint32_t k, uint32_t ss) {
  return brick ? child_lb<D, 2>(q, X, Y, Z, k, 0u) : child_lb<D, 4>(q, X, Y, Z, k, ss);
}

// The warp's smallest key among the voxels of the bricks given to this lane
// (occupancy m, voxel origin (bx, by, bz)) that beat `best`, merged into it.
template <typename D>
__device__ __forceinline__ void brick_voxels(unsigned long long m, uint32_t bx, uint32_t by,
                                             uint32_t bz, const Qry& q, uint32_t b, D& cd,
                                             unsigned long long& ck) {
  while (m != 0ull) {
    const uint32_t v = (uint32_t)__ffsll((long long)m) - 1u;
    m &= m - 1ull;
    const uint32_t x = bx + (v >> 4), y = by + ((v >> 2) & 3u), z = bz + (v & 3u);
    const D dx = absdiff(x, q.x), dy = absdiff(y, q.y), dz = absdiff(z, q.z);
    const D d = dx * dx + dy * dy + dz * dz;
    if (d <= cd) {  // the key is formed only for a voxel that can win
      const unsigned long long k = ((unsigned long long)x << (2 * b)) |
                                   ((unsigned long long)y << b) | z;
      if (d < cd || k < ck) {
        cd = d;
        ck = k;
      }
    }
  }
}

template <typename D>
__device__ void search_tree(const NnSeg& sg, const Qry& q, uint32_t lane, TreeFrame* fr,
                            uint32_t* lbc, uint32_t* pos, BestKey<D>& best) {
  const uint32_t full = 0xffffffffu;
  const TreeView& tv = sg.tree;
  const uint32_t T = tv.levels, b = sg.a.bits;
  if (T == 1) {
    tree_brick(__ldg(tv.brick), 0, 0, 0, q, b, lane, best);
    return;
  }
  uint32_t lvl = T;
  const uint4 r0 = __ldg(tv.node[T]);
  unsigned long long mask = r0.x | ((unsigned long long)r0.y << 32), rem = mask;
  uint32_t first = r0.z, ox = 0, oy = 0, oz = 0;
  int depth = 0;
  bool s_pop = false;
  // fresh: the current frame was just entered (its children's bounds are
  // computed and, above level 2, kept in lbc[depth] for the way back)
  bool fresh = true;
  while (true) {
    // a stored voxel at distance 0 is the answer (voxels are unique, so no
    // other voxel can tie with it)
    if (best.d2 == (D)0) break;
    // The children still to visit, compacted: lane k takes the k-th of them
    // (and the (k+32)-th when more than 32 are left), so a node with few
    // children keeps few lanes busy instead of two fixed slots per lane.
    // Each lane loads the record of its child (a node's child set and first
    // child, or a brick's voxels) with its box code, so that the chosen
    // child's record is already in a register when the warp enters it.
    const uint32_t rlo = (uint32_t)rem, rhi = (uint32_t)(rem >> 32);
    const uint32_t nlo = __popc(rlo), nr = nlo + __popc(rhi);
    const uint32_t ltm = lanemask_lt();
    __syncwarp();
    if ((rlo >> lane) & 1u) pos[__popc(rlo & ltm)] = lane;
    if ((rhi >> lane) & 1u) pos[nlo + __popc(rhi & ltm)] = lane + 32;
    __syncwarp();
    const bool two = nr > 32;  // warp-uniform
    const bool h0 = lane < nr, h1 = two && lane + 32 < nr;
    const uint32_t c0 = h0 ? pos[lane] : 0u, c1 = h1 ? pos[lane + 32] : 0u;
    // box codes: bricks (children of level 2) in voxels, 2 bits per bound;
    // nodes in their grandchild units (4^(lvl-3) voxels), 4 bits per bound
    const uint32_t sh = 2 * (lvl - 1);
    const uint32_t ss = lvl == 2 ? 0u : sh - 4;
    const uint32_t cap = tv.cap[lvl - 1];
    const uint32_t i0 = first + (uint32_t)__popcll(mask & ((1ull << c0) - 1ull));
    const uint32_t i1 = first + (uint32_t)__popcll(mask & ((1ull << c1) - 1ull));
    const bool cached = CGA_NN_TREE_CACHE && !fresh;
    uint4 k0 = make_uint4(0u, 0u, 0u, 0u), k1 = make_uint4(0u, 0u, 0u, 0u);
    D lb0 = (D)~(D)0, lb1 = (D)~(D)0;
    if (cached) {
      // back in a frame above level 2: its bounds are kept (no loads; a kept
      // bound saturates at 2^32 - 1, still a lower bound)
      if (h0) lb0 = (D)lbc[depth * 64 + c0];
      if (h1) lb1 = (D)lbc[depth * 64 + c1];
    } else {
      if (lvl == 2) {
        if (h0 && i0 < cap) {
          const unsigned long long m0 = __ldg(tv.brick + i0);
          k0 = make_uint4((uint32_t)m0, (uint32_t)(m0 >> 32), 0u, __ldg(tv.bcode + i0));
        }
        if (h1 && i1 < cap) {
          const unsigned long long m1 = __ldg(tv.brick + i1);
          k1 = make_uint4((uint32_t)m1, (uint32_t)(m1 >> 32), 0u, __ldg(tv.bcode + i1));
        }
      } else {
        const uint4* nd = tv.node[lvl - 1];
        if (h0 && i0 < cap) k0 = __ldg(nd + i0);
        if (h1 && i1 < cap) k1 = __ldg(nd + i1);
      }
      if (h0) {
        lb0 = child_lb_any<D>(lvl == 2, q, ((ox << 2) + (c0 >> 4)) << sh,
                              ((oy << 2) + ((c0 >> 2) & 3u)) << sh, ((oz << 2) + (c0 & 3u)) << sh,
                              k0.w, ss);
      }
      if (two && h1) {
        lb1 = child_lb_any<D>(lvl == 2, q, ((ox << 2) + (c1 >> 4)) << sh,
                              ((oy << 2) + ((c1 >> 2) & 3u)) << sh, ((oz << 2) + (c1 & 3u)) << sh,
                              k1.w, ss);
      }
      if (CGA_NN_TREE_CACHE && lvl > 2) {
        if (h0) lbc[depth * 64 + c0] = lb0 > (D)0xfffffffeu ? 0xffffffffu : (uint32_t)lb0;
        if (h1) lbc[depth * 64 + c1] = lb1 > (D)0xfffffffeu ? 0xffffffffu : (uint32_t)lb1;
      }
    }
    const bool in0 = h0 && i0 < cap && lb0 <= best.d2;
    const bool in1 = h1 && i1 < cap && lb1 <= best.d2;
    const uint32_t s0 = __ballot_sync(full, in0), s1 = __ballot_sync(full, in1);
    // the surviving children as a child set
    const uint32_t o0 = in0 ? c0 : 64u, o1 = in1 ? c1 : 64u;
    unsigned long long surv = 0ull;
    if (s0 | s1) {
      const uint32_t bl0 = o0 < 32 ? 1u << o0 : 0u, bh0 = o0 >= 32 && o0 < 64 ? 1u << (o0 - 32) : 0u;
      const uint32_t bl1 = o1 < 32 ? 1u << o1 : 0u, bh1 = o1 >= 32 && o1 < 64 ? 1u << (o1 - 32) : 0u;
      const uint32_t sl = __reduce_or_sync(full, bl0 | bl1), shi = __reduce_or_sync(full, bh0 | bh1);
      surv = ((unsigned long long)shi << 32) | sl;
    }
    if (lvl == 2 && surv != 0ull) {
      // Children are bricks.  Without a candidate yet only the nearest brick
      // is examined (its voxels set a bound that prunes its siblings), else
      // every lane examines the voxels of its surviving bricks (a loop over
      // their occupancy bits) and the level-2 node is done.
      const bool only_nearest = best.d2 == (D)~(D)0;
      bool e0 = in0, e1 = in1;
      uint32_t cs_first = 64;
      if (only_nearest) {
        D v = in0 ? lb0 : (D)~(D)0;
        uint32_t c = c0;
        if (in1 && lb1 < v) {
          v = lb1;
          c = c1;
        }
        const D mv = warp_min_d(v);
        const uint32_t win = __ballot_sync(full, (in0 || in1) && v == mv);
        cs_first = __shfl_sync(full, c, __ffs(win) - 1);
        e0 = in0 && cs_first == c0;
        e1 = in1 && cs_first == c1;
      }
      D cd = (D)~(D)0;
      unsigned long long ck = ~0ull;
      if (e0) {
        brick_voxels<D>(k0.x | ((unsigned long long)k0.y << 32),
                        ((ox << 2) + (c0 >> 4)) << 2, ((oy << 2) + ((c0 >> 2) & 3u)) << 2,
                        ((oz << 2) + (c0 & 3u)) << 2, q, b, cd, ck);
      }
      if (e1) {
        brick_voxels<D>(k1.x | ((unsigned long long)k1.y << 32),
                        ((ox << 2) + (c1 >> 4)) << 2, ((oy << 2) + ((c1 >> 2) & 3u)) << 2,
                        ((oz << 2) + (c1 & 3u)) << 2, q, b, cd, ck);
      }
      const bool better = cd < best.d2 || (cd == best.d2 && ck < best.key);
      if (__any_sync(full, better)) {
        best.warp_min_of(better ? cd : best.d2, better ? ck : best.key);
      }
      if (only_nearest) {
        rem = surv & ~(1ull << cs_first);
        continue;
      }
      s_pop = true;
    }
    if (surv == 0ull || s_pop) {
      s_pop = false;
      if (depth == 0) break;
      --depth;
      fresh = false;
      __syncwarp();
      const TreeFrame f = fr[depth];
      lvl = f.lvl;
      mask = f.mask;
      rem = f.rem;
      first = f.first;
      ox = f.ox;
      oy = f.oy;
      oz = f.oz;
      continue;
    }
    // the surviving child with the least bound, and its record from the lane
    // that loaded it
    D v = in0 ? lb0 : (D)~(D)0;
    uint32_t c = c0;
    if (in1 && lb1 < v) {
      v = lb1;
      c = c1;
    }
    const D mv = warp_min_d(v);
    const uint32_t win = __ballot_sync(full, (in0 || in1) && v == mv);
    const int owner = __ffs(win) - 1;
    const uint32_t cs = __shfl_sync(full, c, owner);
    uint32_t rx, ry, rz;
    if (cached) {
      const uint32_t ci = first + (uint32_t)__popcll(mask & ((1ull << cs) - 1ull));
      const uint4 r = __ldg(tv.node[lvl - 1] + ci);  // ci < cap: cs survived the check above
      rx = r.x;
      ry = r.y;
      rz = r.z;
    } else {
      const uint4 mine = cs == c1 && in1 ? k1 : k0;
      rx = __shfl_sync(full, mine.x, owner);
      ry = __shfl_sync(full, mine.y, owner);
      rz = __shfl_sync(full, mine.z, owner);
    }
    rem = surv & ~(1ull << cs);
    const uint32_t nx = (ox << 2) + (cs >> 4), ny = (oy << 2) + ((cs >> 2) & 3u),
                   nz = (oz << 2) + (cs & 3u);
    // (lvl > 2 here: a level-2 node was settled above.)  The last surviving
    // child replaces its parent's frame (nothing to come back to); otherwise
    // the parent's frame is kept for the way back.
    if (rem != 0ull) {
      __syncwarp();
      if (lane == 0) fr[depth] = TreeFrame{mask, rem, first, ox, oy, oz, lvl, 0u};
      __syncwarp();
      ++depth;
    }
    --lvl;
    mask = rx | ((unsigned long long)ry << 32);
    rem = mask;
    first = rz;
    ox = nx;
    oy = ny;
    oz = nz;
    fresh = true;
  }
}

// CGA index of the stored voxel with key `key` (the Sec. V-A lookup by the
// whole warp: x directory or X_index, the slab's Y range, the column's Z
// range).
__device__ __forceinline__ uint32_t stored_index(const NnSeg& sg, unsigned long long key) {
  const Levels& a = sg.a;
  const uint32_t b = a.bits, mk = (1u << b) - 1u;
  const uint32_t x = (uint32_t)(key >> (2 * b)), y = (uint32_t)(key >> b) & mk,
                 z = (uint32_t)key & mk;
  const uint32_t h = (uint32_t)a.hdr->cnt[2];
  const uint32_t slab = sg.xdir != nullptr ? __ldg(sg.xdir + x) : warp_lower_bound_u16(a.idx2, 0, h, x);
  const uint32_t ys = __ldg(a.ptr2 + slab), ye = __ldg(a.ptr2 + slab + 1);
  const uint32_t c = warp_lower_bound_u16(a.idx1, ys, ye, y);
  // the column's voxel range from Y_pointer (4 bytes a column; the 16-byte
  // column table is left out of L2's working set here)
  const uint32_t zs = __ldg(a.ptr1 + c), ze = __ldg(a.ptr1 + c + 1);
  return warp_lower_bound_u16(a.idx0, zs, ze, z);
}

// NC: the most coarse levels any segment of the launch carries (0, 1 or 2).
// The fine-only instantiation is held to 40 registers (six blocks per SM),
// the coarse ones to 48 (five blocks per SM): the extra warps hide more of
// the search's load latency than the spilled values cost (eight and six
// blocks respectively spill enough to be slower).
template <int NC>
__global__ void __launch_bounds__(256, NC == 3 ? CGA_NN_TREE_BLOCKS
                                               : (NC > 0 ? CGA_NN_COARSE_BLOCKS : CGA_NN_FINE_BLOCKS))
    k_nn_warp(const NnSeg* __restrict__ segs, int S, NnSeg inline_seg, uint32_t total_slots,
              const unsigned long long* __restrict__ order,
              const unsigned int* __restrict__ order_err) {
  __shared__ TreeFrame s_fr[NC == 3 ? 8 * kTreeMaxLevels : 1];
  __shared__ uint32_t s_lbc[NC == 3 && CGA_NN_TREE_CACHE ? 8 * kTreeMaxLevels * 64 : 1];
  __shared__ uint32_t s_pos[NC == 3 ? 8 * 64 : 1];
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const bool sorted = order != nullptr && (order_err == nullptr || *order_err == 0u);
  for (uint32_t slot = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; slot < total_slots;
       slot += nwarps) {
    const uint32_t tile = slot / (uint32_t)kTile;
    const NnSeg& sg = segs != nullptr ? segs[find_nn_seg(segs, S, tile)] : inline_seg;
    const uint32_t local = slot - sg.tile_base * (uint32_t)kTile;
    if (local >= sg.m) continue;
    // queries, the order and the results stream through once: loaded and
    // stored evict-first, so that L2 keeps the CGA and the search structures
    const uint32_t j = sorted ? (uint32_t)__ldcs(order + slot) : local;
    if (j >= sg.m) continue;  // a caller-given order that is not a permutation
    const Levels& a = sg.a;
    const uint32_t u = (uint32_t)a.hdr->cnt[0], h = (uint32_t)a.hdr->cnt[2];
    // query voxel, clamped to +-2^30 (so every coordinate difference fits 31 bits)
    int qx, qy, qz;
    bool valid;
    if (sg.qv != nullptr) {
      const int* v = sg.qv + 3 * (size_t)j;
      qx = min(max(__ldg(v), -kQueryLimit), kQueryLimit);
      qy = min(max(__ldg(v + 1), -kQueryLimit), kQueryLimit);
      qz = min(max(__ldg(v + 2), -kQueryLimit), kQueryLimit);
      valid = true;
    } else {
      const float* p = sg.q + 3 * (size_t)j;
      const float px = __ldcs(p), py = __ldcs(p + 1), pz = __ldcs(p + 2);
      valid = isfinite(px) && isfinite(py) && isfinite(pz);
      qx = valid ? (int)quantize_query(px, sg.scale, sg.off[0]) : 0;
      qy = valid ? (int)quantize_query(py, sg.scale, sg.off[1]) : 0;
      qz = valid ? (int)quantize_query(pz, sg.scale, sg.off[2]) : 0;
    }
    if (!valid || u == 0) {
      if (lane == 0) {
        __stcs(sg.idx + j, 0xffffffffu);
        __stcs(sg.d2 + j, ~0ull);
      }
      continue;
    }
    const uint32_t b = a.bits;
    const int top = (1 << b) - 1;
    const uint32_t cqx = (uint32_t)min(max(qx, 0), top);
    const uint32_t cqy = (uint32_t)min(max(qy, 0), top);
    const uint32_t cqz = (uint32_t)min(max(qz, 0), top);
    if constexpr (NC == 3) {
      if (sg.tree.levels > 0) {
        // 32-bit distances when every one fits: a query inside a grid of at
        // most 15 bits per axis (3 * (2^15 - 1)^2 < 2^32)
        const Qry qq{qx, qy, qz, cqx, cqy, cqz};
        TreeFrame* fr = s_fr + (threadIdx.x >> 5) * kTreeMaxLevels;
        uint32_t* lbc = CGA_NN_TREE_CACHE ? s_lbc + (threadIdx.x >> 5) * kTreeMaxLevels * 64 : s_lbc;
        uint32_t* pos = s_pos + (threadIdx.x >> 5) * 64;
        const bool narrow = b <= 15 && (uint32_t)qx == cqx && (uint32_t)qy == cqy &&
                            (uint32_t)qz == cqz;
        unsigned long long d2 = ~0ull, key = ~0ull;
        if (narrow) {
          BestKey<uint32_t> bk{0xffffffffu, ~0ull};
          search_tree<uint32_t>(sg, qq, lane, fr, lbc, pos, bk);
          if (bk.d2 != 0xffffffffu) {
            d2 = bk.d2;
            key = bk.key;
          }
        } else {
          BestKey<unsigned long long> bk{~0ull, ~0ull};
          search_tree<unsigned long long>(sg, qq, lane, fr, lbc, pos, bk);
          d2 = bk.d2;
          key = bk.key;
        }
        const uint32_t ix = d2 != ~0ull ? stored_index(sg, key) : 0xffffffffu;
        if (lane == 0) {
          __stcs(sg.idx + j, ix);
          __stcs(sg.d2 + j, d2);
        }
        continue;
      }
    }
    Best best{~0ull, 0xffffffffu};
    // (the tree kernel searches a segment without a tree by the fine search)
    if (NC == 2 && sg.ncoarse >= 2) {
      if constexpr (NC == 2) search_levels<2>(sg, Qry{qx, qy, qz, cqx, cqy, cqz}, lane, best);
    } else if ((NC == 1 || NC == 2) && sg.ncoarse >= 1) {
      if constexpr (NC == 1 || NC == 2) {
        search_levels<1>(sg, Qry{qx, qy, qz, cqx, cqy, cqz}, lane, best);
      }
    } else {
      search_fine(a, sg.xdir, sg.ctab, h, qx, qy, qz, cqx, cqy, cqz, lane, best);
    }
    if (lane == 0) {
      __stcs(sg.idx + j, best.idx);
      __stcs(sg.d2 + j, best.d2);
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

// Blocks of k_nn_warp<kind> that fit on one SM (queried once per kind).
static uint32_t resident_blocks(uint32_t kind) {
  static std::atomic<int> cache[4] = {{0}, {0}, {0}, {0}};
  int n = cache[kind].load(std::memory_order_relaxed);
  if (n == 0) {
    cudaError_t e = cudaErrorInvalidValue;
    if (kind == 0) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_nn_warp<0>, 256, 0);
    if (kind == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_nn_warp<1>, 256, 0);
    if (kind == 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_nn_warp<2>, 256, 0);
    if (kind == 3) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_nn_warp<3>, 256, 0);
    if (e != cudaSuccess || n <= 0) {
      cudaGetLastError();
      n = 4;
    }
    cache[kind].store(n, std::memory_order_relaxed);
  }
  return (uint32_t)n;
}

static void launch_search(const NnSeg* d_segs, int S, const NnSeg& inline_seg,
                          uint32_t total_tiles, const unsigned long long* order,
                          const unsigned int* order_err, uint32_t kind,
                          cudaStream_t stream) {
  const uint32_t total_slots = total_tiles * (uint32_t)kTile;
  // one wave: as many blocks as stay resident (the warps stride over the
  // query slots, so a second wave would only add its own tail)
  kind = std::min(kind, 3u);
  const uint32_t blocks = std::min<uint32_t>((total_slots + 7) / 8,
                                             (uint32_t)device_sm_count() * resident_blocks(kind));
  if (kind == 3) {
    k_nn_warp<3><<<blocks, 256, 0, stream>>>(d_segs, S, inline_seg, total_slots, order,
                                             order_err);
  } else if (kind == 2) {
    k_nn_warp<2><<<blocks, 256, 0, stream>>>(d_segs, S, inline_seg, total_slots, order,
                                             order_err);
  } else if (kind == 1) {
    k_nn_warp<1><<<blocks, 256, 0, stream>>>(d_segs, S, inline_seg, total_slots, order,
                                             order_err);
  } else {
    k_nn_warp<0><<<blocks, 256, 0, stream>>>(d_segs, S, inline_seg, total_slots, order,
                                             order_err);
  }
  count_launch(1);
}

void init_nn_kernels() {
  for (uint32_t k = 0; k < 4; ++k) resident_blocks(k);
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
  launch_search(nullptr, 1, seg, seg.num_tiles, order, nullptr, nn_kind(seg), stream);
  return cudaGetLastError();
}

cudaError_t run_nn_device(int S, uint32_t total_tiles, const NnTables& t, cudaStream_t stream,
                          uint32_t max_kind) {
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
                static_cast<const unsigned long long*>(t.sort.keys0), &t.err->err, max_kind,
                stream);
  return cudaGetLastError();
}

cudaError_t run_nn(const NnSeg* h_segs, int S, uint32_t total_tiles, void* scratch,
                   cudaStream_t stream) {
  if (total_tiles == 0) return cudaSuccess;
  if (scratch == nullptr) {
    if (S != 1) return cudaErrorInvalidValue;
    launch_search(nullptr, 1, h_segs[0], total_tiles, nullptr, nullptr, nn_kind(h_segs[0]),
                  stream);
    return cudaGetLastError();
  }
  const NnTables t = nn_tables(scratch, total_tiles, S);
  const cudaError_t e = nn_upload(h_segs, S, t, stream);
  if (e != cudaSuccess) return e;
  uint32_t max_kind = 0;
  for (int s = 0; s < S; ++s) max_kind = std::max(max_kind, nn_kind(h_segs[s]));
  return run_nn_device(S, total_tiles, t, stream, max_kind);
}

}  // namespace libcga
