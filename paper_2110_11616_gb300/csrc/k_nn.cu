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
// of the four passes over bits 32..63.  A block covers one tile.
__global__ void __launch_bounds__(256) k_nn_keys(const NnSeg* __restrict__ segs, int S,
                                                 unsigned long long* __restrict__ keys,
                                                 uint32_t* __restrict__ hist) {
  __shared__ uint32_t s_hist[4][kRadix];
  for (int i = threadIdx.x; i < 4 * kRadix; i += blockDim.x) (&s_hist[0][0])[i] = 0;
  __syncthreads();
  // one block per tile: its digit counts reach the global histogram once
  const uint32_t tile = blockIdx.x;
  const int s = find_nn_seg(segs, S, tile);
  const NnSeg& sg = segs[s];
  const uint32_t bits = sg.a.bits;
  for (uint32_t e = threadIdx.x; e < (uint32_t)kTile; e += 256u) {
    const uint32_t slot = tile * (uint32_t)kTile + e;
    const uint32_t local = slot - sg.tile_base * (uint32_t)kTile;
    if (local >= sg.m) break;
    uint32_t mort = 0x3fffffffu;
    if (sg.qv != nullptr) {
      // integer query voxels: clamped to the grid for the ordering only
      const int top = (1 << bits) - 1;
      uint32_t c[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const uint32_t u = (uint32_t)min(max(__ldg(sg.qv + 3 * (size_t)local + a), 0), top);
        c[a] = bits >= 10 ? (u >> (bits - 10)) : (u << (10 - bits));
      }
      mort = (spread3(c[0]) << 2) | (spread3(c[1]) << 1) | spread3(c[2]);
    } else {
      const float* p = sg.q + 3 * (size_t)local;
      const float px = p[0], py = p[1], pz = p[2];
      if (isfinite(px) && isfinite(py) && isfinite(pz)) {
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

// Blocks per SM the fine-only, the coarse and the tree searches are compiled
// for (their register budgets; measured on GB300: fine 6 beats 5 and 8,
// coarse 5 beats 4 and 6), and the lanes per query of the tree search.
#ifndef CGA_NN_FINE_BLOCKS
#define CGA_NN_FINE_BLOCKS 6
#endif
#ifndef CGA_NN_COARSE_BLOCKS
#define CGA_NN_COARSE_BLOCKS 5
#endif
#ifndef CGA_NN_TREE_BLOCKS
#define CGA_NN_TREE_BLOCKS 4
#endif
#ifndef CGA_NN_HEAD_GROUP
#define CGA_NN_HEAD_GROUP 16
#endif
#ifndef CGA_NN_TREE_GROUP
#define CGA_NN_TREE_GROUP 4
#endif

// Voxel of query j of a segment, clamped to +-2^30 (so every coordinate
// difference fits 31 bits); false for a non-finite query point.
__device__ __forceinline__ bool query_voxel(const NnSeg& sg, uint32_t j, int& qx, int& qy,
                                            int& qz) {
  if (sg.qv != nullptr) {
    const int* v = sg.qv + 3 * (size_t)j;
    qx = min(max(__ldg(v), -kQueryLimit), kQueryLimit);
    qy = min(max(__ldg(v + 1), -kQueryLimit), kQueryLimit);
    qz = min(max(__ldg(v + 2), -kQueryLimit), kQueryLimit);
    return true;
  }
  // queries stream through once: loaded evict-first, so that L2 keeps the
  // CGA and the search structures
  const float* p = sg.q + 3 * (size_t)j;
  const float px = __ldcs(p), py = __ldcs(p + 1), pz = __ldcs(p + 2);
  const bool valid = isfinite(px) && isfinite(py) && isfinite(pz);
  qx = valid ? (int)quantize_query(px, sg.scale, sg.off[0]) : 0;
  qy = valid ? (int)quantize_query(py, sg.scale, sg.off[1]) : 0;
  qz = valid ? (int)quantize_query(pz, sg.scale, sg.off[2]) : 0;
  return valid;
}

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
    const uint32_t xi = (uint32_t)(gr ? r : l);
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
// child first, by a group of G lanes per query (32 / G queries per warp).
// Lane g of a group owns the children numbered [g * 64/G, (g + 1) * 64/G)
// of every node (tree_child numbers, so the children of a planar patch of
// surface spread evenly over the lanes).  Each step the lanes bound their
// children still to visit (box distance of the child's occupied voxels),
// drop every child whose bound exceeds the best distance so far, and the
// group enters the surviving child with the least bound.  Children of a
// level-2 node are bricks: until a first candidate exists the nearest brick
// is examined alone (its voxels give a bound that prunes its siblings), after
// that every surviving brick at once, and the node is done.  A child is
// dropped only when its bound exceeds the best distance, and the best
// distance never falls below the final one, so every cell holding a voxel at
// the final distance is entered: the result is Eq. 8's nearest voxel, ties to
// the smaller key.

// Minimum of a D value over the lanes in gm (64-bit: high word first).
__device__ __forceinline__ uint32_t group_min(uint32_t gm, uint32_t v) {
  return __reduce_min_sync(gm, v);
}
__device__ __forceinline__ unsigned long long group_min(uint32_t gm, unsigned long long v) {
  const uint32_t vh = (uint32_t)(v >> 32), vl = (uint32_t)v;
  const uint32_t mh = __reduce_min_sync(gm, vh);
  const uint32_t ml = __reduce_min_sync(gm, vh == mh ? vl : 0xffffffffu);
  return ((unsigned long long)mh << 32) | ml;
}

// The best (distance^2, key) of the tree search, the same in every lane of
// the group.
template <typename D>
struct BestKey {
  D d2;
  unsigned long long key;
  // Merge the lanes' candidates (d, k): lexicographic minimum over the group
  // with the current best.
  __device__ __forceinline__ void merge(uint32_t gm, D d, unsigned long long k) {
    const bool better = d < d2 || (d == d2 && k < key);
    if (!__any_sync(gm, better)) return;
    if (!better) {
      d = d2;
      k = key;
    }
    const D md = group_min(gm, d);
    const bool at = d == md;
    const uint32_t kh = __reduce_min_sync(gm, at ? (uint32_t)(k >> 32) : 0xffffffffu);
    const uint32_t kl =
        __reduce_min_sync(gm, at && (uint32_t)(k >> 32) == kh ? (uint32_t)k : 0xffffffffu);
    d2 = md;
    key = ((unsigned long long)kh << 32) | kl;
  }
};

// Bound of a child from its box in the parent's frame (TreeView::pcode):
// (tx, ty, tz) is the query's offset from the parent's origin, ub = 1 - 2^ss
// and 2^ss voxels the box unit.  Along an axis the distance to [L u, (H + 1) u - 1]
// is max(L u - t, t + ub - H u, 0).
template <typename D>
__device__ __forceinline__ D parent_frame_lb(uint2 c, int tx, int ty, int tz, int ub, uint32_t ss) {
  const int lx = (int)((c.x & 63u) << ss), hx = (int)(((c.x >> 6) & 63u) << ss);
  const int ly = (int)(((c.x >> 12) & 63u) << ss), hy = (int)(((c.x >> 18) & 63u) << ss);
  const int lz = (int)((c.y & 63u) << ss), hz = (int)(((c.y >> 6) & 63u) << ss);
  const D dx = (uint32_t)max(max(lx - tx, tx + ub - hx), 0);
  const D dy = (uint32_t)max(max(ly - ty, ty + ub - hy), 0);
  const D dz = (uint32_t)max(max(lz - tz, tz + ub - hz), 0);
  return dx * dx + dy * dy + dz * dz;
}

// The smallest (distance^2, key) among the voxels of set m (tree_child
// numbers) of the brick at voxel origin (bx, by, bz), merged into (cd, ck).
template <typename D>
__device__ __forceinline__ void brick_voxels(unsigned long long m, uint32_t bx, uint32_t by,
                                             uint32_t bz, const Qry& q, uint32_t b, D& cd,
                                             unsigned long long& ck) {
  while (m != 0ull) {
    const uint32_t v = (uint32_t)__ffsll((long long)m) - 1u;
    m &= m - 1ull;
    uint32_t vx, vy, vz;
    tree_cell(v, vx, vy, vz);
    const uint32_t x = bx + vx, y = by + vy, z = bz + vz;
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

// One brick examined by the whole group: lane g takes the voxels numbered
// [g * 64/G, (g + 1) * 64/G).
template <int G, typename D>
__device__ __forceinline__ void group_brick(uint32_t gm, uint32_t g, unsigned long long m,
                                            uint32_t bx, uint32_t by, uint32_t bz, const Qry& q,
                                            uint32_t b, BestKey<D>& best) {
  constexpr uint32_t NB = 64 / G;
  const unsigned long long own = (G == 1 ? ~0ull : ((1ull << NB) - 1ull)) << (g * NB);
  D cd = (D)~(D)0;
  unsigned long long ck = ~0ull;
  brick_voxels<D>(m & own, bx, by, bz, q, b, cd, ck);
  best.merge(gm, cd, ck);
}

// The search state of one lane: the current node (its cell, level and the
// lane's share of its children), and the same for each node on the path
// above it, in local memory (two words per frame).
template <int G, typename D>
struct TreeWalk {
  static constexpr uint32_t NB = 64 / G;
  unsigned long long stk[2 * kTreeMaxLevels];
  uint32_t base;  // tree index of the lane's first child
  uint32_t mine;  // the lane's children (bit k: child g * NB + k)
  uint32_t rem;   // those still to visit
  uint32_t ox, oy, oz, lvl;
  int depth;
  bool done;

  __device__ __forceinline__ void enter(const uint4& r, uint32_t g) {
    const unsigned long long m = r.x | ((unsigned long long)r.y << 32);
    mine = (uint32_t)(m >> (g * NB)) & (uint32_t)((1ull << NB) - 1ull);
    base = r.z + (uint32_t)__popcll(m & ((1ull << (g * NB)) - 1ull));
    rem = mine;
  }

  __device__ __forceinline__ void pop() {
    if (depth == 0) {
      done = true;
      return;
    }
    --depth;
    const unsigned long long f0 = stk[2 * depth], f1 = stk[2 * depth + 1];
    base = (uint32_t)f0;
    mine = (uint32_t)(f0 >> 32) & 0xFFFFu;
    rem = (uint32_t)(f0 >> 48);
    ox = (uint32_t)f1 & 0xFFFFu;
    oy = (uint32_t)(f1 >> 16) & 0xFFFFu;
    oz = (uint32_t)(f1 >> 32) & 0xFFFFu;
    lvl = (uint32_t)(f1 >> 48);
  }

  // One step of the descent (the group's lanes together).
  __device__ __forceinline__ void step(const TreeView& tv, const Qry& q, uint32_t b, uint32_t gm,
                                       uint32_t g, BestKey<D>& best) {
    // a stored voxel at distance 0 is the answer (voxels are unique)
    if (best.d2 == (D)0) {
      done = true;
      return;
    }
    const bool bricks = lvl == 2;
    const uint32_t cap = tv.cap[lvl - 1];
    const uint4* nd = tv.node[lvl - 1];
    const uint2* pc = tv.pcode[lvl - 1];
    const uint32_t OX = ox << 2, OY = oy << 2, OZ = oz << 2;
    // the query from the node's origin, and the same less the width of a box
    // unit (the children's boxes are in cells of 2^ss voxels from there)
    const uint32_t ss = bricks ? 0u : 2 * (lvl - 3);
    const int tx = q.x - (int)(ox << (2 * lvl)), ty = q.y - (int)(oy << (2 * lvl)),
              tz = q.z - (int)(oz << (2 * lvl));
    const int ub = 1 - (1 << ss);
    D mlb = (D)~(D)0;
    uint32_t mk = 0, mci = 0, surv = 0;
    for (uint32_t r = rem; r != 0u; r &= r - 1u) {
      const uint32_t k = (uint32_t)__ffs((int)r) - 1u;
      const uint32_t ci = base + (uint32_t)__popc(mine & ((1u << k) - 1u));
      if (ci >= cap) continue;
      const D lb = parent_frame_lb<D>(__ldg(pc + ci), tx, ty, tz, ub, ss);
      if (lb <= best.d2) {
        surv |= 1u << k;
        if (lb < mlb) {
          mlb = lb;
          mk = k;
          mci = ci;
        }
      }
    }
    if (__ballot_sync(gm, surv != 0u) == 0u) {
      pop();
      return;
    }
    // the surviving child with the least bound (the lowest lane on a tie)
    const D gmin = group_min(gm, mlb);
    const uint32_t ow = (uint32_t)__ffs((int)__ballot_sync(gm, surv != 0u && mlb == gmin)) - 1u;
    const uint32_t cs = __shfl_sync(gm, g * NB + mk, ow);
    const uint32_t csi = __shfl_sync(gm, mci, ow);
    rem = surv;
    if ((threadIdx.x & 31u) == ow) rem &= ~(1u << mk);
    uint32_t cx, cy, cz;
    tree_cell(cs, cx, cy, cz);
    const uint32_t nx = OX + cx, ny = OY + cy, nz = OZ + cz;
    if (bricks) {
      if (best.key == ~0ull) {
        // no stored voxel found yet: the nearest brick alone; the next step
        // bounds the node's other bricks against the distance it gives
        group_brick<G, D>(gm, g, __ldg(tv.brick + csi), nx << 2, ny << 2, nz << 2, q, b, best);
        return;
      }
      // every surviving brick, each lane its own, and the node is done
      D cd = (D)~(D)0;
      unsigned long long ck = ~0ull;
      for (uint32_t r = surv; r != 0u; r &= r - 1u) {
        const uint32_t k = (uint32_t)__ffs((int)r) - 1u;
        const uint32_t ci = base + (uint32_t)__popc(mine & ((1u << k) - 1u));
        uint32_t bx, by, bz;
        tree_cell(g * NB + k, bx, by, bz);
        brick_voxels<D>(__ldg(tv.brick + ci), (OX + bx) << 2, (OY + by) << 2, (OZ + bz) << 2, q,
                        b, cd, ck);
      }
      best.merge(gm, cd, ck);
      pop();
      return;
    }
    // the node's frame is kept only while a lane has children left to visit
    if (__any_sync(gm, rem != 0u)) {
      stk[2 * depth] = base | ((unsigned long long)mine << 32) | ((unsigned long long)rem << 48);
      stk[2 * depth + 1] = ox | ((unsigned long long)oy << 16) | ((unsigned long long)oz << 32) |
                           ((unsigned long long)lvl << 48);
      ++depth;
    }
    enter(__ldg(nd + csi), g);
    --lvl;
    ox = nx;
    oy = ny;
    oz = nz;
  }
};

// CGA index of the stored voxel with key `key` (the Sec. V-A lookup: x
// directory or X_index, the slab's Y range, the column's Z range).
__device__ __forceinline__ uint32_t stored_index(const NnSeg& sg, unsigned long long key) {
  const Levels& a = sg.a;
  const uint32_t b = a.bits, mk = (1u << b) - 1u;
  const uint32_t x = (uint32_t)(key >> (2 * b)), y = (uint32_t)(key >> b) & mk,
                 z = (uint32_t)key & mk;
  const uint32_t h = (uint32_t)a.hdr->cnt[2];
  const uint32_t slab = sg.xdir != nullptr ? __ldg(sg.xdir + x) : lower_bound_u16(a.idx2, 0, h, x);
  const uint32_t c = lower_bound_u16(a.idx1, __ldg(a.ptr2 + slab), __ldg(a.ptr2 + slab + 1), y);
  return lower_bound_u16(a.idx0, __ldg(a.ptr1 + c), __ldg(a.ptr1 + c + 1), z);
}

// The whole descent.  The loop runs while any group of the warp is still
// searching (a warp vote each step), so the warp's lanes re-converge at
// every step.  `best` may start from an upper bound without a voxel (key all
// ones): every voxel at or below the bound is still examined.
template <int G, typename D>
__device__ void search_tree(const TreeView& tv, const Qry& q, uint32_t b, bool active,
                            uint32_t gm, uint32_t g, BestKey<D>& best) {
  TreeWalk<G, D> w;
  w.done = true;
  if (active) {
    if (tv.levels == 1) {
      group_brick<G, D>(gm, g, __ldg(tv.brick), 0u, 0u, 0u, q, b, best);
    } else {
      w.lvl = tv.levels;
      w.ox = w.oy = w.oz = 0;
      w.depth = 0;
      w.done = false;
      w.enter(__ldg(tv.node[tv.levels]), g);
    }
  }
  while (__any_sync(0xffffffffu, !w.done)) {
    if (!w.done) w.step(tv, q, b, gm, g, best);
  }
}

// Slots of the Morton order taken by one pass of a sorted search: every
// stride-th slot that is not a multiple of `parent` (parent 0: every
// stride-th slot).  The passes of a sorted search run with strides
// CGA_NN_SEED_TOP, CGA_NN_SEED_MID (if not 0) and 1, each seeded from the
// slots of the one before.
#ifndef CGA_NN_SEED_TOP
#define CGA_NN_SEED_TOP 32
#endif
#ifndef CGA_NN_SEED_MID
#define CGA_NN_SEED_MID 0
#endif
static_assert(kTile % CGA_NN_SEED_TOP == 0 && CGA_NN_SEED_TOP % (CGA_NN_SEED_MID ? CGA_NN_SEED_MID : 1) == 0,
              "seed groups nest and lie in one tile");

__device__ __forceinline__ uint32_t pass_count(uint32_t total, uint32_t stride, uint32_t parent) {
  return parent == 0 ? total / stride : total / stride - total / parent;
}

__device__ __forceinline__ uint32_t pass_slot(uint32_t i, uint32_t stride, uint32_t parent) {
  if (parent == 0) return i * stride;
  const uint32_t r = parent / stride - 1;  // slots of the pass per parent group
  return (i / r) * parent + (i % r + 1) * stride;
}

// Upper bound on the squared distance from query voxel q to the answer of
// query voxel q0 (squared distance d0 from q0): (sqrt(d0) + |q - q0|)^2 by the
// triangle inequality, in single precision (correctly rounded square roots,
// each step off by at most a few units in the last place) enlarged by a
// relative 1e-4 and 16 so that it stays above the exact value; all ones when
// it does not fit.
__device__ __forceinline__ unsigned long long seed_bound(unsigned long long d0, int qx, int qy,
                                                         int qz, int px, int py, int pz) {
  const float dx = (float)qx - (float)px, dy = (float)qy - (float)py, dz = (float)qz - (float)pz;
  const float r = (__fsqrt_ru((float)d0) + __fsqrt_ru(dx * dx + dy * dy + dz * dz)) * 1.0001f;
  const float bnd = r * r + 16.0f;
  return bnd < 1.8e19f ? (unsigned long long)bnd : ~0ull;
}

// The seed of slot `slot` (query voxel q) in a pass with seed groups of
// `parent` slots: the tighter of the bounds that the answers of the slot's
// own group head and of the next group's head give (all ones: none).
__device__ __forceinline__ unsigned long long seed_of(const NnSeg& sg, uint32_t slot,
                                                      uint32_t parent, bool sorted,
                                                      const unsigned long long* order, int qx,
                                                      int qy, int qz) {
  unsigned long long seed = ~0ull;
  const uint32_t h0 = slot - slot % parent;
#pragma unroll
  for (uint32_t e = 0; e < 2; ++e) {
    const uint32_t s0 = h0 + e * parent, l0 = s0 - sg.tile_base * (uint32_t)kTile;
    if (l0 >= sg.m) continue;  // (beyond the segment's queries)
    const uint32_t j0 = sorted ? (uint32_t)__ldg(order + s0) : l0;
    if (j0 >= sg.m) continue;
    const unsigned long long d0 = __ldg(sg.d2 + j0);
    int px, py, pz;
    if (d0 != ~0ull && query_voxel(sg, j0, px, py, pz)) {
      seed = min(seed, seed_bound(d0, qx, qy, qz, px, py, pz));
    }
  }
  return seed;
}

// G lanes per query slot over every segment with a tree (a segment without
// one is left to k_nn_warp).  A warp takes 32 / G consecutive slots of the
// pass at a time (neighbouring queries in Morton order) and moves on when all
// are answered; the loop is warp-uniform, so that the descent's warp votes
// see every lane.  The pass takes the slots pass_slot gives; with parent > 0
// each search starts from the bound that the answer of the slot's parent
// group head (found by an earlier pass) gives: a bound without a voxel, so
// the result is the same.
template <int G>
__global__ void __launch_bounds__(256, CGA_NN_TREE_BLOCKS)
    k_nn_tree(const NnSeg* __restrict__ segs, int S, NnSeg inline_seg, uint32_t total_slots,
              const unsigned long long* __restrict__ order,
              const unsigned int* __restrict__ order_err, uint32_t stride, uint32_t parent) {
  constexpr uint32_t QW = 32 / G;
  const bool sorted = order != nullptr && (order_err == nullptr || *order_err == 0u);
  const uint32_t lane = threadIdx.x & 31, g = lane % G;
  const uint32_t gm = G == 32 ? 0xffffffffu : (uint32_t)((1ull << G) - 1ull) << (lane - g);
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t n_pass = pass_count(total_slots, stride, parent);
  for (uint32_t base = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * QW; base < n_pass;
       base += nwarps * QW) {
    const uint32_t i = base + lane / G;
    bool active = i < n_pass;
    const uint32_t slot = pass_slot(active ? i : base, stride, parent);
    const NnSeg& sg = segs != nullptr ? segs[find_nn_seg(segs, S, slot / (uint32_t)kTile)]
                                      : inline_seg;
    const uint32_t local = slot - sg.tile_base * (uint32_t)kTile;
    active = active && sg.tree.levels > 0 && local < sg.m;
    const uint32_t j = active ? (sorted ? (uint32_t)__ldcs(order + slot) : local) : 0u;
    active = active && j < sg.m;
    int qx = 0, qy = 0, qz = 0;
    if (active) {
      const bool valid = query_voxel(sg, j, qx, qy, qz);
      if (!valid || sg.a.hdr->cnt[0] == 0) {
        if (g == 0) {
          __stcs(sg.idx + j, 0xffffffffu);
          __stcs(sg.d2 + j, ~0ull);
        }
        active = false;
      }
    }
    const unsigned long long seed =
        parent != 0 && active ? seed_of(sg, slot, parent, sorted, order, qx, qy, qz) : ~0ull;
    const uint32_t b = sg.a.bits;
    const int top = (1 << b) - 1;
    const uint32_t cqx = (uint32_t)min(max(qx, 0), top);
    const uint32_t cqy = (uint32_t)min(max(qy, 0), top);
    const uint32_t cqz = (uint32_t)min(max(qz, 0), top);
    const Qry qq{qx, qy, qz, cqx, cqy, cqz};
    unsigned long long d2 = ~0ull, key = ~0ull;
    const bool narrow = b <= 15 && (uint32_t)qx == cqx && (uint32_t)qy == cqy &&
                        (uint32_t)qz == cqz;
    if (__all_sync(0xffffffffu, narrow || !active)) {
      BestKey<uint32_t> best{seed < 0xffffffffull ? (uint32_t)seed : 0xffffffffu, ~0ull};
      search_tree<G, uint32_t>(sg.tree, qq, b, active, gm, g, best);
      // (a seeded search always meets the group's first answer; searched
      // again without the seed should it not)
      const bool again = active && best.key == ~0ull && seed != ~0ull;
      if (__any_sync(0xffffffffu, again)) {
        if (again) best = BestKey<uint32_t>{0xffffffffu, ~0ull};
        search_tree<G, uint32_t>(sg.tree, qq, b, again, gm, g, best);
      }
      if (best.key != ~0ull) {
        d2 = best.d2;
        key = best.key;
      }
    } else {
      BestKey<unsigned long long> best{seed, ~0ull};
      search_tree<G, unsigned long long>(sg.tree, qq, b, active, gm, g, best);
      const bool again = active && best.key == ~0ull && seed != ~0ull;
      if (__any_sync(0xffffffffu, again)) {
        if (again) best = BestKey<unsigned long long>{~0ull, ~0ull};
        search_tree<G, unsigned long long>(sg.tree, qq, b, again, gm, g, best);
      }
      if (best.key != ~0ull) {
        d2 = best.d2;
        key = best.key;
      }
    }
    if (active && g == 0) {
      __stcs(sg.idx + j, d2 != ~0ull ? stored_index(sg, key) : 0xffffffffu);
      __stcs(sg.d2 + j, d2);
    }
  }
}

// NC: the most coarse levels any segment of the launch carries (0, 1 or 2).
// The fine-only instantiation is held to 40 registers (six blocks per SM),
// the coarse ones to 48 (five blocks per SM): the extra warps hide more of
// the search's load latency than the spilled values cost (eight and six
// blocks respectively spill enough to be slower).
template <int NC>
__global__ void __launch_bounds__(256, NC > 0 ? CGA_NN_COARSE_BLOCKS : CGA_NN_FINE_BLOCKS)
    k_nn_warp(const NnSeg* __restrict__ segs, int S, NnSeg inline_seg, uint32_t total_slots,
              const unsigned long long* __restrict__ order,
              const unsigned int* __restrict__ order_err) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  const bool sorted = order != nullptr && (order_err == nullptr || *order_err == 0u);
  for (uint32_t slot = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; slot < total_slots;
       slot += nwarps) {
    const uint32_t tile = slot / (uint32_t)kTile;
    const NnSeg& sg = segs != nullptr ? segs[find_nn_seg(segs, S, tile)] : inline_seg;
    if (sg.tree.levels > 0) continue;  // searched by k_nn_tree
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
    const bool valid = query_voxel(sg, j, qx, qy, qz);
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
    Best best{~0ull, 0xffffffffu};
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

// Blocks of a search kernel that fit on one SM (queried once per kernel:
// 0-2 k_nn_warp of that many coarse levels, 3 k_nn_tree).
static uint32_t resident_blocks(uint32_t kind) {
  static std::atomic<int> cache[4] = {{0}, {0}, {0}, {0}};
  int n = cache[kind].load(std::memory_order_relaxed);
  if (n == 0) {
    cudaError_t e = cudaErrorInvalidValue;
    if (kind == 0) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_nn_warp<0>, 256, 0);
    if (kind == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_nn_warp<1>, 256, 0);
    if (kind == 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_nn_warp<2>, 256, 0);
    if (kind == 3) {
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_nn_tree<CGA_NN_TREE_GROUP>, 256, 0);
    }
    if (e != cudaSuccess || n <= 0) {
      cudaGetLastError();
      n = 4;
    }
    cache[kind].store(n, std::memory_order_relaxed);
  }
  return (uint32_t)n;
}

// kinds: bit k set when some segment of the launch has nn_kind k.  Segments
// with a tree go to k_nn_tree, the others to k_nn_warp of their largest kind.
// Each kernel runs one wave of resident blocks striding over the query slots
// (a second wave would only add its own tail).
static void launch_search(const NnSeg* d_segs, int S, const NnSeg& inline_seg,
                          uint32_t total_tiles, const unsigned long long* order,
                          const unsigned int* order_err, uint32_t kinds,
                          cudaStream_t stream) {
  const uint32_t total_slots = total_tiles * (uint32_t)kTile;
  const uint32_t sms = (uint32_t)device_sm_count();
  if (kinds & 8u) {
    // in Morton order: every CGA_NN_SEED_TOP-th query, then (seeded by those)
    // every CGA_NN_SEED_MID-th, then the rest; in query order one pass
    // (neighbouring slots are not close queries)
    constexpr uint32_t qpb = 256 / CGA_NN_TREE_GROUP;  // queries per block and round
    const uint32_t cap_blocks = sms * resident_blocks(3);
    uint32_t pstride[3], pparent[3];
    int np = 0;
    if (order != nullptr) {
      pstride[np] = CGA_NN_SEED_TOP;
      pparent[np++] = 0;
      if (CGA_NN_SEED_MID > 1) {
        pstride[np] = CGA_NN_SEED_MID;
        pparent[np++] = CGA_NN_SEED_TOP;
      }
      pstride[np] = 1;
      pparent[np++] = CGA_NN_SEED_MID > 1 ? CGA_NN_SEED_MID : CGA_NN_SEED_TOP;
    } else {
      pstride[np] = 1;
      pparent[np++] = 0;
    }
    for (int k = 0; k < np; ++k) {
      const uint32_t n = pparent[k] == 0 ? total_slots / pstride[k]
                                         : total_slots / pstride[k] - total_slots / pparent[k];
#if CGA_NN_HEAD_GROUP
      if (np > 1 && k == 0) {
        constexpr uint32_t hq = 256 / CGA_NN_HEAD_GROUP;
        k_nn_tree<CGA_NN_HEAD_GROUP><<<std::min<uint32_t>((n + hq - 1) / hq, cap_blocks), 256, 0,
                                       stream>>>(d_segs, S, inline_seg, total_slots, order,
                                                 order_err, pstride[k], pparent[k]);
        count_launch(1);
        continue;
      }
#endif
      const uint32_t blocks = std::min<uint32_t>((n + qpb - 1) / qpb, cap_blocks);
      k_nn_tree<CGA_NN_TREE_GROUP><<<blocks, 256, 0, stream>>>(d_segs, S, inline_seg,
                                                               total_slots, order, order_err,
                                                               pstride[k], pparent[k]);
      count_launch(1);
    }
  }
  kinds &= 7u;
  if (kinds == 0) return;
  const uint32_t kind = kinds >= 4u ? 2u : (kinds >= 2u ? 1u : 0u);
  const uint32_t blocks = std::min<uint32_t>((total_slots + 7) / 8, sms * resident_blocks(kind));
  if (kind == 2) {
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
  k_nn_keys<<<total_tiles, 256, 0, stream>>>(
      t.segs, S, static_cast<unsigned long long*>(t.sort.keys0), t.sort.hist);
  count_launch(1);
  return run_radix_passes(S, total_tiles, 4, true, t.sort, stream);
}

cudaError_t run_nn_search(const NnSeg& seg, const unsigned long long* order, cudaStream_t stream) {
  if (seg.m == 0) return cudaSuccess;
  launch_search(nullptr, 1, seg, seg.num_tiles, order, nullptr, 1u << nn_kind(seg), stream);
  return cudaGetLastError();
}

cudaError_t run_nn_device(int S, uint32_t total_tiles, const NnTables& t, cudaStream_t stream,
                          uint32_t kinds) {
  if (total_tiles == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(t.err, 0, sizeof(Header), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(t.sort.hist, 0, t.sort.zero_bytes, stream);
  if (e != cudaSuccess) return e;
  k_nn_keys<<<total_tiles, 256, 0, stream>>>(
      t.segs, S, static_cast<unsigned long long*>(t.sort.keys0), t.sort.hist);
  count_launch(1);
  e = run_radix_passes(S, total_tiles, 4, true, t.sort, stream);
  if (e != cudaSuccess) return e;
  // four passes leave the sorted keys in keys0
  launch_search(t.segs, S, NnSeg{}, total_tiles,
                static_cast<const unsigned long long*>(t.sort.keys0), &t.err->err, kinds, stream);
  return cudaGetLastError();
}

cudaError_t run_nn(const NnSeg* h_segs, int S, uint32_t total_tiles, void* scratch,
                   cudaStream_t stream) {
  if (total_tiles == 0) return cudaSuccess;
  if (scratch == nullptr) {
    if (S != 1) return cudaErrorInvalidValue;
    launch_search(nullptr, 1, h_segs[0], total_tiles, nullptr, nullptr, 1u << nn_kind(h_segs[0]),
                  stream);
    return cudaGetLastError();
  }
  const NnTables t = nn_tables(scratch, total_tiles, S);
  const cudaError_t e = nn_upload(h_segs, S, t, stream);
  if (e != cudaSuccess) return e;
  uint32_t kinds = 0;
  for (int s = 0; s < S; ++s) kinds |= 1u << nn_kind(h_segs[s]);
  return run_nn_device(S, total_tiles, t, stream, kinds);
}

}  // namespace libcga
